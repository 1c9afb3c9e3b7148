"""ddm_scan_counts_noalloc against the offsets of ddm_plan (GPU).

The allocation-free scan is for callers that cannot allocate device memory
when they need the offsets (for example while a stream is being captured
into a CUDA graph).  It must give exactly the offsets that ddm_plan gives
for the same per-update counts, call after call, although its scratch array
is shared and keeps the previous call's contents.  This file is collected
last so that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


def test_noalloc_scan_equals_plan_offsets_on_consecutive_calls(ctx):
    import torch
    # two calls in a row; the second has fewer tiles than the first, so
    # stale tile sums from the first call sit in the shared array
    for name, scale in (("uniform_d2_N1e6_a100", 0.2), ("clustered_d3_N1e7_a100", 0.01)):
        arrays = W.make(name, scale)
        U = tuple(torch.from_numpy(a).cuda() for a in arrays)
        ddm.ddm_build(ctx, U[2], U[3])
        m = U[0].shape[1]
        ref = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        K = ddm.ddm_plan(ctx, U[0], U[1], offsets=ref)
        counts = (ref[1:] - ref[:-1]).to(torch.int32)
        out = torch.full((m + 1,), -1, dtype=torch.int64, device="cuda")
        ddm.ddm_scan_counts_noalloc(counts, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert int(out[-1]) == K > 0


def test_noalloc_scan_rejects_oversized_input():
    import torch
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = ddm.lib().ddm_scan_counts_noalloc(buf.data_ptr(), ddm.DDM_NOALLOC_MAX_UPDATES + 1,
                                           buf.data_ptr(), None)
    assert rc == ddm.DDM_ERR_ARG
    assert ddm.lib().ddm_scan_counts_noalloc(None, 4, buf.data_ptr(), None) == ddm.DDM_ERR_ARG
    # empty input: offsets[0] = 0
    buf.fill_(7)
    assert ddm.lib().ddm_scan_counts_noalloc(None, 0, buf.data_ptr(), None) == ddm.DDM_OK
    torch.cuda.synchronize()
    assert int(buf[0]) == 0 and int(buf[1]) == 7
