"""ddm_scan_counts_noalloc: the allocation-free offsets scan (GPU).

The entry point is for callers that cannot allocate device memory when they
need the offsets: a real-time loop that must not block in the allocator, or
a host whose device memory all belongs to another pool.  Its scratch is one
array inside the library, shared by every call and keeping the last call's
contents, so the checks below make calls in a row, from large to small and
back, and compare each against an independent host prefix sum (and, on real
plans, against the offsets ddm_plan computes).  This file is collected last
so that a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILE = 4096  # counts per scan tile


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


def host_offsets(counts_u32: np.ndarray) -> np.ndarray:
    """Exclusive prefix sum in uint64 (counts are uint32)."""
    out = np.zeros(counts_u32.shape[0] + 1, dtype=np.uint64)
    np.cumsum(counts_u32, dtype=np.uint64, out=out[1:])
    return out


def scan_on_gpu(counts_u32: np.ndarray) -> np.ndarray:
    import torch
    m = counts_u32.shape[0]
    c = torch.from_numpy(counts_u32.view(np.int32)).cuda()
    out = torch.full((m + 1,), -1, dtype=torch.int64, device="cuda")
    ddm.ddm_scan_counts_noalloc(c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


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
        host = host_offsets(counts.cpu().numpy().view(np.uint32))
        assert np.array_equal(out.cpu().numpy().view(np.uint64), host)


def test_noalloc_scan_sizes_against_host_prefix_sum(ctx):
    """Full-range uint32 counts (64-bit carries in every tile) at the limit,
    above 2^24, at whole tiles and inside one tile, one call after another."""
    rng = np.random.default_rng(7)
    sizes = [ddm.DDM_NOALLOC_MAX_UPDATES,      # 16,384 tiles: the single-CTA scan of all tile sums
             3 * TILE,                          # whole tiles, stale sums of the call before
             1000,                              # part of one tile
             TILE,                              # exactly one tile
             (1 << 24) + 5,                     # ragged last tile
             ddm.DDM_NOALLOC_MAX_UPDATES]       # the limit again, after smaller calls
    for m in sizes:
        counts = rng.integers(0, 1 << 32, size=m, dtype=np.uint32)
        got = scan_on_gpu(counts)
        want = host_offsets(counts)
        assert np.array_equal(got, want), m
    # small counts too (the offsets of a real plan), twice in a row
    for _ in range(2):
        counts = rng.integers(0, 50, size=5 * TILE + 17, dtype=np.uint32)
        assert np.array_equal(scan_on_gpu(counts), host_offsets(counts))


def test_noalloc_scan_limits_and_null_pointers(ctx):
    import torch
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    # one past the limit: refused by the binding and by the library itself
    with pytest.raises(ValueError):
        ddm.ddm_scan_counts_noalloc(
            torch.zeros(ddm.DDM_NOALLOC_MAX_UPDATES + 1, dtype=torch.int32, device="cuda"),
            torch.zeros(ddm.DDM_NOALLOC_MAX_UPDATES + 2, dtype=torch.int64, device="cuda"))
    rc = ddm.lib().ddm_scan_counts_noalloc(buf.data_ptr(), ddm.DDM_NOALLOC_MAX_UPDATES + 1,
                                           buf.data_ptr(), None)
    assert rc == ddm.DDM_ERR_ARG
    # NULL counts with m > 0, NULL offsets: refused
    assert ddm.lib().ddm_scan_counts_noalloc(None, 4, buf.data_ptr(), None) == ddm.DDM_ERR_ARG
    assert ddm.lib().ddm_scan_counts_noalloc(buf.data_ptr(), 4, None, None) == ddm.DDM_ERR_ARG
    # m == 0: counts may be NULL (as the header states); offsets[0] = 0, nothing else written
    buf.fill_(7)
    assert ddm.lib().ddm_scan_counts_noalloc(None, 0, buf.data_ptr(), None) == ddm.DDM_OK
    torch.cuda.synchronize()
    assert int(buf[0]) == 0 and int(buf[1]) == 7
