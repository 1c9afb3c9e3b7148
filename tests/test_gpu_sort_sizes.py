"""Sort sizes around the kernels' thresholds (GPU).

The radix sort takes one of several forms by size: one thread-block
cluster for up to 16 x 2,048 keys, one cooperative launch with tiles of
2,048, 4,096 or 8,192 keys while every tile can be resident (up to
1,245,184 keys on a 152-SM GB300), the multi-launch onesweep beyond (and one
CTA for up to 8,192 keys under stream capture).  For d = 1
both orders are fixed exactly: the tree order is the lexicographic order of
(lower bound, upper bound, id) under the IEEE total order with -0 = +0
(Section IV's sort by lower bound, ties as the stable passes leave them),
and the updates' plan order is the stable order of the top 24 bits of the
lower bound's key.  Both are compared with numpy's stable sorts at sizes on
each side of every threshold, with ties in every digit.  The plan's offsets
(the multi-job scan) are compared with a host prefix sum of the counts.
"""
import numpy as np
import pytest

import paper_1309_3458_gb300 as ddm
from tests.helpers import to_dev
from tests.test_gpu_parity import order_key

pytestmark = pytest.mark.gpu

SIZES = [2, 33, 2048, 2049, 4097, 8192, 8193, 16385, 32768, 32769, 100_003, 311_296, 311_297,
         1_245_184, 1_245_185, 1_500_000]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


def tied_set(n, seed):
    """d = 1 extents on a coarse grid (ties in whole keys and in single
    digits), a few signed zeros and infinities, random ids."""
    rng = np.random.default_rng(seed)
    lo = rng.integers(-300, 300, size=n).astype(np.float32) * np.float32(0.25)
    w = rng.integers(0, 40, size=n).astype(np.float32) * np.float32(0.5)
    hi = lo + w
    lo[:3] = -0.0
    lo[3:5] = -np.inf
    hi[5:7] = np.inf
    big = rng.random(n) < 0.1   # keys that differ in the low digits only
    lo[big] = np.float32(1e6) + rng.integers(0, 2048, size=int(big.sum())).astype(np.float32)
    hi[big] = lo[big] + np.float32(1.0)
    hi = np.maximum(hi, lo)
    return lo[None, :].copy(), hi[None, :].copy()


@pytest.mark.parametrize("n", SIZES)
def test_tree_order_exact(ctx, n):
    import torch
    lo, hi = tied_set(n, seed=n)
    S = to_dev((lo, hi))
    ddm.ddm_build(ctx, S[0], S[1])
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    _, _, total = ddm.ddm_tree_shape(ctx)
    nlo = torch.empty(total, dtype=torch.float32, device="cuda")
    nhi = torch.empty(total, dtype=torch.float32, device="cuda")
    ddm.ddm_tree_export(ctx, order, nlo, nhi)
    got = order.cpu().numpy().view(np.uint32)
    want = np.lexsort((np.arange(n), order_key(hi[0]), order_key(lo[0]))).astype(np.uint32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("m", SIZES)
def test_plan_order_and_offsets_exact(ctx, m):
    import torch
    slo, shi = tied_set(200, seed=1)
    ulo, uhi = tied_set(m, seed=m + 1)
    S = to_dev((slo, shi))
    U = to_dev((ulo, uhi))
    ddm.ddm_build(ctx, S[0], S[1])
    K = ddm.ddm_plan(ctx, U[0], U[1])
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    offs = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    ddm.ddm_plan_order(ctx, order, offs)
    got = order.cpu().numpy().view(np.uint32)
    want = np.argsort(order_key(ulo[0]) >> np.uint32(8), kind="stable").astype(np.uint32)
    assert np.array_equal(got, want)
    # per-position counts from a brute-force 1-D test on a sample, and the
    # offsets as a prefix sum of the per-position counts
    po = offs.cpu().numpy()
    cnt = np.diff(po)
    assert po[0] == 0 and po[-1] == K and (cnt >= 0).all()
    rng = np.random.default_rng(m)
    for p in rng.choice(m, size=min(200, m), replace=False):
        u = got[p]
        meet = (slo[0] <= uhi[0, u]) & (ulo[0, u] <= shi[0])
        assert cnt[p] == int(meet.sum())
