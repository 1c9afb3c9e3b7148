"""Dynamic interval management (Section IV): after extents move, the rows
(moved updates) and columns (moved subscriptions) recomputed by one query
against the other set's tree are exactly those of a fresh match of the new
coordinates, and the refitted or rebuilt trees still give the full pair set."""
import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W
from paper_1309_3458_gb300.dynamic import DynamicMatching
from tests.helpers import keys, to_dev

pytestmark = pytest.mark.gpu


def fresh_pairs(ctx, U, flags=0):
    import torch
    K = ddm.ddm_count(ctx, *U, flags=flags)
    buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    ddm.ddm_match(ctx, *U, buf, flags=flags)
    return buf[:K].cpu().numpy().view(np.uint32).copy()


@pytest.mark.parametrize("d,flags", [(1, 0), (2, 0), (3, 0), (2, 1)])
def test_moved_rows_and_columns(d, flags):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(d)
    a = W.uniform_fixed_length(6000, 5000, d, 30.0, seed=d)
    U = to_dev(a)
    dm = DynamicMatching(*U, flags=flags, rebuild_every=3)
    ctx = ddm.ddm_create(0)
    buf = torch.empty((1 << 22, 2), dtype=torch.int32, device="cuda")
    l = float(a[1][0, 0] - a[0][0, 0])
    try:
        for step in range(6):
            kind = step % 2
            total = 5000 if kind == 0 else 6000
            k = int(rng.integers(1, 400))
            ids_np = rng.choice(total, size=k, replace=False).astype(np.int32)
            lo_np = rng.uniform(0, W.ROUTING_L - l, size=(d, k)).astype(np.float32)
            hi_np = (lo_np + np.float32(l)).astype(np.float32)
            if step == 3:   # a few degenerate and touching extents
                hi_np[:, :3] = lo_np[:, :3]
            ids = torch.from_numpy(ids_np).cuda()
            lo, hi = torch.from_numpy(lo_np).cuda(), torch.from_numpy(hi_np).cuda()
            if kind == 0:
                K = dm.move_updates(ids, lo, hi, buf)
            else:
                K = dm.move_subscriptions(ids, lo, hi, buf)
            got = buf[:K].cpu().numpy().view(np.uint32)
            full = fresh_pairs(ctx, dm.sets(), flags)
            col = 0 if kind == 0 else 1
            want = full[np.isin(full[:, col], ids_np.astype(np.uint32))]
            assert K == len(want)
            assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])),
                                  np.sort(keys(want[:, 0], want[:, 1])))
            # grouped by moved extent, in the order of ids
            order = {int(v): i for i, v in enumerate(ids_np)}
            g = np.array([order[int(v)] for v in got[:, col]])
            assert (np.diff(g) >= 0).all()
        # the refitted / rebuilt T_S still gives every pair of the moved sets
        K = dm.match_all(buf)
        got = buf[:K].cpu().numpy().view(np.uint32)
        host = [x.cpu().numpy() for x in dm.sets()]
        Ko, ou, os_ = oracle.itm_pairs(*host, flags=flags)
        assert K == Ko
        assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_)))
    finally:
        dm.close()
        ddm.ddm_destroy(ctx)


def test_match_moved_errors_and_ids():
    import torch
    ctx = ddm.ddm_create(0)
    try:
        lo = torch.zeros((2, 4), device="cuda")
        hi = torch.ones((2, 4), device="cuda")
        buf = torch.empty((64, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(ddm.DDMError) as e:   # no tree yet
            ddm.ddm_match_moved(ctx, lo, hi, None, buf)
        assert e.value.code == ddm.DDM_ERR_STATE
        ddm.ddm_build(ctx, lo, hi)
        K = ddm.ddm_match_moved(ctx, lo[:, :2].contiguous(), hi[:, :2].contiguous(), None, buf)
        assert K == 8
        p = buf[:K].cpu().numpy()
        assert sorted(set(p[:, 0].tolist())) == [0, 1]             # NULL ids: 0..k-1
        ids = torch.tensor([7, 9], dtype=torch.int32, device="cuda")
        K = ddm.ddm_match_moved(ctx, lo[:, :2].contiguous(), hi[:, :2].contiguous(), ids, buf,
                                flags=ddm.DDM_SWAP_ROLES)
        p = buf[:K].cpu().numpy()
        assert sorted(set(p[:, 1].tolist())) == [7, 9] and sorted(set(p[:, 0].tolist())) == [0, 1, 2, 3]
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_match_moved(ctx, lo, hi, None, buf[:3])
        assert e.value.code == ddm.DDM_ERR_CAPACITY and e.value.k == 16
        bad = hi.clone()
        bad[0, 1] = -5.0
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_match_moved(ctx, lo, bad, None, buf)
        assert e.value.code == ddm.DDM_ERR_EXTENT
    finally:
        ddm.ddm_destroy(ctx)
