"""Runs with DDM_LIBRARY=checked (the bounds-checking build): every call must
succeed -- no kernel found an index out of bounds (DDM_ERR_INTERNAL) -- and
give the oracle's pairs.  Started in its own process by test_gpu_checked.py,
so that only the checked library is loaded in it."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_1309_3458_gb300 as ddm  # noqa: E402
from paper_1309_3458_gb300 import workloads as W  # noqa: E402
from tests.helpers import gpu_match, keys, to_dev  # noqa: E402


def main():
    import torch
    assert ddm.LIB_PATH.endswith("libddm_checked.so"), ddm.LIB_PATH
    ctx = ddm.ddm_create(0)
    try:
        # one-shot matches, every leaf-test form, both rules
        for qpp, swap in ((32, 12), (32, 1), (16, 1), (32, 33)):
            ddm.ddm_set_tiling(ctx, qpp, swap)
            for d in (1, 2, 3, 5):
                for seed in range(3):
                    a = W.grid_random(150 + 40 * seed, 200, d, seed=seed, grid=5)
                    for flags in (0, 1):
                        K, pu, ps = gpu_match(ctx, a, flags)
                        Ko, ou, os_ = oracle.itm_pairs(*a, flags=flags)
                        assert K == Ko and np.array_equal(np.sort(keys(pu, ps)), np.sort(keys(ou, os_)))
        ddm.ddm_set_tiling(ctx, 32, 12)
        # staged, chunked: ordered pairs (32- and 64-bit positions), ids, by update id
        a = W.make("clustered_d3_N1e7_a100", 0.01)
        U = to_dev(a)
        ddm.ddm_build(ctx, U[2], U[3])
        K = ddm.ddm_plan(ctx, U[0], U[1])
        m = a[0].shape[1]
        got = []
        buf = torch.empty((K // 5 + 1, 2), dtype=torch.int32, device="cuda")
        b = 0
        while b < m:
            e = ddm.ddm_chunk_end_ordered(ctx, b, buf.shape[0])
            k = ddm.ddm_write_ordered(ctx, b, e, buf)
            got.append(buf[:k].cpu().numpy().copy())
            b = e
        p = np.concatenate(got).view(np.uint32)
        ids = torch.empty(K, dtype=torch.int32, device="cuda")
        assert ddm.ddm_write_ordered_ids(ctx, 0, m, ids) == K
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), p[:, 1])
        Ko, ou, os_ = oracle.itm_pairs(*a)
        assert K == Ko and np.array_equal(np.sort(keys(p[:, 0], p[:, 1])), np.sort(keys(ou, os_)))
        # batched instances
        inst = W.batched_instances(64, d=2, alpha=1.0, size_lo=100, size_hi=20_000, seed=3)
        ulo, uhi, uoff, slo, shi, soff = W.concat_instances(inst)
        B = to_dev((ulo, uhi, slo, shi))
        uo = torch.from_numpy(uoff.astype(np.int64)).cuda()
        so = torch.from_numpy(soff.astype(np.int64)).cuda()
        Kb = sum(oracle.itm_count(*x)[0] for x in inst)
        pb = torch.empty((Kb + 1, 2), dtype=torch.int32, device="cuda")
        assert ddm.ddm_batch_match(ctx, B[0], B[1], uo, B[2], B[3], so, pb) == Kb
        # refit after a move, then a plan against the refitted tree
        ddm.ddm_build(ctx, U[2], U[3])
        moved = (U[2] + 5.0).contiguous(), (U[3] + 5.0).contiguous()
        ddm.ddm_refit(ctx, *moved)
        Kr = ddm.ddm_plan(ctx, U[0], U[1])
        assert Kr == oracle.itm_count(a[0], a[1], a[2] + np.float32(5.0), a[3] + np.float32(5.0))[0]
    finally:
        ddm.ddm_destroy(ctx)
    print("checked build ok")


if __name__ == "__main__":
    main()
