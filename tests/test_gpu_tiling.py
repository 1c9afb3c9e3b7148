"""Tiling and tuning knobs change speed only (GPU).

Queries per packet (16 or 32), the swapped-loop threshold, the re-sort group
shift, the CTAs per SM and replay on or off: every combination the autotuner
may pick gives the pairs of the default setting on single problems (d = 1,
2, 3, both rules) and on batched instances -- element by element, except
that a re-sort group shift changes the tree order of d >= 2 and so the order
of an update's pairs (then the update column is identical and each update's
set is); the autotuner's choice on the batched workload is checked against
the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import autotune as AT
from paper_1309_3458_gb300 import workloads as W
from tests.helpers import keys, to_dev
from tests.test_gpu_batch import make_batch, run_batch

pytestmark = pytest.mark.gpu

SETTINGS = [dict(queries_per_packet=16), dict(queries_per_packet=16, swap_min=8),
            dict(swap_min=1), dict(swap_min=33), dict(queries_per_packet=16, swap_min=33),
            dict(str_shift=1, ctas_per_sm=4, queries_per_packet=16, swap_min=16),
            dict(replay=0, queries_per_packet=16, swap_min=12)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    AT.apply(h, {})
    ddm.ddm_destroy(h)


def same(got, ref, st):
    if st.get("str_shift", 0) == 0:
        return np.array_equal(got, ref)
    u = ref.view(np.uint32)
    g = got.view(np.uint32)
    return (np.array_equal(g[:, 0], u[:, 0]) and
            np.array_equal(np.sort(keys(g[:, 0], g[:, 1])), np.sort(keys(u[:, 0], u[:, 1]))))


def match(ctx, U, flags=0):
    import torch
    K = ddm.ddm_count(ctx, *U, flags=flags)
    pairs = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    assert ddm.ddm_match(ctx, *U, pairs, flags=flags) == K
    return pairs[:K].cpu().numpy().copy()


@pytest.mark.parametrize("name,scale,flags", [
    ("uniform_d1_N1e4_a1", 1.0, 0), ("uniform_d1_N1e6_a100", 0.1, 1),
    ("uniform_d2_N1e6_a100", 0.05, 0), ("clustered_d3_N1e7_a100", 0.01, 0),
    ("clustered_d3_N1e7_a100", 0.01, 1)])
def test_every_setting_gives_the_default_pairs(ctx, name, scale, flags):
    arrays = W.make(name, scale)
    U = to_dev(arrays)
    AT.apply(ctx, {})
    ref = match(ctx, U, flags)
    assert ref.shape[0] > 0
    for st in SETTINGS:
        AT.apply(ctx, st)
        assert same(match(ctx, U, flags), ref, st), st
    AT.apply(ctx, {})


def test_every_setting_on_uneven_batches(ctx):
    inst = make_batch(2, 300, seed=11)
    AT.apply(ctx, {})
    K, ref, po, _ = run_batch(ctx, inst)
    for st in SETTINGS:
        AT.apply(ctx, st)
        K2, p2, po2, _ = run_batch(ctx, inst)
        assert K2 == K and np.array_equal(po2, po) and same(p2, ref, st), st
    AT.apply(ctx, {})


def test_plan_dropped_when_packets_change(ctx):
    import torch
    arrays = W.make("uniform_d2_N1e6_a1", 0.01)
    U = to_dev(arrays)
    AT.apply(ctx, {})
    ddm.ddm_build(ctx, U[2], U[3])
    K = ddm.ddm_plan(ctx, U[0], U[1])
    buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    ddm.ddm_set_tiling(ctx, 32, 16)          # same packets: the plan stays
    assert ddm.ddm_write(ctx, 0, arrays[0].shape[1], buf) == K
    ddm.ddm_set_tiling(ctx, 16, 16)          # other packets: the records no longer apply
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_write(ctx, 0, arrays[0].shape[1], buf)
    assert e.value.code == ddm.DDM_ERR_STATE
    for bad in ((8, 24), (64, 24), (32, 0), (32, 34)):
        with pytest.raises(ddm.DDMError):
            ddm.ddm_set_tiling(ctx, *bad)
    AT.apply(ctx, {})


def test_autotuned_batched_workload_against_oracle(ctx):
    """The autotuner's pick on a slice of the batched workload (the first
    512 instances) reproduces the oracle's pairs instance by instance."""
    import torch
    inst = W.batched_instances(4096, d=2, alpha=1.0, size_lo=100, size_hi=100_000, seed=0)[:512]
    ulo, uhi, uoff, slo, shi, soff = W.concat_instances(inst)
    U = to_dev((ulo, uhi, slo, shi))
    uo = torch.from_numpy(uoff.astype(np.int64)).cuda()
    so = torch.from_numpy(soff.astype(np.int64)).cuda()
    K0, _, _, _ = run_batch(ctx, inst)
    buf = torch.empty((K0 + 1, 2), dtype=torch.int32, device="cuda")
    po = torch.empty(len(inst) + 1, dtype=torch.int64, device="cuda")

    def run():
        ddm.ddm_batch_match_async(ctx, U[0], U[1], uo, U[2], U[3], so, buf, po)

    best, table = AT.autotune(ctx, run, reps=1)
    assert len(table) == len(AT.candidates())
    K, p, pof, _ = run_batch(ctx, inst)          # under the chosen setting
    assert K == K0
    for i, a in enumerate(inst):
        got = p[pof[i]:pof[i + 1]]
        _, ou, os_ = oracle.itm_pairs(*a)
        assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_))), (i, best)
    AT.apply(ctx, {})


@pytest.mark.parametrize("qpp,swap_min", [(32, 1), (16, 1), (32, 33), (32, 12)])
@pytest.mark.parametrize("flags", [0, 1])
def test_leaf_test_forms_exact_against_oracle(ctx, qpp, swap_min, flags):
    """Every leaf visit through one form: swap_min 1 sends all of them
    through the rank tables (d <= 3), 33 through the per-query comparisons;
    tie-heavy grids, signed zeros, infinite bounds, degenerate and identical
    extents, ragged leaves -- pair sets equal to the oracle's."""
    from tests.test_gpu_parity import check_exact
    ddm.ddm_set_tiling(ctx, qpp, swap_min)
    try:
        for d in (1, 2, 3):
            for seed in range(6):
                rng = np.random.default_rng(77 + seed)
                n, m = (int(v) for v in rng.integers(1, 400, size=2))
                arrays = W.grid_random(n, m, d, seed=seed, grid=5)
                if seed == 5:   # infinite bounds in the mix
                    arrays[3][0, :3] = np.inf
                    arrays[2][d - 1, :2] = -np.inf
                    arrays[0][0, :2] = -np.inf
                check_exact(ctx, arrays, flags)
        lo = np.array([[-0.0, 0.0, -np.inf, 5.0, 5.0, 5.0, 1e30, -1e-30] * 5], np.float32)
        hi = np.array([[0.0, 0.0, np.inf, 5.0, 5.0, 6.0, np.inf, 0.0] * 5], np.float32)
        check_exact(ctx, (lo.copy(), hi.copy(), lo.copy(), hi.copy()), flags)
        same = (np.full((3, 700), 7.0, np.float32), np.full((3, 700), 9.0, np.float32))
        check_exact(ctx, (same[0][:, :90].copy(), same[1][:, :90].copy(), same[0], same[1]), flags)
        for n, m in ((33, 64), (1025, 300), (4097, 97)):
            check_exact(ctx, W.uniform_fixed_length(n, m, 3, 0.2 * (n + m), seed=n), flags)
    finally:
        AT.apply(ctx, {})
