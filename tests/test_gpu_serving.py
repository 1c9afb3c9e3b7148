"""Serving: requests admitted while others run overlap on the GPU, and each
request's pairs are exactly those of the same request run alone against the
same (pinned) version of the moving subscriptions."""
import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import serving as S
from tests.helpers import keys

pytestmark = pytest.mark.gpu


def test_refit_matches_fresh_build():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_3458_gb300 import workloads as W
    a = W.uniform_fixed_length(30000, 20000, 2, 20.0, seed=1)
    b = W.uniform_fixed_length(30000, 20000, 2, 20.0, seed=2)   # "moved" subscriptions
    ctx = ddm.ddm_create(0)
    try:
        U = [torch.from_numpy(x).cuda() for x in a]
        ddm.ddm_build(ctx, U[2], U[3])
        slo, shi = torch.from_numpy(b[2]).cuda(), torch.from_numpy(b[3]).cuda()
        ddm.ddm_refit(ctx, slo, shi)
        K = ddm.ddm_plan(ctx, U[0], U[1])
        buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
        ddm.ddm_write(ctx, 0, 20000, buf)
        got = buf[:K].cpu().numpy().view(np.uint32)
    finally:
        ddm.ddm_destroy(ctx)
    Ko, ou, os_ = oracle.itm_pairs(a[0], a[1], b[2], b[3])
    assert K == Ko
    assert np.array_equal(got[:, 0], ou)
    assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_)))


def test_serving_mix_equals_alone():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    d, n, l = 2, 50000, 5000.0
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    lo = (torch.rand((d, n), generator=g, device="cuda") * (S.L - l)).contiguous()
    hi = (lo + l).contiguous()
    # odd steps refit the idle version in place, even steps rebuild it
    regions = S.ResidentRegions(lo, hi, keep_history=True, rebuild_every=2)
    state = {"lo": lo, "hi": hi}
    mg = torch.Generator(device="cuda")
    mg.manual_seed(11)

    def mover(step):
        state["lo"], state["hi"] = S.random_walk(state["lo"], state["hi"], 1000.0, mg)
        return state["lo"], state["hi"]

    sched = S.poisson_schedule(rate=20000.0, duration=0.01, federates=8, size_lo=1000,
                               size_hi=200000, seed=3)
    assert len(sched) >= 100
    srv = S.Server(regions, l, slots=2, pair_capacity=1 << 22, keep_pairs=True)
    try:
        done = srv.run(sched, mover=mover, step_s=0.002)
    finally:
        srv.close()
    # launches overlapped on the device, and some launch batched several requests
    overlap = any(a.batch != b.batch and a.admitted < b.done and b.admitted < a.done
                  for i, a in enumerate(done) for b in done[i + 1:])
    assert overlap
    per_launch = {}
    for r in done:
        per_launch[r.batch] = per_launch.get(r.batch, 0) + 1
    assert max(per_launch.values()) >= 2
    assert len({r.step for r in done}) >= 2          # the regions moved during the run
    assert regions.refits >= 1 and regions.rebuilds >= 1
    ctx = ddm.ddm_create(0)
    try:
        for r in done:
            plo, phi = regions.history[r.step]
            ulo, uhi = S.request_updates(r.seed, r.size, d, l)
            K = ddm.ddm_count(ctx, ulo, uhi, plo, phi)
            assert K == r.K
            buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
            ddm.ddm_match(ctx, ulo, uhi, plo, phi, buf)
            alone = buf[:K].cpu().numpy().view(np.uint32)
            assert np.array_equal(np.sort(keys(r.pairs[:, 0], r.pairs[:, 1])),
                                  np.sort(keys(alone[:, 0], alone[:, 1])))
        # and against the oracle for a few of them
        for r in done[:5]:
            plo, phi = regions.history[r.step]
            ulo, uhi = S.request_updates(r.seed, r.size, d, l)
            Ko, ou, os_ = oracle.itm_pairs(ulo.cpu().numpy(), uhi.cpu().numpy(),
                                           plo.cpu().numpy(), phi.cpu().numpy())
            assert Ko == r.K
            assert np.array_equal(np.sort(keys(r.pairs[:, 0], r.pairs[:, 1])),
                                  np.sort(keys(ou, os_)))
    finally:
        ddm.ddm_destroy(ctx)
        regions.close()


def test_refit_state_errors():
    import torch
    ctx = ddm.ddm_create(0)
    other = ddm.ddm_create(0)
    try:
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_refit(ctx, None, None)
        assert e.value.code == ddm.DDM_ERR_STATE
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_attach(other, ctx)
        assert e.value.code == ddm.DDM_ERR_STATE
        lo = torch.zeros((2, 64), device="cuda")
        hi = torch.ones((2, 64), device="cuda")
        ddm.ddm_build(ctx, lo, hi)
        ddm.ddm_attach(other, ctx)
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_refit(other, lo, hi)      # attached contexts do not own the tree
        assert e.value.code == ddm.DDM_ERR_STATE
        bad = hi.clone()
        bad[1, 5] = -1.0
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_refit(ctx, lo, bad)
        assert e.value.code == ddm.DDM_ERR_EXTENT
    finally:
        ddm.ddm_destroy(other)
        ddm.ddm_destroy(ctx)


def test_pair_offsets_of_concatenated_sets():
    """One plan over several update sets: ddm_pair_offsets_async gives each
    set's slice of the output laid out by update id."""
    import torch
    from paper_1309_3458_gb300 import workloads as W
    a = W.uniform_fixed_length(40000, 30000, 2, 30.0, seed=5)
    U = [torch.from_numpy(x).cuda() for x in a]
    m = 30000
    ctx = ddm.ddm_create(0)
    try:
        ddm.ddm_build(ctx, U[2], U[3])
        offsets = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        K = ddm.ddm_plan(ctx, U[0], U[1], offsets=offsets)
        bounds = [0, 1, 1, 777, 12345, 29999, m, m + 5]       # the last reads as m
        uoff = torch.tensor(bounds, dtype=torch.int64, device="cuda")
        poff = torch.full((len(bounds),), -1, dtype=torch.int64, device="cuda")
        ddm.ddm_pair_offsets_async(ctx, uoff, poff)
        torch.cuda.synchronize()
        off = offsets.cpu().numpy()
        want = [off[min(b, m)] for b in bounds]
        assert poff.cpu().tolist() == want
        assert want[-1] == K
        buf = torch.empty((K, 2), dtype=torch.int32, device="cuda")
        ddm.ddm_write(ctx, 0, m, buf)
        upd = buf[:, 0].cpu().numpy()
        for i in range(len(bounds) - 2):   # slice i holds exactly updates [b_i, b_{i+1})
            sl = upd[want[i]:want[i + 1]]
            assert np.all((sl >= bounds[i]) & (sl < bounds[i + 1]))
    finally:
        ddm.ddm_destroy(ctx)


def test_serving_scale_requests_exact():
    """The serving workload's scale: 1e6 resident regions (d = 2, side 1e3)
    moving every 2 ms, requests of 1e3 .. 2e5 updates admitted together;
    every request's pairs equal a fresh match against the version it pinned,
    and four of them equal the oracle's."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    d, n, l = 2, 1_000_000, 1000.0
    g = torch.Generator(device="cuda")
    g.manual_seed(2026)
    lo = (torch.rand((d, n), generator=g, device="cuda") * (S.L - l)).contiguous()
    hi = (lo + l).contiguous()
    regions = S.ResidentRegions(lo, hi, keep_history=True, rebuild_every=1)
    state = {"lo": lo, "hi": hi}
    mg = torch.Generator(device="cuda")
    mg.manual_seed(5)

    def mover(step):
        state["lo"], state["hi"] = S.random_walk(state["lo"], state["hi"], 1000.0, mg)
        return state["lo"], state["hi"]

    sched = S.poisson_schedule(rate=2000.0, duration=0.015, federates=64, size_lo=1000,
                               size_hi=200_000, seed=8)
    assert len(sched) >= 15
    srv = S.Server(regions, l, slots=4, pair_capacity=1 << 24, keep_pairs=True)
    ctx = ddm.ddm_create(0)
    try:
        done = srv.run(sched, mover=mover, step_s=0.002)
        for r in done:
            plo, phi = regions.history[r.step]
            ulo, uhi = S.request_updates(r.seed, r.size, d, l)
            K = ddm.ddm_count(ctx, ulo, uhi, plo, phi)
            assert K == r.K
            buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
            ddm.ddm_match(ctx, ulo, uhi, plo, phi, buf)
            alone = buf[:K].cpu().numpy().view(np.uint32)
            assert np.array_equal(np.sort(keys(r.pairs[:, 0], r.pairs[:, 1])),
                                  np.sort(keys(alone[:, 0], alone[:, 1])))
        for r in sorted(done, key=lambda r: r.size)[-4:]:
            plo, phi = regions.history[r.step]
            ulo, uhi = S.request_updates(r.seed, r.size, d, l)
            Ko, ou, os_ = oracle.itm_pairs(ulo.cpu().numpy(), uhi.cpu().numpy(),
                                           plo.cpu().numpy(), phi.cpu().numpy())
            assert Ko == r.K
            assert np.array_equal(np.sort(keys(r.pairs[:, 0], r.pairs[:, 1])),
                                  np.sort(keys(ou, os_)))
    finally:
        srv.close()
        ddm.ddm_destroy(ctx)
        regions.close()


def test_adaptive_refit_policy_rebuilds_and_stays_exact():
    """Refit every step with a probe-triggered rebuild: regions moving by
    their own side per step age the order fast, so the probe finds the
    refitted tree slower than the threshold and the version is rebuilt; every
    request's pairs still equal its pinned version's, alone."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    d, n, l = 2, 40000, 3000.0
    g = torch.Generator(device="cuda")
    g.manual_seed(21)
    lo = (torch.rand((d, n), generator=g, device="cuda") * (S.L - l)).contiguous()
    hi = (lo + l).contiguous()
    regions = S.ResidentRegions(lo, hi, keep_history=True, rebuild_every=0, adaptive=1.2)
    state = {"lo": lo, "hi": hi}
    mg = torch.Generator(device="cuda")
    mg.manual_seed(5)

    def mover(step):
        state["lo"], state["hi"] = S.random_walk(state["lo"], state["hi"], 3000.0, mg)
        return state["lo"], state["hi"]

    sched = S.poisson_schedule(rate=8000.0, duration=0.02, federates=8, size_lo=500,
                               size_hi=50000, seed=9)
    srv = S.Server(regions, l, slots=2, pair_capacity=1 << 22, keep_pairs=True)
    try:
        done = srv.run(sched, mover=mover, step_s=0.002)
    finally:
        srv.close()
    assert regions.refits >= 1 and regions.rebuilds >= 1
    assert regions.tests_ratio and max(regions.tests_ratio) > 1.2
    ctx = ddm.ddm_create(0)
    try:
        for r in done[::3]:
            plo, phi = regions.history[r.step]
            ulo, uhi = S.request_updates(r.seed, r.size, d, l)
            K = ddm.ddm_count(ctx, ulo, uhi, plo, phi)
            assert K == r.K
            buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
            ddm.ddm_match(ctx, ulo, uhi, plo, phi, buf)
            alone = buf[:K].cpu().numpy().view(np.uint32)
            assert np.array_equal(np.sort(keys(r.pairs[:, 0], r.pairs[:, 1])),
                                  np.sort(keys(alone[:, 0], alone[:, 1])))
    finally:
        ddm.ddm_destroy(ctx)
        regions.close()


def test_context_used_from_two_streams_with_workspace_growth():
    """A context's calls may come on different streams: each call waits for
    the context's previous one, so workspace grown (and freed in stream order)
    on one stream never overlaps work still running on the other."""
    import torch
    from paper_1309_3458_gb300 import workloads as W
    small = W.uniform_fixed_length(20000, 5000, 2, 10.0, seed=3)
    big = W.uniform_fixed_length(20000, 400000, 2, 30.0, seed=4)
    ctx = ddm.ddm_create(0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        S_ = [torch.from_numpy(x).cuda() for x in small[2:]]
        Us = [torch.from_numpy(x).cuda() for x in small[:2]]
        Ub = [torch.from_numpy(x).cuda() for x in big[:2]]
        torch.cuda.synchronize()
        for rep in range(3):
            with torch.cuda.stream(s1):
                ddm.ddm_build(ctx, *S_, stream=s1)
                ddm.ddm_plan_async(ctx, *Us, stream=s1)
            with torch.cuda.stream(s2):      # larger plan: the workspace grows on s2
                kb = ddm.ddm_plan(ctx, *Ub, stream=s2)
                buf = torch.empty((kb, 2), dtype=torch.int32, device="cuda")
                assert ddm.ddm_write(ctx, 0, big[0].shape[1], buf, stream=s2) == kb
            torch.cuda.synchronize()
            got = buf.cpu().numpy().view(np.uint32)
            Ko, ou, os_ = oracle.itm_pairs(big[0], big[1], small[2], small[3])
            assert kb == Ko
            assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_)))
            del buf
    finally:
        ddm.ddm_destroy(ctx)
