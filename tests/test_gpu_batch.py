"""Batched instances on the GPU: one call over many independent problems
must give, for every instance, exactly the pairs of that instance alone
(instance-local ids), as the oracle and the single-problem call compute
them; the host-sync-free variant must give the same result from a CUDA
graph."""
import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W
from tests.helpers import keys, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


def make_batch(d, count, seed):
    rng = np.random.default_rng(seed)
    inst = []
    for i in range(count):
        kind = rng.integers(0, 5)
        if kind == 0:     # empty on one side
            n, m = (0, int(rng.integers(1, 50))) if rng.integers(0, 2) else (int(rng.integers(1, 50)), 0)
            a = W.uniform_fixed_length(max(n, 1), max(m, 1), d, 1.0, seed=seed * 7919 + i)
            inst.append((a[0][:, :m].copy(), a[1][:, :m].copy(), a[2][:, :n].copy(), a[3][:, :n].copy()))
        elif kind == 1:   # tie-heavy grid
            inst.append(W.grid_random(int(rng.integers(1, 120)), int(rng.integers(1, 120)), d,
                                      seed=seed * 7919 + i, grid=6))
        else:             # uniform, log-uniform size
            N = int(np.exp(rng.uniform(np.log(4), np.log(20000))))
            alpha = min(float(rng.choice([1.0, 30.0])), 0.25 * N)
            inst.append(W.uniform_fixed_length(max(1, N - N // 2), max(1, N // 2), d, alpha,
                                               seed=seed * 7919 + i))
    return inst


def run_batch(ctx, inst, flags=0):
    import torch
    ulo, uhi, uoff, slo, shi, soff = W.concat_instances(inst)
    U = to_dev((ulo, uhi, slo, shi))
    uo = torch.from_numpy(uoff.astype(np.int64)).cuda()
    so = torch.from_numpy(soff.astype(np.int64)).cuda()
    po = torch.empty(len(inst) + 1, dtype=torch.int64, device="cuda")
    try:   # count first: no buffer, so the call reports the capacity it needs
        K = ddm.ddm_batch_match(ctx, U[0], U[1], uo, U[2], U[3], so, None, pair_off=po,
                                flags=flags)
    except ddm.DDMError as e:
        assert e.code == ddm.DDM_ERR_CAPACITY
        K = e.k
    pairs = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    assert ddm.ddm_batch_match(ctx, U[0], U[1], uo, U[2], U[3], so, pairs, pair_off=po,
                               flags=flags) == K
    return K, pairs[:K].cpu().numpy().view(np.uint32).copy(), po.cpu().numpy(), (U, uo, so)


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("flags", [0, 1])
def test_batch_equals_each_instance_alone(ctx, d, flags):
    inst = make_batch(d, 120, seed=d * 10 + flags)
    K, p, po, _ = run_batch(ctx, inst, flags)
    assert po[0] == 0 and po[-1] == K
    total = 0
    for i, a in enumerate(inst):
        got = p[po[i]:po[i + 1]]
        Ko, ou, os_ = oracle.itm_pairs(*a, flags=flags)
        total += Ko
        assert len(got) == Ko, i
        assert np.array_equal(got[:, 0], ou)            # grouped by local update id
        assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_))), i
    assert total == K


def test_batch_d2_matches_single_problem_calls(ctx):
    import torch
    inst = make_batch(2, 60, seed=99)
    K, p, po, _ = run_batch(ctx, inst)
    for i, a in enumerate(inst):
        if a[0].shape[1] == 0 or a[2].shape[1] == 0:
            assert po[i + 1] == po[i]
            continue
        U = to_dev(a)
        k = ddm.ddm_count(ctx, *U)
        buf = torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda")
        ddm.ddm_match(ctx, *U, buf)
        mine = buf[:k].cpu().numpy().view(np.uint32)
        got = p[po[i]:po[i + 1]]
        assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(mine[:, 0], mine[:, 1])))


@pytest.mark.parametrize("small", [False, True])
def test_batch_async_in_cuda_graph(ctx, small):
    """Graph replay equals the plain call.  Under capture the sorts take
    their recorded forms (one CTA for a small set, the multi-launch sort
    otherwise) while the plain call uses the cooperative one: the pairs
    must not differ."""
    import torch
    if small:   # every set below 8,192 extents
        inst = [W.grid_random(int(n), int(m), 2, seed=40 + i, grid=6)
                for i, (n, m) in enumerate(np.random.default_rng(3).integers(1, 150, size=(20, 2)))]
    else:
        inst = make_batch(2, 200, seed=5)
    K, p, po, (U, uo, so) = run_batch(ctx, inst)
    pairs = torch.zeros((K + 16, 2), dtype=torch.int32, device="cuda")
    pof = torch.zeros(len(inst) + 1, dtype=torch.int64, device="cuda")
    kd = torch.zeros(1, dtype=torch.int64, device="cuda")
    ed = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # warm-up with the same sizes (allocations happen here)
        ddm.ddm_batch_match_async(ctx, U[0], U[1], uo, U[2], U[3], so, pairs, pof, kd, ed, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    pairs.zero_()
    with torch.cuda.graph(g, stream=s):
        ddm.ddm_batch_match_async(ctx, U[0], U[1], uo, U[2], U[3], so, pairs, pof, kd, ed, stream=s)
    for _ in range(2):
        pairs.zero_()
        kd.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(kd[0]) == K and int(ed[0]) == 0
        assert np.array_equal(pairs[:K].cpu().numpy().view(np.uint32), p)
        assert np.array_equal(pof.cpu().numpy(), po)


def test_batch_errors(ctx):
    import torch
    inst = make_batch(2, 10, seed=3)
    ulo, uhi, uoff, slo, shi, soff = W.concat_instances(inst)
    slo[1, 3] = np.nan
    U = to_dev((ulo, uhi, slo, shi))
    uo = torch.from_numpy(uoff.astype(np.int64)).cuda()
    so = torch.from_numpy(soff.astype(np.int64)).cuda()
    buf = torch.empty((1000000, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_batch_match(ctx, U[0], U[1], uo, U[2], U[3], so, buf)
    assert e.value.code == ddm.DDM_ERR_EXTENT
    rc = ddm.lib().ddm_batch_match(ctx, 2, 0, None, None, None, 0, None, None, None, 0, 0, None, 0,
                                   None, None, None)
    assert rc == ddm.DDM_ERR_ARG


def test_batched_workload_exact(ctx):
    """The batched workload itself (4,096 independent d = 2 problems, sizes
    log-uniform in [1e2, 1e5], 5.8e7 extents): every instance's per-update
    counts and order-independent digests equal the oracle's, and 40
    instances match pair by pair."""
    from tests.helpers import digests_from_pairs
    inst = W.batched_instances(4096, d=2, alpha=1.0, size_lo=100, size_hi=100_000, seed=0)
    K, p, po, _ = run_batch(ctx, inst)
    threads = oracle.threads()
    sample = set(np.random.default_rng(4).choice(len(inst), 40, replace=False).tolist())
    total = 0
    for i, a in enumerate(inst):
        got = p[po[i]:po[i + 1]]
        m_i = a[0].shape[1]
        Ko, counts, digests = oracle.itm_count(*a, threads=threads)
        total += Ko
        assert len(got) == Ko, i
        gc = np.bincount(got[:, 0], minlength=m_i).astype(np.uint32)
        assert np.array_equal(gc, counts), i
        assert (np.diff(got[:, 0].astype(np.int64)) >= 0).all()      # grouped by update
        off = np.concatenate([[0], np.cumsum(gc, dtype=np.int64)])
        assert np.array_equal(digests_from_pairs(off, got[:, 1]), digests), i
        if i in sample:
            _, ou, os_ = oracle.itm_pairs(*a)
            assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_))), i
    assert total == K == 58345727
