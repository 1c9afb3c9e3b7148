"""Full-size parity: the named workloads at their real sizes (GPU).

* d = 1, N = 1e4 and N = 1e6 (three overlap degrees): the whole pair list,
  element by element, against the oracle's interval tree.
* d = 2, N = 1e6 (three overlap degrees): per-update counts and
  order-independent digests of every update against the oracle's interval
  tree (OpenMP), plus the whole pair set where it is small.
* d = 3, N = 1e7, clustered (about 4.4e10 pairs, more than device memory):
  run exactly as the benchmark runs it -- plan, then ordered chunks of a
  pair buffer (chunks alternating above and below 2^32 pairs).  10^4 random
  updates and whole dense packets are checked pair by pair against brute
  force, 10^4 more by count and digest against the oracle's interval tree,
  and properties that hold at any size are checked on every chunk.
  The compressed output (subscription ids only) of more than 2^32 pairs in
  one call equals the pair list's subscription column.
"""
import os

import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W
from tests.helpers import digests_from_pairs, gpu_match, keys, to_dev

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


@pytest.mark.parametrize("name", ["uniform_d1_N1e4_a1", "uniform_d1_N1e6_a0.01",
                                  "uniform_d1_N1e6_a1", "uniform_d1_N1e6_a100"])
def test_d1_full_pair_lists(ctx, name):
    arrays = W.make(name)
    K, pu, ps = gpu_match(ctx, arrays)
    Ko, ou, os_ = oracle.itm_pairs(*arrays)
    assert K == Ko
    assert np.array_equal(pu, ou) and np.array_equal(ps, os_)
    Kb, cb = oracle.bits_count(*arrays)          # independent count (Section II)
    assert Kb == K and np.array_equal(np.bincount(pu, minlength=arrays[0].shape[1]), cb)


@pytest.mark.parametrize("name", ["uniform_d2_N1e6_a0.01", "uniform_d2_N1e6_a1",
                                  "uniform_d2_N1e6_a100"])
def test_d2_full_counts_and_digests(ctx, name):
    import torch
    arrays = W.make(name)
    K, pu, ps = gpu_match(ctx, arrays)
    m = arrays[0].shape[1]
    counts = np.bincount(pu, minlength=m)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    Ko, co, go = oracle.itm_count(*arrays, threads=THREADS)
    assert K == Ko
    assert np.array_equal(counts, co)
    assert np.array_equal(digests_from_pairs(offsets, ps), go)
    if K <= 2_000_000:
        _, ou, os_ = oracle.itm_pairs(*arrays)
        assert np.array_equal(np.sort(keys(pu, ps)), np.sort(keys(ou, os_)))


# Brute force (Alg. 2) on the sampled updates runs in a spawned process pool:
# each worker regenerates the seeded subscriptions once and takes chunks of
# the sampled updates.
_BF_SUBS = None


def _bf_init(name):
    global _BF_SUBS
    a = W.make(name)
    _BF_SUBS = (a[2], a[3])


def _bf_chunk(args):
    ulo_c, uhi_c = args
    _, counts, _, _, ps = oracle.bf(ulo_c, uhi_c, *_BF_SUBS)
    return counts, ps


def brute_force_sets(name, ulo, uhi, ids):
    """Per sampled update, its subscription ids in ascending order (BF)."""
    import multiprocessing as mp
    chunks = np.array_split(np.asarray(ids), max(1, 4 * THREADS))
    work = [(np.ascontiguousarray(ulo[:, c]), np.ascontiguousarray(uhi[:, c])) for c in chunks if len(c)]
    with mp.get_context("spawn").Pool(THREADS, initializer=_bf_init, initargs=(name,)) as pool:
        res = pool.map(_bf_chunk, work)
    out = {}
    for c, (counts, ps) in zip([c for c in chunks if len(c)], res):
        at = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
        for i, j in enumerate(c):
            out[int(j)] = ps[at[i]:at[i + 1]]
    return out


def test_d3_clustered_full_size_chunked(ctx):
    """Run as the benchmark runs it, checked on a sample of 10^4 random
    updates plus whole 32-query packets pair by pair against brute force
    (Alg. 2), and 10^4 more by count and digest against the oracle's
    interval tree.  The packets are the densest of the plan (by pairs per
    packet: their leaves are tested with the swapped loops, lane = query,
    which runs for most of this workload's tests) and some chosen at random.
    Chunks alternate between a pair buffer above 2^32 pairs (64-bit output
    positions in the write kernel) and one below (32-bit positions), so both
    write kernels expand sampled updates.  Every query touches leaves of
    several size classes of the tree order."""
    import torch
    name = "clustered_d3_N1e7_a100"
    arrays = W.make(name)
    ulo, uhi, slo, shi = arrays
    d, m = ulo.shape
    n = slo.shape[1]
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    off = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    K = ddm.ddm_plan(ctx, U[0], U[1], offsets=off)
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    ooff = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    ddm.ddm_plan_order(ctx, order, ooff)
    torch.cuda.synchronize()
    off_h, order_h, ooff_h = off.cpu().numpy(), order.cpu().numpy(), ooff.cpu().numpy()
    counts = np.diff(off_h)
    assert off_h[-1] == K == ooff_h[-1] and K > 1e10
    assert np.array_equal(np.diff(ooff_h), counts[order_h])

    rng = np.random.default_rng(2024)
    packets = m // 32
    per_packet = ooff_h[32 * np.arange(packets + 1)[1:]] - ooff_h[32 * np.arange(packets)]
    dense = np.argsort(per_packet)[-8:]
    chosen = np.concatenate([dense, rng.choice(packets, 8, replace=False)])
    packet_ids = order_h[(32 * chosen[:, None] + np.arange(32)[None, :]).ravel()]
    exact = np.unique(np.concatenate([rng.choice(m, 10_000, replace=False), packet_ids]))
    sampled = np.sort(rng.choice(m, 10_000, replace=False))     # count + digest vs ITM
    pos_of = np.empty(m, np.int64)
    pos_of[order_h] = np.arange(m)
    want_pos = {int(pos_of[j]): int(j) for j in np.concatenate([exact, sampled])}

    cap = int(64e9) // 8                 # above 2^32 pairs: 64-bit positions
    small_cap = int(16e9) // 8           # below: 32-bit positions
    buf = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    got = {}
    b, written, chunk = 0, 0, 0
    while b < m:
        cap_i = cap if chunk % 2 == 0 else small_cap
        e = ddm.ddm_chunk_end_ordered(ctx, b, cap_i)
        k = ddm.ddm_write_ordered(ctx, b, e, buf[:cap_i])
        assert k == ooff_h[e] - ooff_h[b]
        written += k
        # properties on the whole chunk: ids in range, each update's run
        # starts and ends where the plan says
        assert bool((buf[:k, 1] >= 0).all()) and bool((buf[:k, 1] < n).all())
        pos = np.arange(b, e)
        nz = pos[counts[order_h[pos]] > 0]
        pick = nz if len(nz) <= 200_000 else rng.choice(nz, 200_000, replace=False)
        first = torch.from_numpy((ooff_h[pick] - ooff_h[b]).astype(np.int64)).cuda()
        last = torch.from_numpy((ooff_h[pick + 1] - ooff_h[b] - 1).astype(np.int64)).cuda()
        ids = torch.from_numpy(order_h[pick].astype(np.int32)).cuda()
        assert torch.equal(buf[first, 0], ids) and torch.equal(buf[last, 0], ids)
        for p in [p for p in want_pos if b <= p < e]:
            lo_, hi_ = ooff_h[p] - ooff_h[b], ooff_h[p + 1] - ooff_h[b]
            got[want_pos[p]] = buf[lo_:hi_, 1].cpu().numpy().view(np.uint32).copy()
        if b == 0:
            # compressed output at full size, more than 2^32 ids in one call (64-bit
            # positions): the subscription column of the pair list, id for id
            e2 = ddm.ddm_chunk_end_ordered(ctx, 0, int(4.5e9))
            k2 = int(ooff_h[e2])
            assert 2**32 < k2 <= k
            sub_ids = torch.empty(k2, dtype=torch.int32, device="cuda")
            assert ddm.ddm_write_ordered_ids(ctx, 0, e2, sub_ids) == k2
            assert torch.equal(sub_ids, buf[:k2, 1])
            del sub_ids
        b = e
        chunk += 1
    assert written == K and chunk >= 4
    del buf
    torch.cuda.empty_cache()

    # pair by pair against brute force (Alg. 2)
    bf_sets = brute_force_sets(name, ulo, uhi, exact)
    for j in exact:
        assert np.array_equal(np.sort(got[int(j)]), bf_sets[int(j)]), j
    # counts and digests against the oracle's interval tree (OpenMP)
    Ks, cs, gs = oracle.itm_count(np.ascontiguousarray(ulo[:, sampled]),
                                  np.ascontiguousarray(uhi[:, sampled]), slo, shi,
                                  threads=THREADS)
    assert np.array_equal(counts[sampled], cs)
    for j, g in zip(sampled, gs):
        assert oracle.digest_of(got[int(j)]) == int(g)
