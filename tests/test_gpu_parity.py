"""GPU parity: libddm (through its C ABI) against the CPU oracle.

Integer results (pair sets, per-update counts, the sorted order) must be
bit-exact.  The method only compares float32 coordinates, so there is no
floating-point tolerance: both sides compare the same bytes.

Both sides group pairs by update id, so the update column is compared
element by element.  Within one update the library reports pairs in the
order of its tree's leaves.  For d = 1 that order is dimension-0 (lower,
upper, id), the order of the oracle's in-order interval tree walk, and the
whole list is compared element by element.  For d > 1 the GPU tree refines
the order near the leaves, so the subscription column is compared as a set
per update, and the order is checked against the tree's exported order.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import workloads as W
from tests.helpers import gpu_match, keys, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = ddm.ddm_create(0)
    yield h
    ddm.ddm_destroy(h)


def tree_rank(ctx, n):
    """rank[sub id] = position of the subscription in the built tree."""
    import torch
    order = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    ddm.ddm_tree_export(ctx, order)
    torch.cuda.synchronize()
    order = order[:n].cpu().numpy().view(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(n, dtype=np.uint32))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    return rank


def check_exact(ctx, arrays, flags=0):
    d, n = arrays[2].shape
    K, pu, ps = gpu_match(ctx, arrays, flags)
    Ko, ou, os_ = oracle.itm_pairs(*arrays, flags=flags)
    assert K == Ko
    assert np.array_equal(pu, ou)
    if d == 1:
        assert np.array_equal(ps, os_)
    else:
        assert np.array_equal(keys(pu, ps) if K == 0 else np.sort(keys(pu, ps)),
                              np.sort(keys(ou, os_)))
    if K:
        # within an update, pairs follow the tree's order; no duplicates
        r = tree_rank(ctx, n)[ps]
        same = pu[1:] == pu[:-1]
        assert (r[1:][same] > r[:-1][same]).all()
    return K


@pytest.mark.parametrize("d", [1, 2, 3, 5])
@pytest.mark.parametrize("flags", [0, 1])
def test_tiny_grids_with_ties(ctx, d, flags):
    for seed in range(10):
        rng = np.random.default_rng(1000 + seed)
        n, m = (int(v) for v in rng.integers(1, 300, size=2))
        arrays = W.grid_random(n, m, d, seed=seed, grid=6)
        check_exact(ctx, arrays, flags)
        K_bf = oracle.bf(*arrays, flags=flags, pairs=False)[0]
        assert K_bf == gpu_match(ctx, arrays, flags)[0]


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 7, 40])
def test_lattice_closed_forms(ctx, d, k):
    if k ** d > 70000:
        k = int(round(70000 ** (1 / d)))
    for shift, want_c, want_o in ((False, (3 * k - 2) ** d, k ** d),
                                  (True, (2 * k - 1) ** d, (2 * k - 1) ** d)):
        arrays = W.lattice(k, d, shift_half=shift)
        assert gpu_match(ctx, arrays, 0)[0] == want_c
        assert gpu_match(ctx, arrays, 1)[0] == want_o


def test_fig1_worked_example(ctx):
    from tests.test_oracle import load_fig1
    arrays, M, _ = load_fig1()
    for flags in (0, 1):
        K, pu, ps = gpu_match(ctx, arrays, flags)
        got = np.zeros(M.shape, int)
        got[ps, pu] = 1
        assert np.array_equal(got, M)


@pytest.mark.parametrize("n,m", [(1, 1), (31, 7), (32, 32), (33, 1), (1023, 999), (1025, 2048),
                                 (4095, 4097), (32769, 5000), (40000, 33)])
def test_ragged_sizes(ctx, n, m):
    arrays = W.uniform_fixed_length(n, m, 2, min(300.0, 0.25 * (n + m)), seed=n + m)
    check_exact(ctx, arrays)


def test_empty_sets(ctx):
    import torch
    for n, m in ((0, 10), (10, 0), (0, 0)):
        arrays = W.uniform_fixed_length(max(n, 1), max(m, 1), 2, 1.0, seed=1)
        arrays = (arrays[0][:, :m].copy(), arrays[1][:, :m].copy(),
                  arrays[2][:, :n].copy(), arrays[3][:, :n].copy())
        U = to_dev(arrays)
        assert ddm.ddm_count(ctx, *U) == 0
        pairs = torch.empty((4, 2), dtype=torch.int32, device="cuda")
        assert ddm.ddm_match(ctx, *U, pairs) == 0


def test_special_values(ctx):
    # -0.0 against +0.0, infinite bounds, identical extents, degenerate points
    lo = np.array([[-0.0, 0.0, -np.inf, 5.0, 5.0, 5.0, 1e30, -1e-30]], np.float32)
    hi = np.array([[0.0, 0.0, np.inf, 5.0, 5.0, 6.0, np.inf, 0.0]], np.float32)
    arrays = (lo.copy(), hi.copy(), lo.copy(), hi.copy())
    for flags in (0, 1):
        check_exact(ctx, arrays, flags)


def test_all_identical_extents(ctx):
    lo = np.full((2, 3000), 7.0, np.float32)
    hi = np.full((2, 3000), 9.0, np.float32)
    K = check_exact(ctx, (lo[:, :1000].copy(), hi[:, :1000].copy(), lo, hi))
    assert K == 1000 * 3000


def test_tree_order_and_node_bounds(ctx):
    import torch
    arrays = W.clustered_lognormal(70000, 10, d=3, alpha=100.0, seed=4)
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    L, counts, total = ddm.ddm_tree_shape(ctx)
    n = arrays[2].shape[1]
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    nlo = torch.empty(3 * total, dtype=torch.float32, device="cuda")
    nhi = torch.empty(3 * total, dtype=torch.float32, device="cuda")
    ddm.ddm_tree_export(ctx, order, nlo, nhi)
    torch.cuda.synchronize()
    order = order.cpu().numpy().view(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(n, dtype=np.uint32))
    # node bounds: per dimension, min lower / max upper over each node's range
    nlo = nlo.cpu().numpy().reshape(3, total)
    nhi = nhi.cpu().numpy().reshape(3, total)
    assert counts[-1] <= 32 and sum(counts) == total
    for k in range(3):
        lo, hi = arrays[2][k][order], arrays[3][k][order]
        pos = 0
        for lvl, c in enumerate(counts, start=1):
            span = 32 ** lvl
            pad = c * span - n
            mn = np.concatenate([lo, np.full(pad, np.inf, np.float32)]).reshape(c, span).min(1)
            mx = np.concatenate([hi, np.full(pad, -np.inf, np.float32)]).reshape(c, span).max(1)
            assert np.array_equal(nlo[k, pos:pos + c], mn) and np.array_equal(nhi[k, pos:pos + c], mx)
            pos += c
    # Order for d >= 2: size classes ascending (the binary exponent of each
    # extent's largest side), and inside a class the dimension-0 lower bounds
    # -- to the 24 bits the locality keys keep -- ascend from one re-sort
    # group to the next (aligned powers of two counted from the class's first
    # position).
    side = (arrays[3] - arrays[2]).max(axis=0)          # float32, as on the device
    cls = (side.view(np.uint32) >> 23) & 0xff
    c_ord = cls[order]
    assert (np.diff(c_ord.astype(np.int64)) >= 0).all()
    lo0 = (order_key(arrays[2][0]) >> np.uint32(8))[order].astype(np.float64)
    for c in np.unique(c_ord):
        pos = np.nonzero(c_ord == c)[0]
        start, cnt = int(pos[0]), len(pos)
        G = 1 << resort_bits(cnt, 3)
        seg = lo0[start:start + cnt]
        nb = -(-cnt // G)
        pad = nb * G - cnt
        bmax = np.concatenate([seg, np.full(pad, -np.inf)]).reshape(nb, G).max(1)
        bmin = np.concatenate([seg, np.full(pad, np.inf)]).reshape(nb, G).min(1)
        assert (bmax[:-1] <= bmin[1:]).all()


def order_key(x):
    """IEEE order as unsigned integers (-0 like +0): the sort keys' mapping."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).copy()
    b[b == np.uint32(0x80000000)] = 0
    return np.where(b & np.uint32(0x80000000), ~b, b | np.uint32(0x80000000)).astype(np.uint32)


def str_group_log2(n, d, k):
    """Re-sort group exponent for dimension k of a set of n extents: groups of
    32 * nb^((d-k)/d) positions (nb = n/32 leaves, sort-tile-recursive
    packing), rounded to a power of two; 0 = no re-sort."""
    if n < 64:
        return 0
    nb = (n + 31) // 32
    g = int(math.floor(math.log2(32.0 * nb ** ((d - k) / d)) + 0.5))
    return 0 if g < 6 or (1 << g) >= n else g


def resort_bits(n, d):
    """Largest re-sort group exponent over dimensions 1..d-1 (each strictly
    smaller than the ones before it, else none)."""
    best = 0
    for k in range(1, d):
        g = str_group_log2(n, d, k)
        for j in range(1, k):
            gp = str_group_log2(n, d, j)
            if gp > 0 and g >= gp:
                g = 0
        best = max(best, g)
    return best


def test_tree_order_d1_is_paper_order(ctx):
    import torch
    arrays = W.grid_random(50000, 10, 1, seed=8, grid=300)
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    order = torch.empty(50000, dtype=torch.int32, device="cuda")
    ddm.ddm_tree_export(ctx, order)
    torch.cuda.synchronize()
    want, _ = oracle.tree_order(arrays[2][0], arrays[3][0])
    assert np.array_equal(order.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("name,scale", [("uniform_d1_N1e4_a1", 1.0),
                                        ("uniform_d1_N1e6_a0.01", 0.01),
                                        ("uniform_d1_N1e6_a1", 0.01),
                                        ("uniform_d1_N1e6_a100", 0.01),
                                        ("uniform_d2_N1e6_a0.01", 0.01),
                                        ("uniform_d2_N1e6_a1", 0.01),
                                        ("uniform_d2_N1e6_a100", 0.01),
                                        ("clustered_d3_N1e7_a100", 0.001)])
def test_scaled_configs_exact(ctx, name, scale):
    arrays = W.make(name, scale)
    for flags in (0, 1):
        check_exact(ctx, arrays, flags)


def test_staged_chunks_reproduce_full_output(ctx):
    import torch
    arrays = W.uniform_fixed_length(20000, 30000, 2, 100.0, seed=9)
    K, pu, ps = gpu_match(ctx, arrays)
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    off = torch.empty(30001, dtype=torch.int64, device="cuda")
    assert ddm.ddm_plan(ctx, U[0], U[1], offsets=off) == K
    off = off.cpu().numpy()
    cap = K // 7 + 1
    buf = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    got, b = [], 0
    while b < 30000:
        e = ddm.ddm_chunk_end(ctx, b, cap)
        assert e > b and off[e] - off[b] <= cap and (e == 30000 or off[e + 1] - off[b] > cap)
        k = ddm.ddm_write(ctx, b, e, buf)
        assert k == off[e] - off[b]
        got.append(buf[:k].cpu().numpy().view(np.uint32).copy())
        b = e
    got = np.concatenate(got)
    assert np.array_equal(got[:, 0], pu) and np.array_equal(got[:, 1], ps)
    # match_range gives the same slice
    buf2 = torch.empty((K, 2), dtype=torch.int32, device="cuda")
    k = ddm.ddm_match_range(ctx, *U, 1234, 4321, buf2)
    sl = buf2[:k].cpu().numpy().view(np.uint32)
    assert np.array_equal(sl[:, 0], pu[off[1234]:off[4321]])
    assert np.array_equal(sl[:, 1], ps[off[1234]:off[4321]])


@pytest.mark.parametrize("flags", [0, 1])
def test_ordered_chunks_cover_the_same_pairs(ctx, flags):
    import torch
    arrays = W.clustered_lognormal(40000, 30000, d=3, alpha=100.0, seed=12)
    K, pu, ps = gpu_match(ctx, arrays, flags)
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    m = 30000
    off = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    assert ddm.ddm_plan(ctx, U[0], U[1], flags=flags, offsets=off) == K
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    ooff = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    ddm.ddm_plan_order(ctx, order, ooff)
    torch.cuda.synchronize()
    off, order, ooff = off.cpu().numpy(), order.cpu().numpy(), ooff.cpu().numpy()
    assert np.array_equal(np.sort(order), np.arange(m))
    assert ooff[0] == 0 and ooff[-1] == K
    assert np.array_equal(np.diff(ooff), np.diff(off)[order])
    cap = K // 5 + 1
    buf = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    got, b = [], 0
    while b < m:
        e = ddm.ddm_chunk_end_ordered(ctx, b, cap)
        assert e > b and ooff[e] - ooff[b] <= cap and (e == m or ooff[e + 1] - ooff[b] > cap)
        k = ddm.ddm_write_ordered(ctx, b, e, buf)
        assert k == ooff[e] - ooff[b]
        got.append(buf[:k].cpu().numpy().view(np.uint32).copy())
        b = e
    got = np.concatenate(got)
    # grouped by update in plan order, same pairs as the one-shot match
    assert np.array_equal(got[:, 0], np.repeat(order, np.diff(ooff)).astype(np.uint32))
    assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(pu, ps)))
    # each update's list is identical (same order) in both layouts
    j = int(order[len(order) // 2])
    sel = got[:, 0] == j
    assert np.array_equal(got[sel, 1], ps[off[j]:off[j + 1]])
    # compressed output (Section III): the subscription ids alone, same chunks
    # and same positions; with order and ooff it is M stored by columns
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    got_ids, b = [], 0
    while b < m:
        e = ddm.ddm_chunk_end_ordered(ctx, b, cap)
        k = ddm.ddm_write_ordered_ids(ctx, b, e, ids)
        assert k == ooff[e] - ooff[b]
        got_ids.append(ids[:k].cpu().numpy().view(np.uint32).copy())
        b = e
    got_ids = np.concatenate(got_ids)
    assert np.array_equal(got_ids, got[:, 1])
    cols = np.repeat(order, np.diff(ooff)).astype(np.uint32)
    _, ou, os_ = oracle.itm_pairs(*arrays, flags=flags)
    assert np.array_equal(np.sort(keys(cols, got_ids)), np.sort(keys(ou, os_)))


def test_replay_and_walking_write_agree(ctx):
    """The write pass expands the count pass's records when they fit the
    record budget and walks the tree otherwise; both give the same list."""
    import torch
    arrays = W.clustered_lognormal(30000, 25000, d=3, alpha=100.0, seed=21)
    U = to_dev(arrays)
    results = []
    fresh = ddm.ddm_create(0)
    try:
        for budget in (None, 0, 1 << 16):
            if budget is not None:
                ddm.ddm_set_replay_budget(fresh, budget)
            for rep in range(2):     # the second plan uses the first one's size hint
                K = ddm.ddm_count(fresh, *U)
                pairs = torch.empty((K, 2), dtype=torch.int32, device="cuda")
                assert ddm.ddm_match(fresh, *U, pairs) == K
                full = pairs.cpu().numpy().view(np.uint32).copy()
                ddm.ddm_build(fresh, U[2], U[3])
                ddm.ddm_plan(fresh, U[0], U[1])
                ooff = torch.empty(25001, dtype=torch.int64, device="cuda")
                ddm.ddm_plan_order(fresh, None, ooff)
                torch.cuda.synchronize()
                ooff = ooff.cpu().numpy()
                a, b = 777, 20001            # a range that starts and ends inside packets
                part = torch.empty((int(ooff[b] - ooff[a]), 2), dtype=torch.int32, device="cuda")
                assert ddm.ddm_write_ordered(fresh, a, b, part) == ooff[b] - ooff[a]
                part_ids = torch.empty(int(ooff[b] - ooff[a]), dtype=torch.int32, device="cuda")
                assert ddm.ddm_write_ordered_ids(fresh, a, b, part_ids) == ooff[b] - ooff[a]
                assert torch.equal(part_ids, part[:, 1])
                sub = torch.empty((K, 2), dtype=torch.int32, device="cuda")
                ks = ddm.ddm_write(fresh, 3000, 9000, sub)
                results.append((full, part.cpu().numpy().copy(), sub[:ks].cpu().numpy().copy()))
    finally:
        ddm.ddm_destroy(fresh)
    for r in results[1:]:
        for x, y in zip(results[0], r):
            assert np.array_equal(x, y)
    Ko, ou, os_ = oracle.itm_pairs(*arrays)
    full = results[0][0]
    assert np.array_equal(full[:, 0], ou)
    assert np.array_equal(np.sort(keys(full[:, 0], full[:, 1])), np.sort(keys(ou, os_)))


@pytest.mark.parametrize("wide", [1, 16])
def test_replay_record_counts_at_block_limits(ctx, wide):
    """Records carry their query's matches since the start of their block in
    16 bits, above a per-block header.  One query (wide = 1) meeting all of
    40,000 points fills whole 512-record blocks of 32-hit records alone, so
    the count reaches 511 x 32 in each block; sixteen such queries (wide =
    16) share every block.  Pairs and compressed ids against the oracle."""
    import torch
    n = 40000
    slo = np.arange(n, dtype=np.float32)[None, :].copy()
    shi = slo.copy()
    m = 40
    ulo = np.full((1, m), 2e6, np.float32)     # lanes past `wide` meet nothing
    uhi = np.full((1, m), 2e6, np.float32)
    ulo[0, :wide] = -1.0 - np.arange(wide, dtype=np.float32)
    uhi[0, :wide] = 1e6
    arrays = (ulo, uhi, slo, shi)
    K, pu, ps = gpu_match(ctx, arrays)
    Ko, ou, os_ = oracle.itm_pairs(*arrays)
    assert K == Ko == wide * n
    assert np.array_equal(pu, ou) and np.array_equal(ps, os_)
    U = to_dev(arrays)
    ddm.ddm_build(ctx, U[2], U[3])
    assert ddm.ddm_plan(ctx, U[0], U[1]) == K
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    ooff = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    ddm.ddm_plan_order(ctx, order, ooff)
    ids = torch.empty(K, dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered_ids(ctx, 0, m, ids) == K
    order = order.cpu().numpy()
    ooff = ooff.cpu().numpy()
    ids = ids.cpu().numpy().view(np.uint32)
    for p in range(m):
        u = order[p]
        assert np.array_equal(ids[ooff[p]:ooff[p + 1]], os_[ou == u])


# --- error paths -------------------------------------------------------------

def test_invalid_extents(ctx):
    base = W.uniform_fixed_length(500, 400, 2, 10.0, seed=2)
    for which, idx, val in ((0, (1, 17), np.nan), (1, (0, 3), -1.0), (2, (1, 499), np.nan),
                            (3, (0, 0), -5.0)):
        arrays = [a.copy() for a in base]
        arrays[which][idx] = val
        U = to_dev(arrays)
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_count(ctx, *U)
        assert e.value.code == ddm.DDM_ERR_EXTENT
    # the context stays usable
    check_exact(ctx, base)


def test_compressed_output_edges(ctx):
    """Compressed output: empty ranges write nothing (a buffer is not even
    needed), single plan positions at packet boundaries equal the matching
    slice of a whole write, and bad ranges are refused."""
    import torch
    arrays = W.uniform_fixed_length(5000, 4000, 2, 10.0, seed=7)
    U = to_dev(arrays)
    m = 4000
    ddm.ddm_build(ctx, U[2], U[3])
    K = ddm.ddm_plan(ctx, U[0], U[1])
    ooff = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    ddm.ddm_plan_order(ctx, None, ooff)
    torch.cuda.synchronize()
    ooff = ooff.cpu().numpy()
    ids = torch.full((K + 8,), -7, dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered_ids(ctx, 100, 100, ids) == 0
    assert ddm.ddm_write_ordered_ids(ctx, m, m, None) == 0
    assert bool((ids == -7).all())
    full = torch.empty(K, dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered_ids(ctx, 0, m, full) == K
    for p in (0, 31, 32, 33, 2047, m - 1):
        k = ddm.ddm_write_ordered_ids(ctx, p, p + 1, ids)
        assert k == ooff[p + 1] - ooff[p]
        assert torch.equal(ids[:k], full[int(ooff[p]):int(ooff[p + 1])])
    for b, e in ((10, 5), (0, m + 1)):
        with pytest.raises(ddm.DDMError) as err:
            ddm.ddm_write_ordered_ids(ctx, b, e, ids)
        assert err.value.code == ddm.DDM_ERR_ARG


def test_capacity_and_state_errors(ctx):
    import torch
    arrays = W.uniform_fixed_length(3000, 3000, 1, 50.0, seed=3)
    U = to_dev(arrays)
    K = ddm.ddm_count(ctx, *U)
    small = torch.full((K - 1, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_match(ctx, *U, small)
    assert e.value.code == ddm.DDM_ERR_CAPACITY and e.value.k == K
    assert (small == -1).all()          # nothing written when it does not fit
    fresh = ddm.ddm_create(0)
    try:
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_plan(fresh, U[0], U[1])
        assert e.value.code == ddm.DDM_ERR_STATE
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_write(fresh, 0, 1, small)
        assert e.value.code == ddm.DDM_ERR_STATE
        small_ids = torch.full((K - 1,), -1, dtype=torch.int32, device="cuda")
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_write_ordered_ids(fresh, 0, 1, small_ids)
        assert e.value.code == ddm.DDM_ERR_STATE
        ddm.ddm_debug_set_alloc_limit(fresh, 1 << 16)
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_count(fresh, *U)
        assert e.value.code == ddm.DDM_ERR_NOMEM
        ddm.ddm_debug_set_alloc_limit(fresh, 0)
        assert ddm.ddm_count(fresh, *U) == K
        ddm.ddm_build(fresh, U[2], U[3])
        assert ddm.ddm_plan(fresh, U[0], U[1]) == K
        with pytest.raises(ddm.DDMError) as e:
            ddm.ddm_write_ordered_ids(fresh, 0, 3000, small_ids)
        assert e.value.code == ddm.DDM_ERR_CAPACITY and e.value.k == K
        assert (small_ids == -1).all()  # nothing written when it does not fit
    finally:
        ddm.ddm_destroy(fresh)
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_match_range(ctx, *U, 10, 5, small)
    assert e.value.code == ddm.DDM_ERR_ARG
    bad = to_dev([np.zeros((9, 4), np.float32)] * 4)
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_count(ctx, *bad)
    assert e.value.code == ddm.DDM_ERR_ARG


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("flags", [0, 1])
def test_swap_roles_same_pairs(ctx, d, flags):
    """DDM_SWAP_ROLES (tree over the updates, one query per subscription;
    Section IV lets the tree be built over either set) reports the same pair
    set, grouped by subscription id."""
    import torch
    for n, m, seed in ((2500, 400, 3), (300, 3100, 4)):
        arrays = W.uniform_fixed_length(n, m, d, 40.0, seed=seed)
        if seed == 4:   # ties and infinities in the mix
            g = W.grid_random(n, m, d, seed=seed, grid=7)
            arrays = g
            arrays[3][0, :5] = np.inf
            arrays[0][0, :5] = -np.inf
        U = to_dev(arrays)
        K = ddm.ddm_count(ctx, *U, flags=flags)
        Ks = ddm.ddm_count(ctx, *U, flags=flags | ddm.DDM_SWAP_ROLES)
        assert Ks == K
        pairs = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
        assert ddm.ddm_match(ctx, *U, pairs, flags=flags | ddm.DDM_SWAP_ROLES) == K
        got = pairs[:K].cpu().numpy().view(np.uint32)
        assert (np.diff(got[:, 1].astype(np.int64)) >= 0).all()   # grouped by subscription
        Ko, ou, os_ = oracle.itm_pairs(*arrays, flags=flags)
        assert Ko == K
        assert np.array_equal(np.sort(keys(got[:, 0], got[:, 1])), np.sort(keys(ou, os_)))


def test_swap_roles_limits(ctx):
    import torch
    arrays = W.uniform_fixed_length(500, 300, 2, 10.0, seed=9)
    U = to_dev(arrays)
    pairs = torch.empty((1 << 16, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ddm.DDMError) as e:   # a partial update range has no meaning swapped
        ddm.ddm_match_range(ctx, *U, 10, 20, pairs, flags=ddm.DDM_SWAP_ROLES)
    assert e.value.code == ddm.DDM_ERR_ARG
    K = ddm.ddm_match_range(ctx, *U, 0, 300, pairs, flags=ddm.DDM_SWAP_ROLES)
    replayed = pairs[:K].cpu().numpy().copy()
    other = ddm.ddm_create(0)
    try:   # the walking write pass (no record arena) swaps the same way
        ddm.ddm_set_replay_budget(other, 0)
        assert ddm.ddm_match(other, *U, pairs, flags=ddm.DDM_SWAP_ROLES) == K
        assert np.array_equal(pairs[:K].cpu().numpy(), replayed)
    finally:
        ddm.ddm_destroy(other)
    with pytest.raises(ddm.DDMError) as e:   # the swapped tree is not left for staged calls
        ddm.ddm_plan(ctx, U[0], U[1])
    assert e.value.code == ddm.DDM_ERR_STATE
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_plan(ctx, U[0], U[1], flags=ddm.DDM_SWAP_ROLES)
    assert e.value.code in (ddm.DDM_ERR_ARG, ddm.DDM_ERR_STATE)


def test_plan_stats_bounds(ctx):
    """ddm_plan_stats: every pair comes from a (query, leaf) test (<= 32 per
    test), and no query tests more leaves than the tree has."""
    import math
    for d, (n, m) in ((1, (5000, 4000)), (3, (20000, 9000))):
        arrays = W.uniform_fixed_length(n, m, d, 50.0, seed=11)
        U = to_dev(arrays)
        K = ddm.ddm_count(ctx, *U)
        t = ddm.ddm_plan_stats(ctx)
        assert K <= 32 * t
        assert t <= m * math.ceil(n / 32)
        assert t > 0


@pytest.mark.parametrize("flags", [0, 1])
def test_maximum_dimensions(ctx, flags):
    """d = DDM_MAX_DIMS (8): the runtime-d kernels at their limit, ties and
    touching faces in every dimension."""
    for seed in range(4):
        rng = np.random.default_rng(77 + seed)
        n, m = (int(v) for v in rng.integers(1, 400, size=2))
        check_exact(ctx, W.grid_random(n, m, 8, seed=seed, grid=3), flags)
    check_exact(ctx, W.uniform_fixed_length(3000, 2000, 8, 5.0, seed=3), flags)


def test_size_and_dimension_limits(ctx):
    """Counts above DDM_MAX_EXTENTS and d outside 1..8 are refused on the
    host, before any device work (the pointers are never read)."""
    import ctypes
    import torch
    lib = ddm.lib()
    lo = torch.zeros((2, 4), device="cuda")
    k = ctypes.c_uint64(0)
    p = lo.data_ptr()
    big = 1073741824  # DDM_MAX_EXTENTS + 1
    s = torch.cuda.current_stream().cuda_stream
    assert lib.ddm_count(ctx, 2, p, p, big, p, p, 4, 0, ctypes.byref(k), s) == ddm.DDM_ERR_ARG
    assert lib.ddm_count(ctx, 2, p, p, 4, p, p, big, 0, ctypes.byref(k), s) == ddm.DDM_ERR_ARG
    assert lib.ddm_count(ctx, 9, p, p, 4, p, p, 4, 0, ctypes.byref(k), s) == ddm.DDM_ERR_ARG
    assert lib.ddm_count(ctx, 0, p, p, 4, p, p, 4, 0, ctypes.byref(k), s) == ddm.DDM_ERR_ARG
    assert lib.ddm_count(ctx, 2, p, p, 4, p, p, 4, 8, ctypes.byref(k), s) == ddm.DDM_ERR_ARG  # flag
    # the context is still usable
    check_exact(ctx, W.uniform_fixed_length(300, 200, 2, 10.0, seed=1))


def test_bounded_wait_times_out_and_context_survives(ctx):
    """Failure detection without a GPU fault: a bounded device wait on a word
    that nothing sets (the sort's look-back poll) gives up, the host reads
    DDM_ERR_TIMEOUT, and the context keeps working."""
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_debug_wait_timeout(ctx, 1 << 14)
    assert e.value.code == ddm.DDM_ERR_TIMEOUT
    check_exact(ctx, W.uniform_fixed_length(5000, 4000, 2, 10.0, seed=3))
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_debug_wait_timeout(ctx, 0)
    assert e.value.code == ddm.DDM_ERR_ARG
