"""Pins for the CPU oracle (no GPU).

Each check fixes the oracle against something other than itself: values
the paper states (the Fig. 1 example), closed-form counts, an independent
counting algorithm (BITS), brute force against the interval tree on tiny
inputs where ties are frequent, and invariants of the problem statement.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1309_3458_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pairset(pu, ps):
    return np.sort(pu.astype(np.uint64) << np.uint64(32) | ps.astype(np.uint64))


# --- Alg. 1 -----------------------------------------------------------------

@pytest.mark.parametrize("x,y,closed,open_", [
    ((0, 1), (2, 3), False, False),    # disjoint
    ((0, 2), (1, 3), True, True),      # proper overlap
    ((0, 1), (1, 2), True, False),     # touching endpoints
    ((1, 1), (1, 1), True, False),     # two degenerate segments at one point
    ((1, 1), (0, 2), True, True),      # degenerate inside another segment
    ((0, 2), (2, 2), True, False),     # degenerate on an endpoint
    ((0, 5), (1, 2), True, True),      # containment
    ((3, 4), (0, 2), False, False),    # disjoint, other side
])
def test_intersect_1d(x, y, closed, open_):
    # Alg. 1 is printed with strict comparisons (the OPEN rule); segments are
    # written [low, high], read as closed by default.
    assert oracle.intersect_1d(*x, *y, 0) == closed
    assert oracle.intersect_1d(*y, *x, 0) == closed          # symmetric
    assert oracle.intersect_1d(*x, *y, oracle.OPEN) == open_
    assert oracle.intersect_1d(*y, *x, oracle.OPEN) == open_


# --- closed forms on the unit lattice ---------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_lattice_closed_forms(d, k):
    # Subscriptions [i, i+1], updates [j, j+1] per dimension: closed rule
    # matches |i - j| <= 1 in every dimension, (3k - 2)^d pairs; open rule
    # needs i == j, k^d pairs.  Updates shifted by 1/2 match j in {i-1, i}
    # under either rule: (2k - 1)^d pairs.
    u = W.lattice(k, d)
    s = W.lattice(k, d, shift_half=True)
    for arrays, flags, want in ((u, 0, (3 * k - 2) ** d), (u, oracle.OPEN, k ** d),
                                (s, 0, (2 * k - 1) ** d), (s, oracle.OPEN, (2 * k - 1) ** d)):
        K_bf, c_bf, _, _, _ = oracle.bf(*arrays, flags=flags, pairs=False)
        K_itm, c_itm, _ = oracle.itm_count(*arrays, flags=flags)
        assert K_bf == want and K_itm == want
        assert np.array_equal(c_bf, c_itm)
        if d == 1 and flags == 0:
            K_bits, c_bits = oracle.bits_count(*arrays)
            assert K_bits == want and np.array_equal(c_bits, c_bf)


def test_lattice_per_update_counts_d2():
    # Per update on the unshifted lattice (closed): (number of neighbours
    # within distance 1 per axis) multiplied over axes; corner updates see 2x2.
    k = 5
    K, counts, _, _, _ = oracle.bf(*W.lattice(k, 2), pairs=False)
    grid = counts.reshape(k, k)
    per_axis = np.array([2] + [3] * (k - 2) + [2])
    assert np.array_equal(grid, np.outer(per_axis, per_axis))


# --- Fig. 1 worked example ---------------------------------------------------

def load_fig1():
    S, U, M, P = {}, {}, [], []
    with open(os.path.join(GOLDEN, "fig1_example.txt")) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] in ("S", "U"):
                (S if t[0] == "S" else U)[int(t[1])] = [float(v) for v in t[2:]]
            elif t[0] == "M":
                M.append([int(v) for v in t[1:]])
            elif t[0] == "P":
                P.append([int(v) for v in t[1:]])

    def soa(D):
        ids = sorted(D)
        lo = np.array([[D[i][2 * k] for i in ids] for k in range(2)], np.float32)
        hi = np.array([[D[i][2 * k + 1] for i in ids] for k in range(2)], np.float32)
        return lo, hi

    ulo, uhi = soa(U)
    slo, shi = soa(S)
    return (ulo, uhi, slo, shi), np.array(M), P


@pytest.mark.parametrize("flags", [0, 1])
def test_fig1_worked_example(flags):
    arrays, M, P = load_fig1()
    n, m = M.shape
    for K, pu, ps in (oracle.bf(*arrays, flags=flags)[0:1] + oracle.bf(*arrays, flags=flags)[3:5],
                      oracle.itm_pairs(*arrays, flags=flags)):
        got = np.zeros((n, m), int)
        got[ps, pu] = 1
        assert np.array_equal(got, M)
        assert K == M.sum()
    # the per-dimension statement about S1 and U2
    ulo, uhi, slo, shi = arrays
    for s_id, u_id, want0, want1 in P:
        i, j = s_id - 1, u_id - 1
        for k, want in ((0, want0), (1, want1)):
            assert oracle.intersect_1d(slo[k, i], shi[k, i], ulo[k, j], uhi[k, j], flags) == bool(want)


# --- brute force against the interval tree on tiny grids --------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("flags", [0, 1])
def test_bf_equals_itm_on_grids(d, flags):
    for seed in range(12):
        rng = np.random.default_rng(seed)
        n, m = (int(v) for v in rng.integers(0, 65, size=2))
        arrays = W.grid_random(n, m, d, seed=seed)
        K1, c1, g1, pu1, ps1 = oracle.bf(*arrays, flags=flags)
        K2, pu2, ps2 = oracle.itm_pairs(*arrays, flags=flags)
        K3, c3, g3 = oracle.itm_count(*arrays, flags=flags, threads=3)
        assert K1 == K2 == K3
        assert np.array_equal(pairset(pu1, ps1), pairset(pu2, ps2))
        assert np.array_equal(c1, c3) and np.array_equal(g1, g3)
        # within one update the tree reports in tree order, i.e. sorted by
        # (lower, upper, id) of dimension 0
        _, slo, shi = arrays[0], arrays[2], arrays[3]
        for j in range(m):
            sel = ps2[pu2 == j]
            keys = list(zip(slo[0, sel], shi[0, sel], sel))
            assert keys == sorted(keys)


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (2, 100.0), (2, 1.0), (3, 100.0)])
def test_bf_equals_itm_uniform(d, alpha):
    arrays = W.uniform_fixed_length(700, 900, d, alpha, seed=3)
    K1, c1, g1, pu1, ps1 = oracle.bf(*arrays)
    K2, pu2, ps2 = oracle.itm_pairs(*arrays)
    assert K1 == K2 > 0
    assert np.array_equal(pairset(pu1, ps1), pairset(pu2, ps2))


def test_bf_equals_itm_clustered():
    arrays = W.clustered_lognormal(1500, 1200, d=3, alpha=100.0, seed=5)
    K1, c1, g1, _, _ = oracle.bf(*arrays, pairs=False)
    K2, c2, g2 = oracle.itm_count(*arrays, threads=4)
    assert K1 == K2 > 0
    assert np.array_equal(c1, c2) and np.array_equal(g1, g2)
    assert (arrays[0] < 0).any()          # negative lower bounds occur


# --- BITS (Section II) --------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.01, 1.0, 100.0])
def test_bits_equals_itm_d1(alpha):
    arrays = W.uniform_fixed_length(3000, 2500, 1, alpha, seed=11)
    K1, c1 = oracle.bits_count(*arrays)
    K2, c2, _ = oracle.itm_count(*arrays, threads=4)
    assert K1 == K2 and np.array_equal(c1, c2)


def test_bits_equals_itm_grid_ties():
    for seed in range(8):
        arrays = W.grid_random(200, 150, 1, seed=100 + seed, grid=6)
        assert np.array_equal(oracle.bits_count(*arrays)[1], oracle.itm_count(*arrays)[1])


def test_degenerate_float32_extents():
    # At alpha = 0.01 with N = 1e6 the length (0.01) is below the float32
    # spacing near 1e6, so many extents collapse to a point (hi == lo).
    ulo, uhi, slo, shi = W.make("uniform_d1_N1e6_a0.01")
    assert 0.6 < (uhi == ulo).mean() < 0.9
    a = tuple(np.ascontiguousarray(x[:, :20000]) for x in (ulo, uhi, slo, shi))
    assert np.array_equal(oracle.bits_count(*a)[1], oracle.itm_count(*a)[1])


# --- invariants of the problem statement ------------------------------------

def test_invariants():
    ulo, uhi, slo, shi = W.uniform_fixed_length(400, 300, 2, 50.0, seed=7)
    K, pu, ps = oracle.itm_pairs(ulo, uhi, slo, shi)
    base = set(zip(pu.tolist(), ps.tolist()))
    # swapping the roles of S and U transposes the pair set
    K2, pu2, ps2 = oracle.itm_pairs(slo, shi, ulo, uhi)
    assert set(zip(ps2.tolist(), pu2.tolist())) == base
    # permuting the inputs relabels the ids
    rng = np.random.default_rng(0)
    pu_perm, ps_perm = rng.permutation(300), rng.permutation(400)
    K3, pu3, ps3 = oracle.itm_pairs(np.ascontiguousarray(ulo[:, pu_perm]),
                                    np.ascontiguousarray(uhi[:, pu_perm]),
                                    np.ascontiguousarray(slo[:, ps_perm]),
                                    np.ascontiguousarray(shi[:, ps_perm]))
    assert set(zip(pu_perm[pu3].tolist(), ps_perm[ps3].tolist())) == base
    # scaling every coordinate by 2 (exact in float32) changes nothing
    two = np.float32(2)
    K4, pu4, ps4 = oracle.itm_pairs(ulo * two, uhi * two, slo * two, shi * two)
    assert set(zip(pu4.tolist(), ps4.tolist())) == base
    # growing an extent only adds pairs
    K5, pu5, ps5 = oracle.itm_pairs(ulo, uhi + np.float32(1000), slo, shi)
    assert base <= set(zip(pu5.tolist(), ps5.tolist())) and K5 > K


# --- tree order ----------------------------------------------------------------

def test_tree_order_and_height():
    arrays = W.grid_random(3000, 1, 1, seed=2, grid=40)
    slo, shi = arrays[2][0], arrays[3][0]
    order, h = oracle.tree_order(slo, shi)
    ids = np.arange(3000)
    assert np.array_equal(order, np.lexsort((ids, shi, slo)))
    # AVL height bound: h < 1.4405 log2(n + 2) - 0.3277
    assert h < 1.4405 * math.log2(3000 + 2) - 0.3277


def test_negative_zero_orders_with_zero():
    # -0.0 and +0.0 compare equal, so the upper bound (then id) decides.
    lo = np.array([0.0, -0.0, 0.0, -0.0], np.float32)
    hi = np.array([2.0, 1.0, 1.0, 3.0], np.float32)
    order, _ = oracle.tree_order(lo, hi)
    assert order.tolist() == [1, 2, 0, 3]


# --- statistical sanity (soft) -----------------------------------------------

def test_expected_pair_count_uniform():
    # Closed rule, lower bounds uniform on [0, W], W = L - l: a pair overlaps
    # on one axis with probability p = 2l/W - (l/W)^2; E[K] = n m p^d.
    for d, alpha in ((1, 1.0), (2, 100.0)):
        n = m = 2000
        ulo, uhi, slo, shi = W.uniform_fixed_length(n, m, d, alpha, seed=21)
        l = W.fixed_length(n + m, d, alpha)
        Wd = W.ROUTING_L - l
        p = 2 * l / Wd - (l / Wd) ** 2
        want = n * m * p ** d
        K, _, _ = oracle.itm_count(ulo, uhi, slo, shi, threads=4)
        assert abs(K - want) < 0.1 * want
