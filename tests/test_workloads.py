"""The seeded input recipes (CPU): the synthetic workloads that stand in for
the paper's experiments (Section V) have the sizes, distributions and
overlap degrees their docstrings state.  These generators feed both the
oracle and the GPU path, so a drift here would silently change every
benchmark and parity case."""
import math

import numpy as np
import pytest

from paper_1309_3458_gb300 import workloads as W


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fixed_length_overlap_degree(d):
    """alpha = N * l^d / L^d; for d = 1 the paper's l = alpha * L / N."""
    for N, alpha in ((10_000, 1.0), (1_000_000, 0.01), (1_000_000, 100.0)):
        l = W.fixed_length(N, d, alpha)
        assert N * l ** d / W.ROUTING_L ** d == pytest.approx(alpha, rel=1e-12)
    assert W.fixed_length(10_000, 1, 1.0) == pytest.approx(100.0)


def test_uniform_fixed_length_recipe():
    ulo, uhi, slo, shi = W.uniform_fixed_length(3000, 2000, 2, 1.0, seed=3)
    assert ulo.shape == uhi.shape == (2, 2000) and slo.shape == shi.shape == (2, 3000)
    assert all(a.dtype == np.float32 and a.flags.c_contiguous for a in (ulo, uhi, slo, shi))
    l32 = np.float32(W.fixed_length(5000, 2, 1.0))
    # upper bound = fl32(lower + fl32(l)), bit for bit
    assert np.array_equal(uhi, ulo + l32) and np.array_equal(shi, slo + l32)
    L = W.ROUTING_L
    for lo in (ulo, slo):
        assert lo.min() >= 0.0 and lo.max() <= np.float32(L - float(l32))
        # uniform: every quarter of [0, L - l] holds about a quarter of them
        q = np.histogram(lo.ravel(), bins=4, range=(0.0, L - float(l32)))[0] / lo.size
        assert np.all(np.abs(q - 0.25) < 0.03)
    again = W.uniform_fixed_length(3000, 2000, 2, 1.0, seed=3)
    other = W.uniform_fixed_length(3000, 2000, 2, 1.0, seed=4)
    assert all(np.array_equal(a, b) for a, b in zip((ulo, uhi, slo, shi), again))
    assert not np.array_equal(ulo, other[0])


def test_clustered_lognormal_recipe():
    n = m = 100_000
    d, alpha = 3, 100.0
    ulo, uhi, slo, shi = W.clustered_lognormal(n, m, d, alpha, seed=0)
    L = W.ROUTING_L
    lo = np.concatenate([ulo, slo], axis=1).astype(np.float64)
    hi = np.concatenate([uhi, shi], axis=1).astype(np.float64)
    assert np.all(hi >= lo)
    # mean overlap degree: N * mean volume / L^d = alpha (volume is a product
    # of three log-normals, sigma^2 = 3 in all: ~1% relative error here)
    vol = np.prod(hi - lo, axis=0)
    assert (n + m) * vol.mean() / L ** d == pytest.approx(alpha, rel=0.05)
    # per-dimension lengths are log-normal with sigma = 1 and the stated mu
    mu = (math.log(alpha * L ** d / (n + m)) - d / 2.0) / d
    logs = np.log(hi - lo)
    assert abs(logs.mean() - mu) < 0.02 and abs(logs.std() - 1.0) < 0.02
    # centres clipped to [0, L) (extents are not clipped: some lower bounds < 0)
    c = (lo + hi) / 2
    assert c.min() > -1.0 and c.max() < L + 1.0
    assert lo.min() < 0.0
    # clustered: 64 Gaussian clusters of sigma 0.02 L leave most of the space empty
    cells = np.floor(np.clip(c, 0, L - 1) / (L / 10)).astype(int)
    occupied = len(np.unique(cells[0] * 100 + cells[1] * 10 + cells[2]))
    assert occupied < 0.5 * 1000


def test_batched_sizes_log_uniform():
    s = W.batched_sizes(4096, 100, 100_000, seed=0)
    assert s.min() >= 100 and s.max() < 100_000 and s.dtype == np.int64
    logs = np.log(s + 0.5)
    # log-uniform: mean of the logs at the midpoint, quarters equally full
    mid = (math.log(100) + math.log(100_000)) / 2
    assert abs(logs.mean() - mid) < 0.1
    q = np.histogram(logs, bins=4, range=(math.log(100), math.log(100_000)))[0] / s.size
    assert np.all(np.abs(q - 0.25) < 0.04)
    inst = W.batched_instances(count=8, seed=0)
    assert [a[0].shape[1] + a[2].shape[1] for a in inst] == list(W.batched_sizes(8, 100, 100_000, 0))


def test_named_configs():
    assert set(W.CONFIGS) == {"uniform_d1_N1e4_a1", "clustered_d3_N1e7_a100"} | {
        f"uniform_d{d}_N1e6_a{a}" for d in (1, 2) for a in ("0.01", "1", "100")}
    ulo, uhi, slo, shi = W.make("uniform_d1_N1e4_a1")
    assert ulo.shape == (1, 5000) and slo.shape == (1, 5000)
    assert np.allclose(uhi - ulo, 1.0 * W.ROUTING_L / 10_000, rtol=1e-3)
    small = W.make("clustered_d3_N1e7_a100", scale=0.001)
    assert small[0].shape == (3, 5000) and small[2].shape == (3, 5000)
