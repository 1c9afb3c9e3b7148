"""Seeded synthetic workloads shaped like the paper's experiments (Section V).

This module only draws inputs. It holds none of the matching arithmetic, so
both the CUDA path and the CPU oracle may consume what it produces.

Every generator returns ``(upd_lo, upd_hi, sub_lo, sub_hi)``: float32 arrays of
shape ``(d, m)`` / ``(d, n)``, C-contiguous, i.e. the structure-of-arrays
layout of the library boundary (row ``k`` holds dimension ``k``).

Coordinates are produced in float32 arithmetic and the saved bytes *are* the
problem: an upper bound is ``fl32(lo + fl32(l))`` (round to nearest), so both
sides compare exactly the same numbers.

Workloads
---------
* ``uniform_fixed_length`` -- Section V: extents placed uniformly at random
  on a routing space of side ``L`` = 1e6, all with the same length ``l``.
  The overlapping degree is the summed extent volume over the routing-space
  volume; for ``d = 1`` that gives ``l = alpha * L / N``.  For ``d > 1`` the
  paper gives no definition; the reading used here keeps the same ratio of
  volumes, ``l = L * (alpha / N) ** (1 / d)`` per dimension.
* ``clustered_lognormal`` -- a large-output stress case in ``d`` dimensions:
  centres drawn from an equal-weight mixture of isotropic Gaussians clipped
  to the routing space, per-dimension lengths log-normal with the log-mean
  chosen so that the expected overlapping degree is ``alpha``.
* ``lattice`` -- unit extents on an integer lattice, whose pair counts have a
  closed form (used to pin the oracle).
* ``batched_instances`` -- many independent uniform problems of log-uniform
  size.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

ROUTING_L = 1.0e6

Arrays = Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def fixed_length(N: int, d: int, alpha: float, L: float = ROUTING_L) -> float:
    """Per-dimension extent length for overlapping degree ``alpha``.

    ``alpha = N * l**d / L**d`` (summed volume over routing-space volume);
    for ``d = 1`` this is the paper's ``l = alpha * L / N``.
    """
    return L * (alpha / N) ** (1.0 / d)


def _upper(lo: np.ndarray, l32: np.float32) -> np.ndarray:
    hi = lo + l32  # float32 + float32, rounded to nearest by numpy
    assert hi.dtype == np.float32
    return hi


def uniform_fixed_length(n: int, m: int, d: int, alpha: float, seed: int,
                         L: float = ROUTING_L) -> Arrays:
    """Uniformly placed, equal-length extents (Section V workload).

    Draw order: subscription lower bounds (d x n), then update lower bounds
    (d x m), each ``uniform(0, L - l)`` in float64 and rounded to float32.
    """
    N = n + m
    l = fixed_length(N, d, alpha, L)
    l32 = np.float32(l)
    rng = _rng(seed)
    sub_lo = rng.uniform(0.0, L - l, size=(d, n)).astype(np.float32)
    upd_lo = rng.uniform(0.0, L - l, size=(d, m)).astype(np.float32)
    return (np.ascontiguousarray(upd_lo), np.ascontiguousarray(_upper(upd_lo, l32)),
            np.ascontiguousarray(sub_lo), np.ascontiguousarray(_upper(sub_lo, l32)))


def clustered_lognormal(n: int, m: int, d: int = 3, alpha: float = 100.0,
                        seed: int = 0, n_clusters: int = 64,
                        sigma_frac: float = 0.02, ln_sigma: float = 1.0,
                        L: float = ROUTING_L) -> Arrays:
    """Gaussian-mixture centres with log-normal per-dimension lengths.

    * ``n_clusters`` centres uniform in ``[0, L)^d``;
    * each extent picks a centre uniformly, adds ``N(0, (sigma_frac*L)^2)``
      per axis and is clipped to ``[0, nextafter(L, 0)]`` (float64), then
      rounded to float32;
    * lengths are log-normal with ``sigma = ln_sigma`` and
      ``mu = (ln(alpha * L**d / N) - d * sigma**2 / 2) / d``, so that the mean
      volume times ``N`` is ``alpha * L**d``;
    * ``lo = fl32(c - l/2)``, ``hi = fl32(c + l/2)``; the extents themselves
      are not clipped, so lower bounds can be negative.

    Draw order: centres, then subscriptions (cluster index, offsets,
    lengths), then updates in the same order.
    """
    N = n + m
    mu = (math.log(alpha * L ** d / N) - d * ln_sigma ** 2 / 2.0) / d
    rng = _rng(seed)
    centres = rng.uniform(0.0, L, size=(n_clusters, d))
    top = np.nextafter(L, 0.0)

    def one_set(size: int):
        which = rng.integers(0, n_clusters, size=size)
        c = centres[which] + rng.normal(0.0, sigma_frac * L, size=(size, d))
        np.clip(c, 0.0, top, out=c)
        c32 = np.ascontiguousarray(c.T).astype(np.float32)
        del c
        lens = rng.lognormal(mu, ln_sigma, size=(size, d))
        h32 = np.ascontiguousarray(lens.T).astype(np.float32) * np.float32(0.5)
        del lens
        lo = c32 - h32
        hi = c32 + h32
        return np.ascontiguousarray(lo), np.ascontiguousarray(hi)

    sub_lo, sub_hi = one_set(n)
    upd_lo, upd_hi = one_set(m)
    return upd_lo, upd_hi, sub_lo, sub_hi


def lattice(k: int, d: int, shift_half: bool = False) -> Arrays:
    """Unit extents on a product lattice.

    Subscriptions are ``[i, i+1]`` and updates ``[j, j+1]`` (or
    ``[j+1/2, j+3/2]`` with ``shift_half``) for ``i, j`` in ``0..k-1`` in every
    dimension, enumerated as the product lattice in row-major order
    (dimension 0 varies slowest).  ``k**d`` extents per set.
    """
    axes = np.meshgrid(*([np.arange(k, dtype=np.float64)] * d), indexing="ij")
    pts = np.stack([a.reshape(-1) for a in axes]).astype(np.float32)  # (d, k^d)
    sub_lo = np.ascontiguousarray(pts)
    sub_hi = np.ascontiguousarray(pts + np.float32(1.0))
    off = np.float32(0.5 if shift_half else 0.0)
    upd_lo = np.ascontiguousarray(pts + off)
    upd_hi = np.ascontiguousarray(pts + off + np.float32(1.0))
    return upd_lo, upd_hi, sub_lo, sub_hi


def grid_random(n: int, m: int, d: int, seed: int, grid: int = 8) -> Arrays:
    """Tiny integer-grid extents (coordinates in ``0..grid-1``) so that shared
    and touching endpoints are frequent; degenerate ``[a, a]`` extents occur."""
    rng = _rng(seed)

    def one(size):
        a = rng.integers(0, grid, size=(d, size))
        b = rng.integers(0, grid, size=(d, size))
        lo = np.minimum(a, b).astype(np.float32)
        hi = np.maximum(a, b).astype(np.float32)
        return np.ascontiguousarray(lo), np.ascontiguousarray(hi)

    sub_lo, sub_hi = one(n)
    upd_lo, upd_hi = one(m)
    return upd_lo, upd_hi, sub_lo, sub_hi


def batched_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` instance sizes ``floor(exp(U[ln lo, ln hi]))``."""
    rng = _rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batched_instances(count: int = 4096, d: int = 2, alpha: float = 1.0,
                      size_lo: int = 100, size_hi: int = 100_000,
                      seed: int = 0) -> List[Arrays]:
    """Independent uniform problems; instance ``i`` has ``N_i`` extents split
    ``m_i = N_i // 2`` updates and ``n_i = N_i - m_i`` subscriptions, each
    drawn by ``uniform_fixed_length`` with seed ``seed * 1_000_003 + i + 1``."""
    sizes = batched_sizes(count, size_lo, size_hi, seed)
    out = []
    for i, N in enumerate(sizes):
        m = int(N) // 2
        n = int(N) - m
        out.append(uniform_fixed_length(n, m, d, alpha, seed * 1_000_003 + i + 1))
    return out


# Named configurations (sizes as in the experiments they stand in for).
CONFIGS = {
    # d=1, 5e3 + 5e3, alpha = 1 (l = 100), seed 0
    "uniform_d1_N1e4_a1": dict(kind="uniform", n=5000, m=5000, d=1, alpha=1.0, seed=0),
}
for _d in (1, 2):
    for _a, _tag in ((0.01, "0.01"), (1.0, "1"), (100.0, "100")):
        CONFIGS[f"uniform_d{_d}_N1e6_a{_tag}"] = dict(kind="uniform", n=500_000, m=500_000,
                                                      d=_d, alpha=_a, seed=0)
CONFIGS["clustered_d3_N1e7_a100"] = dict(kind="clustered", n=5_000_000, m=5_000_000, d=3,
                                         alpha=100.0, seed=0)


def make(name: str, scale: float = 1.0) -> Arrays:
    """Generate a named configuration; ``scale`` shrinks n and m (for
    oracle-sized versions of the same distribution; alpha is kept)."""
    c = dict(CONFIGS[name])
    n = max(1, int(round(c["n"] * scale)))
    m = max(1, int(round(c["m"] * scale)))
    if c["kind"] == "uniform":
        return uniform_fixed_length(n, m, c["d"], c["alpha"], c["seed"])
    return clustered_lognormal(n, m, c["d"], c["alpha"], c["seed"])


def concat_instances(instances) -> Tuple[np.ndarray, np.ndarray, np.ndarray,
                                          np.ndarray, np.ndarray, np.ndarray]:
    """Concatenate independent problems for the batched call: returns
    ``(upd_lo, upd_hi, upd_off, sub_lo, sub_hi, sub_off)`` with the sets laid
    out instance after instance (SoA over the whole batch) and uint64 offset
    arrays of ``count + 1`` entries."""
    d = instances[0][0].shape[0]
    ms = [a[0].shape[1] for a in instances]
    ns = [a[2].shape[1] for a in instances]
    upd_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.uint64)
    sub_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.uint64)

    def cat(i):
        parts = [a[i] for a in instances]
        return np.ascontiguousarray(np.concatenate(parts, axis=1)) if parts else np.zeros((d, 0), np.float32)

    return cat(0), cat(1), upd_off, cat(2), cat(3), sub_off
