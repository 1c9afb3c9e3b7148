"""CPU oracle for interval-tree DDM matching -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this package.  The GPU library never does, and this
package never imports the GPU library: the two share no code.  The shared
seeded input generators live in ``paper_1309_3458_gb300.workloads``, which
holds no matching arithmetic.

The arithmetic is in ``ddm_oracle.c`` (plain C, comparisons on values widened
to double).  What each entry point follows:

* ``bf``         -- Alg. 2 (Brute Force) with the d-dimensional reduction of
                    Section III-A and the segment test of Alg. 1.
* ``itm_count`` / ``itm_pairs`` -- Algs. 4 and 5 (Interval-Query and
                    IntTree-Matching) over an augmented AVL tree (Section IV),
                    queries split over threads as in "Parallelizing ITM".
* ``bits_count`` -- BITS counting (Section II, related work), d = 1, closed
                    rule; an independent check of per-update counts.
* ``tree_order`` -- in-order sequence of the interval tree (ids by lower,
                    upper, id on dimension 0).

Readings of the paper (closed vs open segments, tie order, 0-based ids) are
stated at the top of ``ddm_oracle.c``.  Parity is pinned for every entry
point by the CPU tests (lattice closed forms, the Fig. 1 example, BITS,
brute force against ITM on tiny grids).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ddm_oracle.c")
LIB = os.path.join(HERE, "libddm_oracle.so")

OPEN = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP enabled) into ``libddm_oracle.so``."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def bind(cdll):
    """Declare the argument and result types of the oracle's entry points."""
    f32 = ctypes.POINTER(ctypes.c_float)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    u64 = ctypes.POINTER(ctypes.c_uint64)
    i32 = ctypes.POINTER(ctypes.c_int32)
    L = cdll
    L.oracle_bf.restype = ctypes.c_uint64
    L.oracle_bf.argtypes = [ctypes.c_int, f32, f32, ctypes.c_uint32, f32, f32, ctypes.c_uint32,
                            ctypes.c_uint32, u32, u64, u32, u32, ctypes.c_uint64]
    L.oracle_itm_count.restype = ctypes.c_uint64
    L.oracle_itm_count.argtypes = [ctypes.c_int, f32, f32, ctypes.c_uint32, f32, f32,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, u32, u64,
                                   ctypes.POINTER(ctypes.c_double)]
    L.oracle_itm_pairs.restype = ctypes.c_uint64
    L.oracle_itm_pairs.argtypes = [ctypes.c_int, f32, f32, ctypes.c_uint32, f32, f32,
                                   ctypes.c_uint32, ctypes.c_uint32, u32, u32, ctypes.c_uint64]
    L.oracle_bits_count.restype = ctypes.c_uint64
    L.oracle_bits_count.argtypes = [f32, f32, ctypes.c_uint32, f32, f32, ctypes.c_uint32, u32]
    L.oracle_tree_order.restype = ctypes.c_int
    L.oracle_tree_order.argtypes = [f32, f32, ctypes.c_uint32, u32, i32]
    L.oracle_intersect_1d.restype = ctypes.c_int
    L.oracle_intersect_1d.argtypes = [ctypes.c_double] * 4 + [ctypes.c_uint32]
    L.oracle_mix64.restype = ctypes.c_uint64
    L.oracle_mix64.argtypes = [ctypes.c_uint64]
    L.oracle_openmp_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = bind(ctypes.CDLL(LIB))
    return _lib


def _f32(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _u32(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _shape(upd_lo, upd_hi, sub_lo, sub_hi) -> Tuple[int, int, int]:
    d, m = upd_lo.shape
    d2, n = sub_lo.shape
    assert d == d2 and upd_hi.shape == upd_lo.shape and sub_hi.shape == sub_lo.shape
    return d, m, n


def intersect_1d(xlo, xhi, ylo, yhi, flags: int = 0) -> bool:
    """Alg. 1 (strict under ``OPEN``, closed otherwise)."""
    return bool(lib().oracle_intersect_1d(xlo, xhi, ylo, yhi, flags))


def mix64(z: int) -> int:
    return int(lib().oracle_mix64(z))


def bf(upd_lo, upd_hi, sub_lo, sub_hi, flags: int = 0, pairs: bool = True):
    """Brute force.  Returns ``(K, counts[m], digests[m], upd_ids, sub_ids)``;
    pairs grouped by update, subscriptions ascending within an update."""
    d, m, n = _shape(upd_lo, upd_hi, sub_lo, sub_hi)
    counts = np.zeros(m, np.uint32)
    digests = np.zeros(m, np.uint64)
    if pairs:
        K = int(lib().oracle_bf(d, _f32(upd_lo), _f32(upd_hi), m, _f32(sub_lo), _f32(sub_hi), n,
                                flags, _u32(counts), _u64(digests), None, None, 0))
        pu = np.zeros(max(K, 1), np.uint32)
        ps = np.zeros(max(K, 1), np.uint32)
        lib().oracle_bf(d, _f32(upd_lo), _f32(upd_hi), m, _f32(sub_lo), _f32(sub_hi), n,
                        flags, None, None, _u32(pu), _u32(ps), K)
        return K, counts, digests, pu[:K], ps[:K]
    K = int(lib().oracle_bf(d, _f32(upd_lo), _f32(upd_hi), m, _f32(sub_lo), _f32(sub_hi), n,
                            flags, _u32(counts), _u64(digests), None, None, 0))
    return K, counts, digests, None, None


def itm_count(upd_lo, upd_hi, sub_lo, sub_hi, flags: int = 0, threads: int = 1,
              timings: Optional[list] = None):
    """Interval tree matching; returns ``(K, counts[m], digests[m])``.  If
    ``timings`` is a list, the build and query wall times (s) are appended."""
    d, m, n = _shape(upd_lo, upd_hi, sub_lo, sub_hi)
    counts = np.zeros(m, np.uint32)
    digests = np.zeros(m, np.uint64)
    sec = (ctypes.c_double * 2)()
    K = int(lib().oracle_itm_count(d, _f32(upd_lo), _f32(upd_hi), m, _f32(sub_lo), _f32(sub_hi),
                                   n, flags, threads, _u32(counts), _u64(digests), sec))
    if K == 2 ** 64 - 1:
        raise MemoryError("oracle tree allocation failed")
    if timings is not None:
        timings.extend([sec[0], sec[1]])
    return K, counts, digests


def itm_pairs(upd_lo, upd_hi, sub_lo, sub_hi, flags: int = 0, cap: Optional[int] = None):
    """Sequential interval tree matching; returns ``(K, upd_ids, sub_ids)``
    grouped by update, in tree order within an update."""
    d, m, n = _shape(upd_lo, upd_hi, sub_lo, sub_hi)
    if cap is None:
        cap, _, _ = itm_count(upd_lo, upd_hi, sub_lo, sub_hi, flags,
                              threads=lib().oracle_openmp_threads())
    pu = np.zeros(max(cap, 1), np.uint32)
    ps = np.zeros(max(cap, 1), np.uint32)
    K = int(lib().oracle_itm_pairs(d, _f32(upd_lo), _f32(upd_hi), m, _f32(sub_lo), _f32(sub_hi),
                                   n, flags, _u32(pu), _u32(ps), cap))
    assert K <= cap
    return K, pu[:K], ps[:K]


def bits_count(upd_lo, upd_hi, sub_lo, sub_hi):
    """BITS per-update counts (d = 1, closed rule); returns ``(K, counts)``."""
    d, m, n = _shape(upd_lo, upd_hi, sub_lo, sub_hi)
    assert d == 1
    counts = np.zeros(m, np.uint32)
    K = int(lib().oracle_bits_count(_f32(upd_lo[0]), _f32(upd_hi[0]), m,
                                    _f32(np.ascontiguousarray(sub_lo[0])),
                                    _f32(np.ascontiguousarray(sub_hi[0])), n, _u32(counts)))
    return K, counts


def tree_order(sub_lo0: np.ndarray, sub_hi0: np.ndarray):
    """In-order ids of the interval tree over one dimension, and its height."""
    n = sub_lo0.shape[0]
    order = np.zeros(max(n, 1), np.uint32)
    h = ctypes.c_int32(0)
    rc = lib().oracle_tree_order(_f32(np.ascontiguousarray(sub_lo0)),
                                 _f32(np.ascontiguousarray(sub_hi0)), n, _u32(order),
                                 ctypes.byref(h))
    if rc != 0:
        raise MemoryError("oracle tree allocation failed")
    return order[:n], h.value


def threads() -> int:
    return int(lib().oracle_openmp_threads())


def digest_of(sub_ids: np.ndarray) -> int:
    """Order-independent digest of a set of subscription ids (SplitMix64
    output function summed modulo 2**64); equals the oracle's per-update
    digest when ``sub_ids`` are one update's matches."""
    z = sub_ids.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return int(z.sum(dtype=np.uint64))
