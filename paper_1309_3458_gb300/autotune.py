"""Autotuner for the library's tuning knobs (``ddm_set_tuning`` and
``ddm_set_tiling``).

The knobs change speed only, never results: the re-sort group exponent shift
of the tree order, the CTAs per SM of the persistent query kernels, whether
the write pass replays the count pass's records or walks the tree, the
queries per warp (16 or 32 per packet: the tile is queries x the leaf's 32
subscriptions), and the number of a packet's queries on a leaf from which the
count pass swaps its loops (lane = query instead of lane = subscription).
The tree's fan-out stays 32: one lane per child, so a node's children are
tested by one coalesced load and one ballot.
``autotune`` times a caller-supplied run (one complete match through the C
ABI) under each candidate with CUDA events and keeps the fastest; the work
itself always runs in the library's kernels.
"""
from __future__ import annotations

import itertools
from typing import Callable, Dict, Iterable, List, Optional, Tuple

import paper_1309_3458_gb300 as ddm

DEFAULT_SPACE = {"str_shift": (-1, 0, 1), "ctas_per_sm": (4, 8), "replay": (1, 0),
                 "queries_per_packet": (32, 16), "swap_min": (8, 12, 24)}
TUNING = ("str_shift", "ctas_per_sm", "replay")
TILING = ("queries_per_packet", "swap_min")
DEFAULTS = {"str_shift": 0, "ctas_per_sm": 8, "replay": 1, "queries_per_packet": 32,
            "swap_min": 12}


def apply(ctx: int, cand: Dict[str, int]) -> None:
    """Set a candidate (missing knobs take their defaults) on a context."""
    full = dict(DEFAULTS, **cand)
    ddm.ddm_set_tuning(ctx, **{k: full[k] for k in TUNING})
    ddm.ddm_set_tiling(ctx, **{k: full[k] for k in TILING})


def candidates(space: Optional[Dict[str, Iterable]] = None) -> List[Dict[str, int]]:
    space = space or DEFAULT_SPACE
    names = list(space)
    return [dict(zip(names, vals)) for vals in itertools.product(*(space[n] for n in names))]


def autotune(ctx: int, run: Callable[[], None], space=None, reps: int = 3,
             stream=None) -> Tuple[Dict[str, int], List[Tuple[float, Dict[str, int]]]]:
    """Time ``run()`` (which must issue its work on ``stream``, default the
    current stream) under every candidate; set the fastest on ``ctx`` and
    return it with the table of (median ms, candidate)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    table = []
    for cand in candidates(space):
        apply(ctx, cand)
        run()  # warm-up: sizes workspace and record arena for this candidate
        times = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        table.append((times[len(times) // 2], cand))
    table.sort(key=lambda x: x[0])
    best = table[0][1]
    apply(ctx, best)
    return best, table
