"""One matching problem split across ranks, one GPU per rank.

Queries are independent (Section IV, "Parallelizing ITM"): every update's
overlap query reads the interval tree and nothing else.  So one problem's
update set U splits into contiguous ranges of update ids, one per rank; every
rank holds the whole subscription set S (replicated: each rank loads it, or
rank ``src`` broadcasts it once per match), builds the same tree (the build is
deterministic), and matches its range.  With the library's update-id base set
to the range's first id, a rank writes global update ids, so its pairs are
exactly the pairs one ``ddm_match`` over all of U writes for that range, in
the same order; the shards concatenated in rank order are that whole output.

Only host metadata crosses ranks on the data path: the per-rank pair counts
(an all-gather of one integer per rank) give every shard its global offset.
Collecting the shards on one rank (``gather_shards``) and broadcasting S
(``broadcast_set``) are optional.  Every step of the matching itself runs in
libddm's kernels on each rank's own GPU.

The distribution logic here (ranges, counts, offsets, gather, broadcast) is
plain ``torch.distributed`` and is tested over ``gloo`` on the CPU; the
matching on GPU is tested with two shards in one process.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import paper_1309_3458_gb300 as ddm


def shard_bounds(m: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous ranges of update ids, one per rank, covering [0, m) in rank
    order; sizes differ by at most one (the first m % world ranks get one
    more)."""
    if world < 1 or m < 0:
        raise ValueError("world must be >= 1 and m >= 0")
    q, r = divmod(m, world)
    out, b = [], 0
    for i in range(world):
        e = b + q + (1 if i < r else 0)
        out.append((b, e))
        b = e
    return out


def exclusive_prefix(counts: Sequence[int]) -> List[int]:
    """Offsets of each rank's pairs in the concatenated output (len + 1
    entries; the last is the total)."""
    out = [0]
    for k in counts:
        out.append(out[-1] + int(k))
    return out


def exchange_counts(k_local: int, group=None, device: str = "cpu") -> List[int]:
    """All ranks' pair counts, in rank order (one all-gather of an int64)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.tensor([int(k_local)], dtype=torch.int64, device=device)
    every = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    return [int(t.item()) for t in every]


def broadcast_set(lo, hi, src: int = 0, group=None) -> None:
    """Replicate a set's coordinates (in place) from rank `src`: every rank
    passes tensors of the same shape; the others' contents are replaced."""
    import torch.distributed as dist
    dist.broadcast(lo, src, group=group)
    dist.broadcast(hi, src, group=group)


def gather_shards(local, counts: Sequence[int], dst: int = 0, group=None):
    """Concatenate every rank's pairs (a (k_r, 2) int32 tensor per rank, k_r =
    counts[r]) on rank `dst`, in rank order; other ranks get None.  Shards
    are padded to the largest count for the all-gather."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    kmax = max(int(k) for k in counts) if counts else 0
    padded = torch.zeros((kmax, 2), dtype=local.dtype, device=local.device)
    padded[: local.shape[0]] = local
    every = [torch.empty_like(padded) for _ in counts]
    dist.all_gather(every, padded, group=group)
    if rank != dst:
        return None
    return torch.cat([t[: int(k)] for t, k in zip(every, counts)], dim=0)


@dataclass
class ShardPlan:
    """A rank's part of one sharded match."""
    rank: int
    world: int
    begin: int                  # first global update id of the shard
    end: int                    # one past the last
    k_local: int                # pairs of this shard
    counts: List[int] = field(default_factory=list)   # every rank's pairs
    offset: int = 0             # this shard's first pair in the whole output
    total: int = 0              # K of the whole problem


def plan_shard(ctx: int, upd_lo_shard, upd_hi_shard, begin: int, sub_lo, sub_hi, rank: int,
               world: int, group=None, counts_device: str = "cpu",
               flags: int = ddm.DDM_CLOSED) -> ShardPlan:
    """Build the tree over the whole subscription set, plan this rank's
    update shard (global ids [begin, begin + m_shard)), and exchange the pair
    counts.  The context then writes global update ids (ddm_write /
    ddm_write_ordered).  With world == 1 or no process group, no collective
    runs and counts holds this shard only."""
    m_shard = upd_lo_shard.shape[1]
    ddm.ddm_build(ctx, sub_lo, sub_hi)
    ddm.ddm_set_update_id_base(ctx, begin)
    k = ddm.ddm_plan(ctx, upd_lo_shard, upd_hi_shard, flags=flags)
    counts = [k]
    if world > 1:
        counts = exchange_counts(k, group, counts_device)
    pre = exclusive_prefix(counts)
    off = pre[rank] if world > 1 else 0
    return ShardPlan(rank, world, begin, begin + m_shard, k, counts, off, pre[-1])


def write_shard(ctx: int, plan: ShardPlan, pairs, consume=None) -> int:
    """Write the shard's pairs by update id in chunks of the `pairs` buffer
    ((capacity, 2) int32 device tensor); `consume(chunk, first_pair)` is
    called with each chunk (a view of `pairs`) and its position in the whole
    output.  Returns the shard's pair count."""
    m = plan.end - plan.begin
    cap = pairs.shape[0]
    b, done = 0, 0
    while b < m:
        e = ddm.ddm_chunk_end(ctx, b, cap)
        k = ddm.ddm_write(ctx, b, e, pairs)
        if consume is not None:
            consume(pairs[:k], plan.offset + done)
        done += k
        b = e
    return done
