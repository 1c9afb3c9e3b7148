"""Dynamic interval management (Section IV): both sets resident, both trees
kept, rows and columns recomputed for the extents that move.

The paper's scheme keeps an interval tree over the updates (T_U) and one
over the subscriptions (T_S).  When an update moves, its row of the
intersection matrix is recomputed by one query against T_S; when a
subscription moves, its column by one query against T_U; the moved extent
is also moved in its own tree.  Here the trees are the library's implicit
trees: moving extents rewrites their coordinates in the resident arrays and
brings their own tree up to date (`ddm_refit`: same order, new node bounds;
or a full rebuild every `rebuild_every`-th move, because a refitted order
ages), and `ddm_match_moved` recomputes the rows or columns.

Host orchestration only: the coordinate scatter is torch indexing of the
resident arrays; every step of the matching runs in libddm's kernels.
"""
from __future__ import annotations

from typing import Tuple

import paper_1309_3458_gb300 as ddm


class DynamicMatching:
    """Resident update set U and subscription set S (d x m and d x n float32
    CUDA tensors, copied) with a tree over each."""

    def __init__(self, upd_lo, upd_hi, sub_lo, sub_hi, flags: int = ddm.DDM_CLOSED,
                 rebuild_every: int = 8, stream=None):
        import torch
        self.flags = flags
        self.rebuild_every = rebuild_every
        self.stream = stream
        dev = upd_lo.device.index or 0
        self.U = [upd_lo.clone(), upd_hi.clone()]
        self.S = [sub_lo.clone(), sub_hi.clone()]
        self.t_u = ddm.ddm_create(dev)   # tree over the updates
        self.t_s = ddm.ddm_create(dev)   # tree over the subscriptions
        self.moves_u = self.moves_s = 0
        ddm.ddm_build(self.t_u, self.U[0], self.U[1], stream=stream)
        ddm.ddm_build(self.t_s, self.S[0], self.S[1], stream=stream)
        self._torch = torch

    def close(self):
        ddm.ddm_destroy(self.t_u)
        ddm.ddm_destroy(self.t_s)

    def match_all(self, pairs) -> int:
        """All pairs of the current coordinates (by update id), from T_S."""
        k = ddm.ddm_plan(self.t_s, self.U[0], self.U[1], flags=self.flags, stream=self.stream)
        if k > pairs.shape[0]:
            raise ddm.DDMError(ddm.DDM_ERR_CAPACITY, "match_all", k)
        return ddm.ddm_write(self.t_s, 0, self.U[0].shape[1], pairs, stream=self.stream)

    @staticmethod
    def _renew(ctx, arrays, moves, every, stream):
        if every and moves % every == 0:
            ddm.ddm_build(ctx, arrays[0], arrays[1], stream=stream)
        else:
            ddm.ddm_refit(ctx, arrays[0], arrays[1], stream=stream)

    def _scatter(self, arrays, ids, lo, hi):
        idx = ids.long()
        arrays[0][:, idx] = lo
        arrays[1][:, idx] = hi

    def move_updates(self, ids, lo, hi, pairs) -> int:
        """Updates `ids` (int32 CUDA tensor of k distinct ids) move to (lo,
        hi) (d x k).  Brings T_U up to date and writes the moved updates' new
        rows into `pairs` ({update id, subscription id}, grouped by moved
        update); returns the pair count."""
        self._scatter(self.U, ids, lo, hi)
        self.moves_u += 1
        self._renew(self.t_u, self.U, self.moves_u, self.rebuild_every, self.stream)
        return ddm.ddm_match_moved(self.t_s, lo.contiguous(), hi.contiguous(), ids, pairs,
                                   flags=self.flags, stream=self.stream)

    def move_subscriptions(self, ids, lo, hi, pairs) -> int:
        """Subscriptions `ids` move to (lo, hi).  Brings T_S up to date and
        writes their new columns ({update id, subscription id}, grouped by
        moved subscription); returns the pair count."""
        self._scatter(self.S, ids, lo, hi)
        self.moves_s += 1
        self._renew(self.t_s, self.S, self.moves_s, self.rebuild_every, self.stream)
        return ddm.ddm_match_moved(self.t_u, lo.contiguous(), hi.contiguous(), ids, pairs,
                                   flags=self.flags | ddm.DDM_SWAP_ROLES, stream=self.stream)

    def sets(self) -> Tuple:
        return self.U[0], self.U[1], self.S[0], self.S[1]
