"""GPU interval tree matching for Data Distribution Management.

Thin Python binding of ``libddm.so`` (C ABI declared in ``include/ddm.h``).
Functions carry the C names and only marshal arguments: device tensors are
passed as raw pointers, the stream is torch's current CUDA stream unless one
is given.  Every step of the matching runs in the library's CUDA kernels;
there is no CPU fallback, and importing a function fails loudly when the
library has not been built (``python -m paper_1309_3458_gb300.build``).

Array conventions (see ``include/ddm.h``): coordinates are float32 device
tensors of shape ``(d, count)`` (row k = dimension k), C-contiguous.  The pair
output is an int32 device tensor of shape ``(capacity, 2)``: column 0 the
update id, column 1 the subscription id.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
# DDM_LIBRARY=checked selects the checked build (kernels verify their indices
# and report DDM_ERR_INTERNAL instead of touching memory out of bounds).
LIB_PATH = os.path.join(HERE, "libddm_checked.so" if os.environ.get("DDM_LIBRARY") == "checked"
                        else "libddm.so")

DDM_OK = 0
DDM_ERR_ARG = 1
DDM_ERR_EXTENT = 2
DDM_ERR_CAPACITY = 3
DDM_ERR_NOMEM = 4
DDM_ERR_CUDA = 5
DDM_ERR_TIMEOUT = 6
DDM_ERR_STATE = 7
DDM_ERR_INTERNAL = 8

DDM_CLOSED = 0
DDM_OPEN = 1
DDM_SWAP_ROLES = 2
DDM_MAX_DIMS = 8
DDM_MAX_EXTENTS = (1 << 30) - 1
DDM_MAX_TREE_LEVELS = 8
DDM_NOALLOC_MAX_UPDATES = 1 << 26

# Every entry point declared in include/ddm.h, with its ctypes signature.
_vp, _i, _u32, _u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
_pu32, _pu64, _pi = (ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                     ctypes.POINTER(ctypes.c_int))
_SET = [_vp, _vp, _u32]  # lo, hi, count
SIGNATURES = {
    "ddm_create": (_i, [ctypes.POINTER(_vp), _i]),
    "ddm_destroy": (_i, [_vp]),
    "ddm_strerror": (ctypes.c_char_p, [_i]),
    "ddm_count": (_i, [_vp, _i] + _SET + _SET + [_u32, _pu64, _vp]),
    "ddm_match": (_i, [_vp, _i] + _SET + _SET + [_u32, _vp, _u64, _pu64, _vp]),
    "ddm_match_range": (_i, [_vp, _i] + _SET + _SET + [_u32, _u32, _u32, _vp, _u64, _pu64, _vp]),
    "ddm_build": (_i, [_vp, _i, _vp, _vp, _u32, _vp]),
    "ddm_plan": (_i, [_vp, _vp, _vp, _u32, _u32, _vp, _pu64, _vp]),
    "ddm_refit": (_i, [_vp, _vp, _vp, _vp]),
    "ddm_plan_async": (_i, [_vp, _vp, _vp, _u32, _u32, _vp]),
    "ddm_write_async": (_i, [_vp, _u32, _u32, _vp, _u64, _vp, _vp, _vp]),
    "ddm_pair_offsets_async": (_i, [_vp, _vp, _u32, _vp, _vp]),
    "ddm_match_moved": (_i, [_vp, _vp, _vp, _u32, _vp, _u32, _vp, _u64, _vp, _vp]),
    "ddm_plan_stats": (_i, [_vp, _vp]),
    "ddm_attach": (_i, [_vp, _vp]),
    "ddm_write": (_i, [_vp, _u32, _u32, _vp, _u64, _pu64, _vp]),
    "ddm_chunk_end": (_i, [_vp, _u32, _u64, _pu32, _vp]),
    "ddm_plan_order": (_i, [_vp, _vp, _vp, _vp]),
    "ddm_write_ordered": (_i, [_vp, _u32, _u32, _vp, _u64, _pu64, _vp]),
    "ddm_write_ordered_ids": (_i, [_vp, _u32, _u32, _vp, _u64, _pu64, _vp]),
    "ddm_chunk_end_ordered": (_i, [_vp, _u32, _u64, _pu32, _vp]),
    "ddm_tree_shape": (_i, [_vp, _pi, _pu32, _pu32]),
    "ddm_tree_export": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "ddm_debug_set_alloc_limit": (_i, [_vp, _u64]),
    "ddm_set_replay_budget": (_i, [_vp, _u64]),
    "ddm_set_tuning": (_i, [_vp, _i, _u32, _u32]),
    "ddm_set_update_id_base": (_i, [_vp, _u32]),
    "ddm_set_tiling": (_i, [_vp, _u32, _u32]),
    "ddm_debug_launch_count": (_u64, []),
    "ddm_debug_wait_timeout": (_i, [_vp, _u32, _vp]),
    "ddm_scan_counts_noalloc": (_i, [_vp, _u32, _vp, _vp]),
    "ddm_batch_match": (_i, [_vp, _i, _u32, _vp, _vp, _vp, _u32, _vp, _vp, _vp, _u32, _u32, _vp,
                             _u64, _vp, _pu64, _vp]),
    "ddm_batch_match_async": (_i, [_vp, _i, _u32, _vp, _vp, _vp, _u32, _vp, _vp, _vp, _u32, _u32,
                                   _vp, _u64, _vp, _vp, _vp, _vp]),
}

_lib = None

# CUDA device of every context this binding created (handle -> device index).
# The kernels dereference the raw pointers they are given, so a tensor on
# another GPU than its context must be refused here: the C side cannot tell.
_CTX_DEVICE = {}


class DDMError(RuntimeError):
    """Non-zero return code of a libddm call; ``k`` holds *k_out when set."""

    def __init__(self, code: int, where: str, k: Optional[int] = None):
        self.code = code
        self.k = k
        super().__init__(f"{where}: {ddm_strerror(code)} (code {code})")


def lib():
    """Load libddm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} missing: build it with "
                               "`python -m paper_1309_3458_gb300.build`"
                               + (" --checked" if LIB_PATH.endswith("_checked.so") else ""))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ddm_strerror(code: int) -> str:
    """Text of a return code."""
    return lib().ddm_strerror(code).decode()


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _device_tensor(t, what: str, dev: Optional[int] = None):
    """Kernels read these arrays directly: a host (pageable) pointer would
    fault the GPU, so only CUDA tensors (or pinned host tensors, which the
    device can address) pass.  With `dev` given, a CUDA tensor must live on
    that device: a peer GPU's pointer is not addressable by the kernels."""
    cuda = bool(getattr(t, "is_cuda", False))
    if not (cuda or (hasattr(t, "is_pinned") and t.is_pinned())):
        raise ValueError(f"{what} must be a CUDA tensor (or pinned host memory)")
    if cuda and dev is not None and t.device.index != dev:
        raise ValueError(f"{what} is on cuda:{t.device.index}, the context on cuda:{dev}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def _dev(ctx) -> Optional[int]:
    """Device of a context made by ddm_create (None for a foreign handle)."""
    return _CTX_DEVICE.get(ctx)


def _arr(t, what: str, itemsize: int, n: Optional[int] = None, dev: Optional[int] = None):
    """Pointer of an optional device array argument (None passes NULL):
    device-addressable (on `dev` when given), contiguous, `itemsize`-byte
    elements, at least `n`."""
    if t is None:
        return None
    _device_tensor(t, what, dev)
    if t.element_size() != itemsize:
        raise TypeError(f"{what} must hold {itemsize}-byte elements")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what} needs at least {n} entries")
    return t.data_ptr()


def _set(lo, hi, dev: Optional[int] = None) -> Tuple[int, int, int, int]:
    import torch
    if lo.dim() != 2 or hi.shape != lo.shape:
        raise ValueError("lo and hi must be (d, count) tensors of the same shape")
    if lo.dtype != torch.float32 or hi.dtype != torch.float32:
        raise TypeError("coordinates must be float32")
    _device_tensor(lo, "lo", dev)
    _device_tensor(hi, "hi", dev)
    d, c = lo.shape
    if c > DDM_MAX_EXTENTS:  # the C ABI takes a uint32 count
        raise ValueError(f"{c} extents in one set; at most {DDM_MAX_EXTENTS}")
    return d, _ptr(lo), _ptr(hi), c


def _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, dev: Optional[int] = None):
    d, ul, uh, m = _set(upd_lo, upd_hi, dev)
    d2, sl, sh, n = _set(sub_lo, sub_hi, dev)
    if d != d2:
        raise ValueError(f"update and subscription sets have {d} and {d2} dimensions")
    return d, ul, uh, m, sl, sh, n


def _pairs(pairs, dev: Optional[int] = None) -> int:
    """Capacity of a pair buffer: an int32 (capacity, 2) tensor."""
    import torch
    if pairs is None:
        return 0
    if pairs.dtype != torch.int32 or pairs.dim() != 2 or pairs.shape[1] != 2:
        raise TypeError("pairs must be an int32 tensor of shape (capacity, 2)")
    _device_tensor(pairs, "pairs", dev)
    return pairs.shape[0]


def _ids(ids, dev: Optional[int] = None) -> int:
    """Capacity of a subscription-id buffer: a 1-D int32 tensor."""
    import torch
    if ids is None:
        return 0
    if ids.dtype != torch.int32 or ids.dim() != 1:
        raise TypeError("sub_ids must be a 1-D int32 tensor")
    _device_tensor(ids, "sub_ids", dev)
    return ids.shape[0]


def _check(rc: int, where: str, k: Optional[int] = None):
    if rc != DDM_OK:
        raise DDMError(rc, where, k)


def ddm_create(device: int = 0) -> int:
    """New context on CUDA device `device`; returns its handle."""
    h = ctypes.c_void_p()
    _check(lib().ddm_create(ctypes.byref(h), device), "ddm_create")
    _CTX_DEVICE[h.value] = device
    return h.value


def ddm_destroy(ctx: int) -> None:
    """Free a context and all its device memory."""
    _check(lib().ddm_destroy(ctx), "ddm_destroy")
    _CTX_DEVICE.pop(ctx, None)


def ddm_count(ctx: int, upd_lo, upd_hi, sub_lo, sub_hi, flags: int = DDM_CLOSED,
              stream=None) -> int:
    """K, the number of intersecting (update, subscription) pairs (Algs. 4-5,
    count only).  Coordinates: float32 device tensors of shape (d, count)."""
    d, ul, uh, m, sl, sh, n = _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_count(ctx, d, ul, uh, m, sl, sh, n, flags, ctypes.byref(k), _stream(stream))
    _check(rc, "ddm_count", k.value)
    return k.value


def ddm_match(ctx: int, upd_lo, upd_hi, sub_lo, sub_hi, pairs, flags: int = DDM_CLOSED,
              stream=None) -> int:
    """Write all K pairs into `pairs` (int32 device tensor (capacity, 2):
    update id, subscription id), grouped by update id; returns K."""
    d, ul, uh, m, sl, sh, n = _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, _dev(ctx))
    cap = _pairs(pairs, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_match(ctx, d, ul, uh, m, sl, sh, n, flags, _ptr(pairs), cap, ctypes.byref(k),
                         _stream(stream))
    _check(rc, "ddm_match", k.value)
    return k.value


def ddm_match_range(ctx: int, upd_lo, upd_hi, sub_lo, sub_hi, upd_begin: int, upd_end: int,
                    pairs, flags: int = DDM_CLOSED, stream=None) -> int:
    """The pairs of the updates with ids in [upd_begin, upd_end) only (chunked
    output); returns their count."""
    d, ul, uh, m, sl, sh, n = _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, _dev(ctx))
    cap = _pairs(pairs, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_match_range(ctx, d, ul, uh, m, sl, sh, n, upd_begin, upd_end, flags,
                               _ptr(pairs), cap, ctypes.byref(k), _stream(stream))
    _check(rc, "ddm_match_range", k.value)
    return k.value


def ddm_build(ctx: int, sub_lo, sub_hi, stream=None) -> None:
    """Build the resident tree over the subscriptions (Interval-Tree-Create,
    Alg. 5); the coordinates are copied."""
    d, sl, sh, n = _set(sub_lo, sub_hi, _dev(ctx))
    _check(lib().ddm_build(ctx, d, sl, sh, n, _stream(stream)), "ddm_build")


def ddm_refit(ctx: int, sub_lo, sub_hi, stream=None) -> None:
    """Recompute the resident tree's node bounds after its extents moved: same
    ids and order, new coordinates in sub_lo / sub_hi (d x n float32 device
    tensors, extent i still at column i; None only for an empty tree)."""
    sl = sh = None
    if sub_lo is not None or sub_hi is not None:
        _, sl, sh, _ = _set(sub_lo, sub_hi, _dev(ctx))
    _check(lib().ddm_refit(ctx, sl, sh, _stream(stream)), "ddm_refit")


def ddm_attach(ctx: int, src: int) -> None:
    """Let `ctx` query the tree built in `src` without copying it."""
    _check(lib().ddm_attach(ctx, src), "ddm_attach")


def ddm_plan(ctx: int, upd_lo, upd_hi, flags: int = DDM_CLOSED, offsets=None,
             stream=None) -> int:
    """Count pass and prefix sum for the updates against the resident tree;
    optional `offsets` (int64 device tensor, m + 1) receives the per-update
    output offsets.  Returns K."""
    d, ul, uh, m = _set(upd_lo, upd_hi, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_plan(ctx, ul, uh, m, flags, _arr(offsets, "offsets", 8, m + 1, dev=_dev(ctx)), ctypes.byref(k),
                        _stream(stream))
    _check(rc, "ddm_plan", k.value)
    return k.value


def ddm_plan_async(ctx: int, upd_lo, upd_hi, flags: int = DDM_CLOSED, stream=None) -> None:
    """ddm_plan without host synchronisation (offsets stay in the context)."""
    d, ul, uh, m = _set(upd_lo, upd_hi, _dev(ctx))
    _check(lib().ddm_plan_async(ctx, ul, uh, m, flags, _stream(stream)), "ddm_plan_async")


def ddm_write_async(ctx: int, upd_begin: int, upd_end: int, pairs, k_dev=None, err_dev=None,
                    stream=None) -> None:
    """ddm_write without host synchronisation; K and the error bits go to the
    optional device tensors k_dev (int64, 1) and err_dev (int32, 1)."""
    cap = _pairs(pairs, _dev(ctx))
    kd, ed = _arr(k_dev, "k_dev", 8, 1, dev=_dev(ctx)), _arr(err_dev, "err_dev", 4, 1, dev=_dev(ctx))
    _check(lib().ddm_write_async(ctx, upd_begin, upd_end, _ptr(pairs), cap, kd, ed,
                                 _stream(stream)), "ddm_write_async")


def ddm_plan_stats(ctx: int) -> int:
    """(query, leaf) tests made by the last count pass that returned."""
    v = ctypes.c_uint64(0)
    _check(lib().ddm_plan_stats(ctx, ctypes.byref(v)), "ddm_plan_stats")
    return v.value


def ddm_match_moved(ctx: int, lo, hi, ids, pairs, flags: int = DDM_CLOSED, stream=None) -> int:
    """Pairs of k moved extents (d x k device tensors) against the context's
    tree, the moved extents named by ids (uint32/int32 device tensor of k
    entries, or None for 0..k-1); see ddm.h."""
    d, l, h, k = _set(lo, hi, _dev(ctx))
    if ids is not None and ids.shape[0] != k:
        raise ValueError("ids needs one entry per moved extent")
    cap = _pairs(pairs, _dev(ctx))
    kk = ctypes.c_uint64(0)
    rc = lib().ddm_match_moved(ctx, l, h, k, _arr(ids, "ids", 4, k, dev=_dev(ctx)), flags, _ptr(pairs), cap,
                               ctypes.byref(kk), _stream(stream))
    _check(rc, "ddm_match_moved", kk.value)
    return kk.value


def ddm_pair_offsets_async(ctx: int, upd_off, pair_off, stream=None) -> None:
    """pair_off[i] = pairs of the updates with id < upd_off[i] in the current
    plan (both uint64/int64 device tensors of count + 1 entries)."""
    count = upd_off.shape[0] - 1
    if count < 0 or pair_off.shape[0] < count + 1:
        raise ValueError("upd_off and pair_off need count + 1 entries")
    _check(lib().ddm_pair_offsets_async(ctx, _arr(upd_off, "upd_off", 8, count + 1, dev=_dev(ctx)), count,
                                        _arr(pair_off, "pair_off", 8, count + 1, dev=_dev(ctx)), _stream(stream)),
           "ddm_pair_offsets_async")


def ddm_write(ctx: int, upd_begin: int, upd_end: int, pairs, stream=None) -> int:
    """Write the pairs of the current plan's updates with ids in [upd_begin,
    upd_end), laid out by update id; returns the pair count."""
    cap = _pairs(pairs, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_write(ctx, upd_begin, upd_end, _ptr(pairs), cap, ctypes.byref(k),
                         _stream(stream))
    _check(rc, "ddm_write", k.value)
    return k.value


def ddm_chunk_end(ctx: int, upd_begin: int, capacity: int, stream=None) -> int:
    """Largest update id e such that the pairs of [upd_begin, e) fit in
    `capacity` pairs."""
    e = ctypes.c_uint32(0)
    rc = lib().ddm_chunk_end(ctx, upd_begin, capacity, ctypes.byref(e), _stream(stream))
    _check(rc, "ddm_chunk_end", e.value)
    return e.value


def ddm_plan_order(ctx: int, order=None, order_offsets=None, stream=None) -> None:
    """The plan's spatial query order: `order` (int32 device tensor, m) gets
    the update at each plan position, `order_offsets` (int64, m + 1) where each
    position's pairs start; either may be None."""
    o, oo = _arr(order, "order", 4, dev=_dev(ctx)), _arr(order_offsets, "order_offsets", 8, dev=_dev(ctx))
    _check(lib().ddm_plan_order(ctx, o, oo, _stream(stream)), "ddm_plan_order")


def ddm_write_ordered(ctx: int, pos_begin: int, pos_end: int, pairs, stream=None) -> int:
    """Write the pairs of plan positions [pos_begin, pos_end), grouped by
    update in plan order; returns the pair count."""
    cap = _pairs(pairs, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_write_ordered(ctx, pos_begin, pos_end, _ptr(pairs), cap, ctypes.byref(k),
                                 _stream(stream))
    _check(rc, "ddm_write_ordered", k.value)
    return k.value


def ddm_write_ordered_ids(ctx: int, pos_begin: int, pos_end: int, sub_ids, stream=None) -> int:
    """Compressed output: the subscription ids of ddm_write_ordered's pairs
    (same positions) into a 1-D int32 tensor; returns the id count."""
    cap = _ids(sub_ids, _dev(ctx))
    k = ctypes.c_uint64(0)
    rc = lib().ddm_write_ordered_ids(ctx, pos_begin, pos_end, _ptr(sub_ids), cap,
                                     ctypes.byref(k), _stream(stream))
    _check(rc, "ddm_write_ordered_ids", k.value)
    return k.value


def ddm_chunk_end_ordered(ctx: int, pos_begin: int, capacity: int, stream=None) -> int:
    """Largest plan position e such that the pairs of [pos_begin, e) fit in
    `capacity` pairs (or ids)."""
    e = ctypes.c_uint32(0)
    rc = lib().ddm_chunk_end_ordered(ctx, pos_begin, capacity, ctypes.byref(e), _stream(stream))
    _check(rc, "ddm_chunk_end_ordered", e.value)
    return e.value


def ddm_tree_shape(ctx: int) -> Tuple[int, Sequence[int], int]:
    """(levels, node count per level, total nodes) of the resident tree."""
    lv = ctypes.c_int(0)
    cnt = (ctypes.c_uint32 * DDM_MAX_TREE_LEVELS)()
    tot = ctypes.c_uint32(0)
    _check(lib().ddm_tree_shape(ctx, ctypes.byref(lv), cnt, ctypes.byref(tot)), "ddm_tree_shape")
    return lv.value, list(cnt)[: lv.value], tot.value


def ddm_tree_export(ctx: int, order=None, node_lo=None, node_hi=None, stream=None) -> None:
    """Copy out the tree: `order` (int32 device tensor, n) the subscription id
    at each sorted position; `node_lo` / `node_hi` (float32, d * total) each
    node's minlower / maxupper per dimension, entry k * total + j, levels
    stored one after another from level 1.  Any output may be None."""
    _check(lib().ddm_tree_export(ctx, _arr(order, "order", 4, dev=_dev(ctx)), _arr(node_lo, "node_lo", 4, dev=_dev(ctx)),
                                 _arr(node_hi, "node_hi", 4, dev=_dev(ctx)),
                                 _stream(stream)), "ddm_tree_export")


def ddm_set_tuning(ctx: int, str_shift: int = 0, ctas_per_sm: int = 8, replay: int = 1) -> None:
    """Speed-only knobs: re-sort group shift, CTAs per SM of the packet
    kernels, replay on (1) or off (0).  Results never depend on them."""
    _check(lib().ddm_set_tuning(ctx, str_shift, ctas_per_sm, replay), "ddm_set_tuning")


def ddm_set_tiling(ctx: int, queries_per_packet: int = 32, swap_min: int = 12) -> None:
    """Speed-only tiling of the query kernels: 16 or 32 queries per warp, and
    the number of a packet's queries on a leaf from which the count pass swaps
    its loops (33 = never).  Results never depend on it."""
    _check(lib().ddm_set_tiling(ctx, queries_per_packet, swap_min), "ddm_set_tiling")


def ddm_set_update_id_base(ctx: int, base: int) -> None:
    """Add `base` to every update id the context writes from now on (a shard
    of updates [base, base + m) of a larger problem); see include/ddm.h."""
    if not 0 <= base < (1 << 32):
        raise ValueError("the update-id base must fit 32 bits")
    _check(lib().ddm_set_update_id_base(ctx, base), "ddm_set_update_id_base")


def ddm_set_replay_budget(ctx: int, nbytes: int) -> None:
    """Upper bound (bytes) of the record arena the count pass may fill."""
    _check(lib().ddm_set_replay_budget(ctx, nbytes), "ddm_set_replay_budget")


def ddm_debug_set_alloc_limit(ctx: int, nbytes: int) -> None:
    """Make device allocations beyond `nbytes` fail (0: no limit), for tests."""
    _check(lib().ddm_debug_set_alloc_limit(ctx, nbytes), "ddm_debug_set_alloc_limit")


def ddm_debug_wait_timeout(ctx: int, polls: int, stream=None) -> None:
    """Make a bounded device wait run out (raises DDMError DDM_ERR_TIMEOUT)."""
    _check(lib().ddm_debug_wait_timeout(ctx, polls, _stream(stream)), "ddm_debug_wait_timeout")


def ddm_debug_launch_count() -> int:
    """Kernels the library has launched so far in this process."""
    return int(lib().ddm_debug_launch_count())


def ddm_scan_counts_noalloc(counts, offsets, stream=None) -> None:
    """Offsets (int64 device tensor, m + 1) from per-update counts (1-D int32
    device tensor of m uint32 counts, m <= DDM_NOALLOC_MAX_UPDATES) without
    any allocation; see include/ddm.h.  Both tensors must be on the current
    CUDA device, whose stream the work goes to unless `stream` is given."""
    import torch
    if counts.dim() != 1 or counts.dtype != torch.int32:
        raise TypeError("counts must be a 1-D int32 tensor (uint32 counts)")
    m = counts.shape[0]
    if m > DDM_NOALLOC_MAX_UPDATES:  # also keeps m inside the uint32 argument
        raise ValueError(f"{m} counts; the allocation-free scan takes at most "
                         f"{DDM_NOALLOC_MAX_UPDATES}")
    if offsets.dim() != 1 or offsets.dtype != torch.int64:
        raise TypeError("offsets must be a 1-D int64 tensor")
    dev = torch.cuda.current_device()
    c = _arr(counts, "counts", 4, dev=dev)
    o = _arr(offsets, "offsets", 8, m + 1, dev=dev)
    _check(lib().ddm_scan_counts_noalloc(c, m, o, _stream(stream)), "ddm_scan_counts_noalloc")


def ddm_batch_match(ctx: int, upd_lo, upd_hi, upd_off, sub_lo, sub_hi, sub_off, pairs,
                    pair_off=None, flags: int = DDM_CLOSED, stream=None) -> int:
    """Batched instances (see include/ddm.h).  upd_off / sub_off: int64 device
    tensors of count + 1 offsets; pairs: int32 device tensor (capacity, 2)."""
    d, ul, uh, m, sl, sh, n = _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, _dev(ctx))
    count = upd_off.shape[0] - 1
    cap = _pairs(pairs, _dev(ctx))
    k = ctypes.c_uint64(0)
    uo = _arr(upd_off, "upd_off", 8, count + 1, dev=_dev(ctx))
    so = _arr(sub_off, "sub_off", 8, count + 1, dev=_dev(ctx))
    po = _arr(pair_off, "pair_off", 8, count + 1, dev=_dev(ctx))
    rc = lib().ddm_batch_match(ctx, d, count, ul, uh, uo, m, sl, sh, so, n, flags, _ptr(pairs), cap,
                               po, ctypes.byref(k), _stream(stream))
    _check(rc, "ddm_batch_match", k.value)
    return k.value


def ddm_batch_match_async(ctx: int, upd_lo, upd_hi, upd_off, sub_lo, sub_hi, sub_off, pairs,
                          pair_off=None, k_dev=None, err_dev=None, flags: int = DDM_CLOSED,
                          stream=None) -> None:
    """Host-synchronisation-free batched match (capturable in a CUDA graph)."""
    d, ul, uh, m, sl, sh, n = _two_sets(upd_lo, upd_hi, sub_lo, sub_hi, _dev(ctx))
    count = upd_off.shape[0] - 1
    cap = _pairs(pairs, _dev(ctx))
    uo = _arr(upd_off, "upd_off", 8, count + 1, dev=_dev(ctx))
    so = _arr(sub_off, "sub_off", 8, count + 1, dev=_dev(ctx))
    po = _arr(pair_off, "pair_off", 8, count + 1, dev=_dev(ctx))
    rc = lib().ddm_batch_match_async(ctx, d, count, ul, uh, uo, m, sl, sh, so, n, flags,
                                     _ptr(pairs), cap, po, _arr(k_dev, "k_dev", 8, 1, dev=_dev(ctx)),
                                     _arr(err_dev, "err_dev", 4, 1, dev=_dev(ctx)), _stream(stream))
    _check(rc, "ddm_batch_match_async")
