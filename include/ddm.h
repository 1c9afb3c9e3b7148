/*
 * ddm.h -- C ABI of libddm, GPU interval tree matching for Data Distribution
 * Management (Marzolla, D'Angelo, Mandrioli, "A Parallel Data Distribution
 * Management Algorithm", DS-RT 2013).
 *
 * Problem (Section III): given subscription extents S_0..S_{n-1} and update
 * extents U_0..U_{m-1}, each a d-dimensional rectangle, report every pair
 * (U_j, S_i) whose intersection is non-empty.  Two d-rectangles intersect
 * iff their projections intersect in every dimension (Section III-A); the
 * per-dimension test is Intersect-1D (Alg. 1).  Ids are the 0-based
 * positions of the extents in their input arrays.
 *
 * Method (Section IV, Algs. 4 and 5): an interval tree is built over the
 * subscriptions, ordered by dimension-0 lower bound (ties by upper bound,
 * then id) with the maximum upper bound and minimum lower bound kept per
 * subtree; every update runs one overlap query against it, testing every
 * dimension with Intersect-1D.  On the GPU the tree is implicit (32 children
 * per node), keeps the subtree bounds for every dimension, and refines the
 * order near the leaves by the lower bounds of dimensions 1..d-1 inside
 * aligned groups of the dimension-0 order; for d >= 2 the subscriptions are
 * first grouped by size class (the binary exponent of their largest side),
 * each class ordered and refined on its own, so that long extents do not
 * widen the boxes of short ones.  Any order gives the same pairs (Section
 * IV allows any interval tree); d = 1 keeps the paper's order exactly.
 * Queries are independent (Section IV, "Parallelizing ITM") and run 32 per
 * warp.
 *
 * Conventions shared by every call:
 *  - Coordinates are float32 in structure-of-arrays layout: for a set of c
 *    extents, lo[k*c + i] / hi[k*c + i] are the lower / upper bound of
 *    extent i in dimension k (0 <= k < d).  Input pointers are DEVICE
 *    pointers (memory of the context's device), read only, owned by the
 *    caller, and must stay valid and unchanged until the call returns (for
 *    the staged calls: until the last call that uses them).
 *  - Every extent must satisfy lo <= hi in every dimension and contain no
 *    NaN; +-inf is allowed.  A violation gives DDM_ERR_EXTENT.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All GPU
 *    work is enqueued on it in order.  Calls that return a count (k_out)
 *    synchronise `stream` once to read it; nothing else blocks the host.
 *  - Output pairs are written to caller-owned DEVICE memory.  Order: update
 *    id ascending, then the subscriptions' position in the tree (for d = 1
 *    that is dimension-0 lower, upper, id); with DDM_SWAP_ROLES subscription
 *    id ascending, then the updates' tree position.  Only the set of pairs
 *    is the result; the order is deterministic for a given input.
 *    ddm_write_ordered_ids writes the compressed form instead: only each
 *    pair's subscription id, with the update of each run given by the plan
 *    order (Section III: M stored by columns).
 *  - Sizes: 1 <= d <= DDM_MAX_DIMS, n and m <= DDM_MAX_EXTENTS; n == 0 or
 *    m == 0 is valid and gives K = 0.
 *  - A context is not thread safe: one host thread at a time per context.
 */
#ifndef DDM_H
#define DDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define DDM_OK            0
#define DDM_ERR_ARG       1  /* null pointer, d out of range, size too large, bad range */
#define DDM_ERR_EXTENT    2  /* an extent has lo > hi or a NaN coordinate */
#define DDM_ERR_CAPACITY  3  /* more pairs than `capacity`; *k_out holds the needed count */
#define DDM_ERR_NOMEM     4  /* device workspace allocation failed */
#define DDM_ERR_CUDA      5  /* a CUDA runtime call or kernel launch failed */
#define DDM_ERR_TIMEOUT   6  /* a bounded device-side wait gave up */
#define DDM_ERR_STATE     7  /* staged call without the build / plan it needs */
#define DDM_ERR_INTERNAL  8  /* checked build (libddm_checked.so) only: a kernel found an
                                index outside its bounds and skipped the access */

/* Flags. */
#define DDM_CLOSED 0u  /* default: closed segments, x.lo <= y.hi && y.lo <= x.hi */
#define DDM_OPEN   1u  /* the strict test of Alg. 1: x.lo < y.hi && y.lo < x.hi */
/* One-shot calls only (ddm_count, ddm_match, ddm_match_range over the whole
 * update range): build the tree over the UPDATE set and run one query per
 * subscription -- the roles of the two sets swapped, as Section IV allows
 * for building over the smaller set.  The pair set is the same (pairs still
 * read {upd, sub}); they come grouped by subscription id instead of by
 * update id. */
#define DDM_SWAP_ROLES 2u

#define DDM_MAX_DIMS    8
#define DDM_MAX_EXTENTS 1073741823u  /* 2^30 - 1 per set */

/* One intersecting pair: update id and subscription id (0-based). */
typedef struct {
    uint32_t upd;
    uint32_t sub;
} ddm_pair;

/* Opaque context: owns the device workspace (sort buffers, the tree, the
 * per-update plan) on one device.  Grows on demand, freed by ddm_destroy. */
typedef struct ddm_ctx ddm_ctx;

/* Create a context on CUDA device `device`.  *ctx is set on success.
 * Errors: DDM_ERR_ARG (ctx NULL), DDM_ERR_CUDA (no such device),
 * DDM_ERR_NOMEM. */
int ddm_create(ddm_ctx **ctx, int device);

/* Free a context and its device workspace (NULL is a no-op).  Waits for
 * work the context enqueued to finish. */
int ddm_destroy(ddm_ctx *ctx);

/* Static description of a return code (never NULL). */
const char *ddm_strerror(int code);

/* ---------------------------------------------------------------------- */
/* One-shot calls                                                          */
/* ---------------------------------------------------------------------- */

/* K = number of intersecting (update, subscription) pairs
 * (Section III problem statement; Algs. 4-5 with the d-dimensional test of
 * Section III-A).  Runs validation, the sort and tree build over S, and one
 * counting query per update.  *k_out = K.  Synchronises `stream`.
 * Errors: DDM_ERR_ARG, DDM_ERR_EXTENT, DDM_ERR_NOMEM, DDM_ERR_CUDA,
 * DDM_ERR_TIMEOUT.  Leaves the tree and the plan in the context, as
 * ddm_build + ddm_plan would. */
int ddm_count(ddm_ctx *ctx, int d,
              const float *upd_lo, const float *upd_hi, uint32_t m,
              const float *sub_lo, const float *sub_hi, uint32_t n,
              uint32_t flags, uint64_t *k_out, void *stream);

/* Enumerate all K pairs into pairs[0..K) (device memory, capacity entries).
 * *k_out = K.  If K > capacity: returns DDM_ERR_CAPACITY, *k_out = K and
 * the contents of `pairs` are unspecified (nothing is written past
 * capacity).  The intersection matrix M of Section III is returned in
 * this compressed (coordinate list) form.  Synchronises `stream` once. */
int ddm_match(ddm_ctx *ctx, int d,
              const float *upd_lo, const float *upd_hi, uint32_t m,
              const float *sub_lo, const float *sub_hi, uint32_t n,
              uint32_t flags, ddm_pair *pairs, uint64_t capacity,
              uint64_t *k_out, void *stream);

/* As ddm_match, but only for updates upd_begin <= j < upd_end (ids stay
 * global).  For outputs larger than device memory, call repeatedly over
 * consecutive ranges, or use the staged calls below, which avoid redoing
 * the tree.  Errors as ddm_match, plus DDM_ERR_ARG when the range is not
 * within [0, m], or with DDM_SWAP_ROLES unless the range is [0, m). */
int ddm_match_range(ddm_ctx *ctx, int d,
                    const float *upd_lo, const float *upd_hi, uint32_t m,
                    const float *sub_lo, const float *sub_hi, uint32_t n,
                    uint32_t upd_begin, uint32_t upd_end,
                    uint32_t flags, ddm_pair *pairs, uint64_t capacity,
                    uint64_t *k_out, void *stream);

/* ---------------------------------------------------------------------- */
/* Staged calls: resident tree, per-update plan, chunked output            */
/* ---------------------------------------------------------------------- */

/* Interval-Tree-Create (Alg. 5, Section IV) over the subscriptions:
 * validates S, sorts it by dimension-0 (lower, upper, id) and builds the
 * tree in the context, replacing any previous tree and plan.  The
 * coordinates are copied, so sub_lo / sub_hi may be released afterwards.
 * Synchronises `stream` (to report DDM_ERR_EXTENT). */
int ddm_build(ddm_ctx *ctx, int d, const float *sub_lo, const float *sub_hi,
              uint32_t n, void *stream);

/* In-place refit after the subscriptions moved (dynamic interval
 * management, Section IV): the subscriptions keep their ids and their
 * position in the tree; sub_lo / sub_hi hold their new coordinates (same d
 * and n as the build).  Every node's per-dimension minlower / maxupper is
 * recomputed, so queries stay exact whatever the movement (the tree may
 * prune less once the order no longer follows the lower bounds; a new
 * ddm_build restores it).  Drops the current plan.  Synchronises `stream`.
 * Errors: DDM_ERR_STATE (no own single-problem tree: none built, attached,
 * or batched), DDM_ERR_ARG, DDM_ERR_EXTENT, DDM_ERR_CUDA. */
int ddm_refit(ddm_ctx *ctx, const float *sub_lo, const float *sub_hi, void *stream);

/* Let `ctx` query the tree built in `src` (same device) without copying it:
 * ctx's plans and writes use its own workspace and src's tree, so several
 * contexts can serve requests against one resident tree on separate
 * streams.  The tree must not be rebuilt, refitted or destroyed while an
 * attached context uses it; after a rebuild of src, attach again.  A later
 * ddm_build on ctx makes it own a tree again.  Errors: DDM_ERR_ARG,
 * DDM_ERR_STATE (src has no single-problem tree). */
int ddm_attach(ddm_ctx *ctx, const ddm_ctx *src);

/* Counting pass (Alg. 4 per update, without output) for all m updates
 * against the built tree, and the exclusive prefix sum of the per-update
 * counts.  offsets (optional, device, m + 1 entries of uint64) receives the
 * prefix: update j's pairs are [offsets[j], offsets[j+1]) of the full
 * output, offsets[m] = K.  *k_out = K.  The context keeps the plan (with its
 * own sorted copy of the update coordinates) for ddm_write /
 * ddm_chunk_end, so upd_lo / upd_hi may be released afterwards.  Synchronises
 * `stream`.  Errors: DDM_ERR_STATE (no tree), DDM_ERR_ARG, DDM_ERR_EXTENT,
 * DDM_ERR_NOMEM, DDM_ERR_CUDA, DDM_ERR_TIMEOUT. */
int ddm_plan(ddm_ctx *ctx, const float *upd_lo, const float *upd_hi, uint32_t m,
             uint32_t flags, uint64_t *offsets, uint64_t *k_out, void *stream);

/* Write the pairs of updates upd_begin <= j < upd_end of the current plan
 * into pairs[0 .. offsets[upd_end] - offsets[upd_begin]).  *k_out = that
 * count.  DDM_ERR_CAPACITY (nothing written) if it exceeds capacity.
 * Synchronises `stream`.  Errors: DDM_ERR_STATE (no plan), DDM_ERR_ARG,
 * DDM_ERR_CAPACITY, DDM_ERR_CUDA. */
int ddm_write(ddm_ctx *ctx, uint32_t upd_begin, uint32_t upd_end,
              ddm_pair *pairs, uint64_t capacity, uint64_t *k_out, void *stream);

/* Chunk planning for ddm_write: *upd_end = the largest e <= m such that
 * the pairs of updates [upd_begin, e) fit in `capacity`.  Returns
 * DDM_ERR_CAPACITY with *upd_end = upd_begin when update upd_begin alone
 * does not fit.  Synchronises `stream`. */
int ddm_chunk_end(ddm_ctx *ctx, uint32_t upd_begin, uint64_t capacity,
                  uint32_t *upd_end, void *stream);

/* Host-synchronisation-free staged calls, for request loops that keep
 * several contexts busy on their own streams.  ddm_plan_async enqueues what
 * ddm_plan does (offsets stay inside the context) and returns at once;
 * ddm_write_async enqueues what ddm_write does and then copies the number of
 * pairs written to k_dev[0] and the device error bits to err_dev[0] (1 =
 * invalid extent in the plan's updates, 2 = bounded wait timed out, 4 =
 * more pairs than capacity, nothing written), both DEVICE pointers (either
 * may be NULL; use pinned host memory to read them after a stream event).
 * The calls allocate device memory only when sizes grow beyond earlier
 * calls on the context.  Errors returned directly: DDM_ERR_ARG,
 * DDM_ERR_STATE, DDM_ERR_NOMEM, DDM_ERR_CUDA. */
int ddm_plan_async(ddm_ctx *ctx, const float *upd_lo, const float *upd_hi, uint32_t m,
                   uint32_t flags, void *stream);
int ddm_write_async(ddm_ctx *ctx, uint32_t upd_begin, uint32_t upd_end, ddm_pair *pairs,
                    uint64_t capacity, uint64_t *k_dev, uint32_t *err_dev, void *stream);

/* Work of the last count pass that returned to the host (ddm_count,
 * ddm_match, ddm_match_range, ddm_plan, ddm_batch_match, ddm_match_moved):
 * *leaf_tests = the (query, leaf) tests it made, each one query against the
 * 32 subscriptions of a leaf whose box meets the query's (2d segment
 * comparisons per subscription, Section III-A).  For measurement; the paper
 * has no counterpart. */
int ddm_plan_stats(ddm_ctx *ctx, uint64_t *leaf_tests);

/* Dynamic interval management (Section IV): with a tree over one set kept
 * current (ddm_build, then ddm_refit as its extents move), the row (or
 * column) of every extent of the other set that moved is recomputed by one
 * query against that tree.  This call matches k moved extents (lo, hi:
 * DEVICE SoA of d x k floats, their new coordinates) against the context's
 * tree and writes all their pairs, each moved extent named by ids[j]
 * (DEVICE, k entries; NULL: j itself):
 *  - flags without DDM_SWAP_ROLES: the tree holds the subscriptions and the
 *    moved extents are updates; pairs read {ids[j], subscription id};
 *  - with DDM_SWAP_ROLES: the tree holds the updates and the moved extents
 *    are subscriptions; pairs read {update id, ids[j]};
 *  DDM_OPEN selects the open rule.  Pairs are grouped by moved extent (in
 * the order 0..k-1).  *k_out = pair count; DDM_ERR_CAPACITY as ddm_match.
 * Replaces the context's plan; the tree is unchanged.  Synchronises
 * `stream` once.  Errors: DDM_ERR_ARG, DDM_ERR_STATE (no tree),
 * DDM_ERR_EXTENT, DDM_ERR_CAPACITY, DDM_ERR_NOMEM, DDM_ERR_CUDA. */
int ddm_match_moved(ddm_ctx *ctx, const float *lo, const float *hi, uint32_t k,
                    const uint32_t *ids, uint32_t flags, ddm_pair *pairs, uint64_t capacity,
                    uint64_t *k_out, void *stream);

/* Output offsets of update-id boundaries, for one plan that matches several
 * update sets at once (concatenated, set r holding update ids
 * [upd_off[r], upd_off[r+1])): pair_off[i] = number of pairs of the updates
 * with id < upd_off[i], 0 <= i <= count, i.e. set r's pairs are
 * [pair_off[r], pair_off[r+1]) of the output of ddm_write(0, m) (pairs by
 * update id, Section IV's per-query result lists one after another).
 *  upd_off[count+1]  (DEVICE, uint64) non-decreasing update ids; entries
 *                    above m are read as m;
 *  pair_off[count+1] (DEVICE, uint64) output.
 * Enqueued on `stream` after the plan; no synchronisation, no allocation.
 * DDM_ERR_ARG for NULL pointers, DDM_ERR_STATE without a plan. */
int ddm_pair_offsets_async(ddm_ctx *ctx, const uint64_t *upd_off, uint32_t count,
                           uint64_t *pair_off, void *stream);

/* Plan order.  The counting pass runs the updates in a spatial order (the
 * same order as the tree, so that the 32 queries of a warp lie close
 * together).  Writing ranges of that order keeps every chunk's queries
 * dense, which makes chunked output cheaper than update-id ranges.
 *  order[m]           (optional, device) update id at each plan position;
 *  order_offsets[m+1] (optional, device) exclusive prefix of the counts in
 *                     plan order: position p's pairs are
 *                     [order_offsets[p], order_offsets[p+1]) of an output laid
 *                     out in plan order.
 * Enqueued on `stream`; no synchronisation.  DDM_ERR_STATE without a plan. */
int ddm_plan_order(ddm_ctx *ctx, uint32_t *order, uint64_t *order_offsets, void *stream);

/* Write the pairs of plan positions pos_begin <= p < pos_end into
 * pairs[0 .. order_offsets[pos_end] - order_offsets[pos_begin]), grouped by
 * update in plan order (each update's pairs in tree order).  *k_out = that
 * count; DDM_ERR_CAPACITY (nothing written) if it exceeds capacity.
 * Synchronises `stream`.  Errors as ddm_write. */
int ddm_write_ordered(ddm_ctx *ctx, uint32_t pos_begin, uint32_t pos_end,
                      ddm_pair *pairs, uint64_t capacity, uint64_t *k_out, void *stream);

/* Compressed output (Section III: the intersection matrix M is sparse and
 * can be stored in compressed form).  Writes what ddm_write_ordered writes
 * for plan positions pos_begin <= p < pos_end, but only the subscription id
 * of each pair (uint32; instance-local when batched), at the same index:
 * sub_ids[0 .. order_offsets[pos_end] - order_offsets[pos_begin]).  With
 * ddm_plan_order's order (the update at each plan position) and
 * order_offsets (where each position's ids start) this is M stored by
 * columns, one column per update holding the ids of the subscriptions it
 * overlaps, in half the bytes of the pair list.  capacity counts ids.
 * *k_out = the id count; DDM_ERR_CAPACITY (nothing written) if it exceeds
 * capacity.  Each id is an index into the set the tree was built over
 * (DDM_SWAP_ROLES does not apply).  Synchronises `stream`.  Errors as
 * ddm_write_ordered. */
int ddm_write_ordered_ids(ddm_ctx *ctx, uint32_t pos_begin, uint32_t pos_end,
                          uint32_t *sub_ids, uint64_t capacity, uint64_t *k_out, void *stream);

/* Chunk planning for ddm_write_ordered (and ddm_write_ordered_ids, whose
 * capacity counts ids): *pos_end = the largest e <= m such
 * that the pairs of plan positions [pos_begin, e) fit in `capacity`;
 * DDM_ERR_CAPACITY with *pos_end = pos_begin when position pos_begin alone
 * does not fit.  Synchronises `stream`. */
int ddm_chunk_end_ordered(ddm_ctx *ctx, uint32_t pos_begin, uint64_t capacity,
                          uint32_t *pos_end, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched instances                                                       */
/* ---------------------------------------------------------------------- */

/* Match `count` independent problems in one call (the per-update queries of
 * every instance are independent, Section IV "Parallelizing ITM", so all
 * instances share one sort, one tree build, one counting launch and one
 * write launch).  Instance i's updates are positions
 * [upd_off[i], upd_off[i+1]) of one SoA update array of m_total extents
 * (row k at k*m_total); its subscriptions are positions
 * [sub_off[i], sub_off[i+1]) of one SoA subscription array of n_total
 * extents.  upd_off / sub_off: DEVICE arrays of count + 1 nondecreasing
 * uint64 with upd_off[0] = sub_off[0] = 0, upd_off[count] = m_total,
 * sub_off[count] = n_total (not checked; empty instances are allowed).
 * An update only matches subscriptions of its own instance.  Pairs carry
 * instance-local ids (update j of instance i is upd_off[i] + j of the
 * array); they are grouped by instance, then by update.  pair_off
 * (optional, DEVICE, count + 1 uint64) receives each instance's first pair;
 * pair_off[count] = K.  *k_out = K.  DDM_ERR_CAPACITY when K > capacity
 * (nothing written).  Synchronises `stream` once.  Errors: DDM_ERR_ARG
 * (count 0, NULL offsets, ...), DDM_ERR_EXTENT, DDM_ERR_CAPACITY,
 * DDM_ERR_NOMEM, DDM_ERR_CUDA, DDM_ERR_TIMEOUT.  Afterwards the staged
 * single-problem calls report DDM_ERR_STATE until the next ddm_build. */
int ddm_batch_match(ddm_ctx *ctx, int d, uint32_t count,
                    const float *upd_lo, const float *upd_hi, const uint64_t *upd_off,
                    uint32_t m_total,
                    const float *sub_lo, const float *sub_hi, const uint64_t *sub_off,
                    uint32_t n_total,
                    uint32_t flags, ddm_pair *pairs, uint64_t capacity, uint64_t *pair_off,
                    uint64_t *k_out, void *stream);

/* As ddm_batch_match without any host synchronisation, so that the call can
 * be recorded into a CUDA graph: K goes to k_dev[0] and the device error
 * bits to err_dev[0] (1 = invalid extent, 2 = bounded wait timed out,
 * 4 = more pairs than capacity, nothing written), both DEVICE pointers
 * (either may be NULL).  The call allocates device memory when its sizes
 * grow, which a captured stream does not allow: make one ddm_batch_match
 * (or ddm_batch_match_async) call with the same sizes before capturing.
 * Returns DDM_OK once the work is enqueued. */
int ddm_batch_match_async(ddm_ctx *ctx, int d, uint32_t count,
                          const float *upd_lo, const float *upd_hi, const uint64_t *upd_off,
                          uint32_t m_total,
                          const float *sub_lo, const float *sub_hi, const uint64_t *sub_off,
                          uint32_t n_total,
                          uint32_t flags, ddm_pair *pairs, uint64_t capacity, uint64_t *pair_off,
                          uint64_t *k_dev, uint32_t *err_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Introspection of the built tree (for checking intermediate results)     */
/* ---------------------------------------------------------------------- */

/* Shape of the implicit tree: *levels = number of internal levels L;
 * counts[l-1] (l = 1..L, at most DDM_MAX_TREE_LEVELS entries) = nodes at
 * level l.  Level-l node g covers the sorted positions
 * [g * 32^l, min(n, (g+1) * 32^l)).  *total = sum of counts. */
#define DDM_MAX_TREE_LEVELS 8
int ddm_tree_shape(ddm_ctx *ctx, int *levels, uint32_t *counts, uint32_t *total);

/* Copy the tree to caller device memory (any pointer may be NULL):
 *  order[n]         -- subscription id at each sorted position (tree order);
 *  node_lo[d*total] -- per dimension k and node, the minimum lower bound of
 *                      the node's range (minlower of Section IV);
 *  node_hi[d*total] -- per dimension k and node, the maximum upper bound of
 *                      the node's range (maxupper of Section IV);
 * entry [k*total + j]: nodes are stored level by level from level 1, in
 * node order, so level l starts at sum of counts[0..l-2].
 * Enqueued on `stream`; no synchronisation.  DDM_ERR_STATE without a tree. */
int ddm_tree_export(ddm_ctx *ctx, uint32_t *order, float *node_lo, float *node_hi,
                    void *stream);

/* Record budget of the write pass.  While counting, ddm_plan (and the
 * one-shot calls) can keep a compact record of every (update, leaf) test
 * that found pairs -- 10 bytes per record plus 64 bytes per block of 512
 * records, about one record per 12 pairs on clustered d = 3 extents --
 * so that the write pass expands the records instead of walking the tree a
 * second time.  The records live in a context arena of at most `bytes`
 * (default: a quarter of the device's memory); the arena is sized from what
 * the previous count pass needed, so the first plan on a large workload may
 * run out of room and fall back to walking.  Results are identical either
 * way.  0 turns recording off.  DDM_ERR_ARG for a NULL context. */
int ddm_set_replay_budget(ddm_ctx *ctx, uint64_t bytes);

/* Tuning knobs (results never depend on them), picked per workload by the
 * autotuner in the Python package:
 *  str_shift   -- added to every re-sort group exponent of the tree order
 *                 (-4..4; 0 = sort-tile-recursive sizes);
 *  ctas_per_sm -- 256-thread CTAs per SM of the query kernels (1..32,
 *                 default 8; the kernels are persistent);
 *  replay      -- nonzero: the write pass may replay the count pass's
 *                 records; 0: it walks the tree again.
 * DDM_ERR_ARG outside these ranges. */
int ddm_set_tuning(ddm_ctx *ctx, int str_shift, uint32_t ctas_per_sm, uint32_t replay);

/* Tiling of the query kernels (speed only, never results; the autotuner in
 * the Python package picks it per workload):
 *  queries_per_packet -- 16 or 32 queries walk the tree together in one warp
 *                        (default 32; the leaves keep 32 subscriptions, one
 *                        per lane);
 *  swap_min           -- 1..33: a leaf met by at least this many of a
 *                        packet's queries is tested with lane = query: for
 *                        d <= 3 from the leaf's rank tables (its bounds
 *                        sorted per dimension, built with the tree), each
 *                        lane finding its query's matches in the leaf by
 *                        binary searches; for d > 3 by comparing the leaf's
 *                        32 subscriptions one by one, from max(swap_min, 24)
 *                        queries on.  33 = never (default 12).
 * Changing queries_per_packet drops the current plan (its records are laid
 * out by packet).  DDM_ERR_ARG outside these values or for a NULL context.
 * The paper has no counterpart (Section IV's queries run one per thread). */
int ddm_set_tiling(ddm_ctx *ctx, uint32_t queries_per_packet, uint32_t swap_min);

/* Update-id base for sharded matching (Section IV, "Parallelizing ITM":
 * queries are independent, so one problem's update set can be split into
 * contiguous ranges matched on different GPUs against the same
 * subscriptions).  Every pair this context writes afterwards carries update
 * id base + j for its update at local position j: ddm_write,
 * ddm_write_ordered, ddm_match and ddm_match_range without DDM_SWAP_ROLES,
 * and ddm_match_moved without ids.  The shard holding global updates
 * [base, base + m) thus writes the same pairs, in the same order, as one
 * ddm_match over the whole update set writes for those updates.  Not applied
 * to the compressed output (subscription ids only), to ddm_plan_order's
 * order (local ids), to batched calls or to swapped roles.  Default 0; a
 * write whose base + m exceeds 2^32 returns DDM_ERR_ARG.  DDM_ERR_ARG for a
 * NULL context.  The paper has no counterpart. */
int ddm_set_update_id_base(ddm_ctx *ctx, uint32_t base);

/* Testing aid: make device workspace allocations that would bring the
 * context's total above `bytes` fail with DDM_ERR_NOMEM (0 = no limit). */
int ddm_debug_set_alloc_limit(ddm_ctx *ctx, uint64_t bytes);

/* ---------------------------------------------------------------------- */
/* Allocation-free offsets scan                                            */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory when they need it: real-time loops that must not
 * block in the allocator (cudaMalloc and cudaFree can synchronise the whole
 * device), and hosts whose device memory all belongs to another allocator.
 *
 * Exclusive prefix sum of per-update match counts: offsets[j] =
 * counts[0] + ... + counts[j-1] for j <= m, so update j's pairs are
 * [offsets[j], offsets[j+1]) of a pair list grouped by update and
 * offsets[m] = K -- the same result as the offsets of ddm_plan for the same
 * counts.  counts (m uint32) and offsets (m + 1 uint64) are DEVICE pointers
 * of the current device, owned by the caller; work is enqueued on `stream`
 * and nothing is synchronised or allocated.  offsets must not be NULL;
 * counts may be NULL only when m == 0 (offsets[0] = 0 is then written).
 * Scratch is a fixed device array inside the library, so m must not exceed
 * DDM_NOALLOC_MAX_UPDATES (DDM_ERR_ARG otherwise, and for a NULL pointer the
 * call needs).  The array is shared by every call on a device and keeps the
 * last call's tile sums; every call rewrites the sums it reads, so nothing
 * needs clearing, but calls whose work may overlap on the GPU race and must
 * be serialised by the caller.  The first call on a device looks up the
 * array's device address (DDM_ERR_CUDA if that fails); make that first call
 * before any stream capture. */
#define DDM_NOALLOC_MAX_UPDATES 67108864u  /* 2^26 updates: 128 KiB of scratch */
int ddm_scan_counts_noalloc(const uint32_t *counts, uint32_t m, uint64_t *offsets,
                            void *stream);

/* Test hook for the bounded device waits (failure detection without a
 * fault): one warp polls a device word that nothing sets, with the same
 * bounded wait as the sort's look-back, at most `polls` times (1..2^22, 64 ns
 * apart), then records the timeout.  Returns DDM_ERR_TIMEOUT; the context
 * stays usable.  DDM_ERR_ARG for polls out of range.  The paper has no
 * counterpart. */
int ddm_debug_wait_timeout(ddm_ctx *ctx, uint32_t polls, void *stream);

/* Number of CUDA kernels this library has launched in the calling process
 * since it was loaded (all contexts).  Host-side counter, no GPU access. */
uint64_t ddm_debug_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DDM_H */
