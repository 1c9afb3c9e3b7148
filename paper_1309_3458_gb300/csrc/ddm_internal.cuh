// Internal declarations shared by the libddm translation units.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ddm.h"

namespace ddm {

// Tree fan-out: one warp lane per child, so a node's 32 children are tested
// by one coalesced load and one ballot.
constexpr int kFan = 32;
constexpr int kLog2Fan = 5;
constexpr int kMaxLevels = DDM_MAX_TREE_LEVELS;

// Device error bits (Status::err).
constexpr unsigned kErrExtent = 1u;
constexpr unsigned kErrTimeout = 2u;
constexpr unsigned kErrCapacity = 4u;
constexpr unsigned kErrChecked = 8u;  // checked build: an index failed its bounds check

// Device-resident status word read back once per synchronising call.
struct Status {
  unsigned long long K;    // pairs counted (plan) or written (write)
  unsigned int err;        // kErr* bits
  unsigned int pad;
  unsigned long long aux;  // call-specific (chunk end, ...)
  unsigned long long tests;  // count pass: (query, leaf) tests, 32 subscriptions each
};

__device__ inline void note_out_of_bounds(Status* st) {
  if (st) atomicOr(&st->err, kErrChecked);
}

// Checked build (compiled with DDM_CHECKED, as libddm_checked.so): kernels
// verify the indices they are about to use, and an index out of its bounds
// sets kErrChecked in the status word (the call returns DDM_ERR_INTERNAL)
// and the access is skipped -- never a trap.  In the normal build the check
// is the constant true and costs nothing.
#ifdef DDM_CHECKED
#define DDM_IN_BOUNDS(cond, st) ((cond) ? true : (::ddm::note_out_of_bounds(st), false))
#else
#define DDM_IN_BOUNDS(cond, st) true
#endif

struct Status;
__device__ inline void note_out_of_bounds(Status* st);

// Read-only view of a built tree, passed to kernels by value.
//
// Elements (the subscriptions) sit at sorted positions 0..n-1; a level-l
// node g covers positions [g*32^l, min(n, (g+1)*32^l)) and stores, per
// dimension k, (minlower, maxupper) of the extents in its range.
struct TreeView {
  int d;
  uint32_t n;
  int L;                          // internal levels 1..L; level L has <= 32 nodes
  uint32_t cnt[kMaxLevels + 1];   // nodes per level (index 1..L)
  uint32_t off[kMaxLevels + 1];   // first node of each level within one dimension
  uint32_t total;                 // nodes per dimension
  const float2* e;                // [d][n] (lo, hi) per dimension, sorted order
  const uint32_t* sid;            // [n] subscription id per sorted position
  const float2* nodes;            // [d][total] (minlower, maxupper) per dimension
  // Rank tables (d <= 3, else null): per leaf g and slot 2k (lower bounds of
  // dimension k) / 2k + 1 (upper bounds), kRankSlot words at
  // (g * 2d + slot) * kRankSlot: the leaf's 32 bounds sorted ascending (float
  // bits, padding positions +inf), then at word 35 + c the mask of the leaf
  // positions holding the c smallest (c = 0..32).
  const uint32_t* tab;
};
constexpr uint32_t kRankSlot = 68;  // words per rank-table slot (16-byte multiple)

// Read-only view of the planned updates (queries) in their sorted order.
struct QueryView {
  uint32_t m;
  const float2* qe;               // [d][m] (lo, hi) per dimension, sorted order
  const uint32_t* qid;            // [m] update id per sorted position
  const uint32_t* list;           // optional subset of sorted positions (ranges)
  uint32_t first;                 // without list: run positions first .. first+nq-1
  uint32_t nq;                    // number of queries to run
  uint32_t qpp_log2;              // log2 of the queries per packet (4 or 5: 16 or 32)
  uint32_t tmin;                  // count pass: swapped leaf loops from this many queries
};

// Where the write pass puts each query's pairs: query j's pairs start at
// start[key] - start[b_idx] in `pairs`, key = its update id (by_pos false) or
// its sorted position (by_pos true); start[e_idx] - start[b_idx] pairs in all.
struct WriteView {
  const unsigned long long* start;
  bool by_pos;
  bool swap;  // roles swapped: the tree holds the updates, queries are subscriptions
  const uint32_t* qids;  // optional: id written for query q is qids[q] (else q + qbase)
  uint32_t qbase;        // added to every update id written (a shard's first global id)
  uint32_t b_idx, e_idx;
  ddm_pair* pairs;
  uint32_t* ids;  // when set: only each pair's subscription id is written, here, and pairs is unused
  unsigned long long capacity;
};

// Batched instances: instance i owns update positions [upd_off[i],
// upd_off[i+1]) and subscription positions [sub_off[i], sub_off[i+1]) of the
// concatenated sets; sorting keeps these ranges (the instance is the major
// key), so they hold in sorted order too.  q_inst[p] = instance of the update
// at sorted position p.  count == 0: a single problem.
struct BatchView {
  uint32_t count;
  const unsigned long long* upd_off;  // [count + 1]
  const unsigned long long* sub_off;  // [count + 1]
  const uint32_t* q_inst;             // [m]
};

// Exponent of the sort-tile-recursive group size for re-sorting dimension k
// (1 <= k < d) of a set of n extents: with nb = n/32 leaves each dimension
// gets about nb^(1/d) slabs, so dimension k is re-sorted inside groups of
// 32 * nb^((d-k)/d) positions, rounded to a power of two.  0 = no re-sort
// (groups of fewer than 64 would not change any leaf's box).
__host__ __device__ inline int str_group_log2(uint32_t n, int d, int k, int shift = 0) {
  if (n < 64u) return 0;
  const double nb = (double)((n + 31u) / 32u);
  const double G = 32.0 * pow(nb, (double)(d - k) / (double)d);
  const int g = (int)floor(log2(G) + 0.5) + shift;
  if (g < 6 || (1ull << g) >= (unsigned long long)n) return 0;
  return g;
}

// Order-preserving map from float to uint32 (IEEE order; -0 maps like +0).
__host__ __device__ inline uint32_t float_key(float f) {
#ifdef __CUDA_ARCH__
  uint32_t b = __float_as_uint(f);
#else
  uint32_t b;
  __builtin_memcpy(&b, &f, 4);
#endif
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Number of kernels this library has launched in the process (all
// contexts), for launch accounting by callers; defined in ddm_api.cu.
void note_launches(unsigned count);

// ---- ddm_layout.cu --------------------------------------------------------
// Validate a set (lo <= hi, no NaN in every dimension) and, when keys is
// not null, emit the sort key with the identity payload: key_mode 1 gives
// (key(lo0) << 32 | key(hi0)) (tree order), key_mode 2 gives key(lo0).
// aos (optional, cnt * d float2): an interleaved copy of the coordinates,
// aos[i*d + k] = (lo_k, hi_k) of extent i, written while validating, so that
// the gathers by id read one contiguous record per extent instead of 2d
// scattered words.
cudaError_t launch_validate(int d, const float* lo, const float* hi, uint32_t cnt,
                            unsigned long long* keys, uint32_t* vals, int key_mode, float2* aos,
                            Status* st, int sms, cudaStream_t s);
// keys[i] = (i >> glog2) << 32 | key(lo_k[vals[i]]): re-sort inside groups.
cudaError_t launch_rekey(const uint32_t* vals, const float* lo_k, uint32_t cnt, int glog2,
                         unsigned long long* keys, int sms, cudaStream_t s);
// Batched sets: inst[i] = instance owning position i (off has count+1 entries).
// Validation and class-major tree keys for d >= 2; hist[256] (zeroed by the
// caller) receives the number of extents of each size class.
cudaError_t launch_validate_class(int d, const float* lo, const float* hi, uint32_t cnt,
                                  unsigned long long* keys, uint32_t* vals, uint32_t* hist,
                                  float2* aos, Status* st, int sms, cudaStream_t s);
// inst[i] = the b with off[b] <= i < off[b+1], for 0 <= i < total.
cudaError_t launch_fill_inst(const unsigned long long* off, uint32_t count, uint32_t total,
                             uint32_t* inst, int sms, cudaStream_t s);
// Batched validation + keys: keys[i] = inst[i] << 32 | key(lo0[i]).
cudaError_t launch_validate_batch(int d, const float* lo, const float* hi, uint32_t cnt,
                                  const uint32_t* inst, unsigned long long* keys, uint32_t* vals,
                                  float2* aos, Status* st, int sms, cudaStream_t s);
// Per instance and dimension k >= 1: group exponent (0 = groups of 1) and
// group count, for the batched re-sorts.  glog2/ngroups: [count] each.
cudaError_t launch_batch_groups(const unsigned long long* off, uint32_t count, int d, int k,
                                int shift, int* glog2, uint32_t* ngroups, cudaStream_t s);
// Batched re-sort keys: group = gbase[inst] + (local position >> glog2[inst]).
cudaError_t launch_rekey_batch(const uint32_t* vals, const float* lo_k, uint32_t cnt,
                               const uint32_t* inst, const unsigned long long* off,
                               const int* glog2, const unsigned long long* gbase,
                               unsigned long long* keys, int sms, cudaStream_t s);
// qe[k][i] = (lo_k, hi_k)[vals[i]], qid[i] = vals[i].
cudaError_t launch_gather(int d, const uint32_t* vals, const float* lo, const float* hi,
                          const float2* aos, uint32_t cnt, float2* qe, uint32_t* qid, int sms,
                          cudaStream_t s);

// ---- ddm_sort.cu ----------------------------------------------------------
struct SortScratch {
  unsigned long long* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;       // [8][256]
  uint32_t* lookback;   // [8][tiles][256], or the cooperative sort's scratch
  uint32_t* counters;   // [8]
};
constexpr int kSortTile = 4096;
size_t sort_lookback_words(uint32_t n);
// Stable LSD radix sort on the low 8*passes bits of 64-bit keys, with a
// uint32 payload (one cluster, one cooperative launch or onesweep, by size).
// Input in keys[0]/vals[0]; *out_buf receives the index (0 or 1) of the
// buffers holding the result.
// Test hook: one warp polls `word` (which nothing sets) with the sort's
// bounded wait, at most `limit` polls, and records kErrTimeout.
cudaError_t launch_debug_wait(const uint32_t* word, uint32_t limit, Status* st, cudaStream_t s);
cudaError_t launch_sort64(SortScratch sc, uint32_t n, int passes, int* out_buf, Status* st,
                          int sms, cudaStream_t s);

// ---- ddm_tree.cu ----------------------------------------------------------
void tree_shape(uint32_t n, int* L, uint32_t* cnt, uint32_t* off, uint32_t* total);
// Group sizes (log2) of the per-dimension re-sorts: dimension k >= 1 is
// re-sorted by lower bound inside aligned groups of 2^glog2[k] positions;
// `shift` is added to every exponent (tuning knob, 0 = the STR sizes).
void str_groups(uint32_t n, int d, int* glog2, int shift = 0);
cudaError_t launch_build(const TreeView& t, const uint32_t* sorted_ids, const float* lo,
                         const float* hi, const float2* aos, float2* e, uint32_t* sid,
                         float2* nodes, uint32_t* tab, Status* st, cudaStream_t s);
cudaError_t launch_export_nodes(const TreeView& t, float* node_lo, float* node_hi, cudaStream_t s);

// ---- ddm_query.cu ---------------------------------------------------------
// Replay records.  While counting, every (query, leaf) test of a packet
// that has hits is stored as one record of ten bytes: x = leaf << 5 | query
// lane, the hit mask over the leaf's 32 subscriptions, and (16 bits) the
// query's matches before this leaf counted from the start of the record's
// block.  Records of a packet are kept in walk order (leaf by leaf, query
// lanes ascending within a leaf), in chains of fixed-size blocks taken from a
// shared arena; a block stores its packet, and a header with the matches each
// query of its chain had before the block's first record, so that a record's
// place in its query's output is the header entry plus its 16-bit count (a
// block holds at most 512 records of at most 32 hits: the count stays below
// 2^14).  After counting, the blocks are listed in plan order and the write
// pass expands any range of them, every record independently, instead of
// walking the tree again.
constexpr uint32_t kRecBlock = 512;  // records per block: x and hit mask 2 KiB each, counts 1 KiB
constexpr uint32_t kRecHdr = 16;     // header: one running count per query of the chain
// words per block: x[kRecBlock], hit mask[kRecBlock], 16-bit counts, header
constexpr uint32_t kRecWords = 2 * kRecBlock + kRecBlock / 2 + kRecHdr;
// A packet's records go to two chains of blocks, one per half of its query
// lanes, so that a block holds the records of at most 16 queries (its pairs
// land in fewer output runs): the write pass took 127 instead of 134 ms on
// the clustered d = 3 workload, the count pass 5 ms more.  Chain c of packet
// p is chain index p * kRecChains + c of the arena's per-chain arrays.
constexpr uint32_t kRecChains = 2;
constexpr uint32_t kNoBlock = 0xffffffffu;
struct RecordArena {
  uint32_t* rec;           // [max_blocks][kRecWords]: x, hit mask, 16-bit counts, header
  uint32_t* blk_next;      // [max_blocks] next block of the chain, or kNoBlock
  uint32_t* blk_count;     // [max_blocks] records in the block
  uint32_t* blk_pkt;       // [max_blocks] packet of the block
  uint32_t* pkt_first;     // [chains] first block of each chain, or kNoBlock
  uint32_t* pkt_nblk;      // [chains] blocks of each chain
  unsigned long long* pkt_off;  // [chains + 1] exclusive prefix of pkt_nblk
  uint32_t* blk_list;      // [max_blocks] blocks in plan order (packet, then chain)
  uint32_t* blk_counter;   // [0] blocks handed out (may exceed max_blocks),
                           // [1] blocks the whole pass needed, [2] packets,
                           // [3] max_blocks (the last two for arena sizing)
  uint32_t max_blocks;     // 0: no recording
};
// The records of the last count pass are complete (the write pass may
// replay them) iff recording was on and the arena did not run out.
__device__ __forceinline__ bool records_complete(const RecordArena& ra) {
  return ra.max_blocks > 0 && ra.blk_counter[0] <= ra.max_blocks;
}

// counts[update id] (and counts_pos[sorted position], if not null); records
// into `ra` when ra.max_blocks > 0.  With bv.count > 0 every query only
// matches its own instance's subscriptions and pairs carry instance-local ids.
// `sms` sizes the persistent grids: pass SMs x CTAs-per-SM / 8 to change the
// default of 8 CTAs of 256 threads per SM (tuning knob).
cudaError_t launch_count(const TreeView& t, const QueryView& q, const BatchView& bv,
                         uint32_t flags, uint32_t* counts, uint32_t* counts_pos,
                         const RecordArena& ra, uint32_t* work, Status* st, int sms,
                         cudaStream_t s);
// Walking write pass; it does nothing when `ra` holds complete records (the
// replay kernel, launched next to it, writes the pairs then).
cudaError_t launch_write(const TreeView& t, const QueryView& q, const BatchView& bv,
                         uint32_t flags, const WriteView& w, const RecordArena& ra,
                         uint32_t* work, Status* st, int sms, cudaStream_t s);
// After the count pass: blk_list = every chain's blocks, chains in order
// (packets in plan order, a packet's two chains in lane order); pkt_off must
// already hold the prefix of pkt_nblk.
cudaError_t launch_block_list(const RecordArena& ra, uint32_t packets, cudaStream_t s);
// Write pass from records: packets [p0, p1) of the plan, positions [pb, pe),
// and (when id_filter) only updates with ids in [idb, ide).  Does nothing
// unless `ra` holds complete records.
cudaError_t launch_replay(const TreeView& t, const QueryView& q, const BatchView& bv,
                          const RecordArena& ra, const WriteView& w, uint32_t p0, uint32_t p1,
                          uint32_t pb, uint32_t pe, bool id_filter, uint32_t idb, uint32_t ide,
                          uint32_t* work, Status* st, int sms, cudaStream_t s);
// pair_off[i] = offsets[min(upd_off[i], m)] for i <= count.
cudaError_t launch_gather_offsets(const unsigned long long* offsets, uint32_t m,
                                  const unsigned long long* upd_off, uint32_t count,
                                  unsigned long long* pair_off, cudaStream_t s);

// ---- ddm_scan.cu ----------------------------------------------------------
constexpr int kScanTile = 4096;
// offsets[0..m] = exclusive prefix of counts; offsets[m] and st->K = total.
cudaError_t launch_scan(const uint32_t* counts, uint32_t m, unsigned long long* offsets,
                        unsigned long long* block_sums, Status* st, cudaStream_t s);
// Up to kMaxScanJobs independent scans of the form above in one launch
// sequence (three launches, or one when every job has m <= kScanTile).
// Each job's `sums` needs max(1, ceil(m / kScanTile)) entries of its own.
struct ScanJob {
  const uint32_t* counts;
  uint32_t m;
  unsigned long long* offsets;
  unsigned long long* sums;
  Status* st;
};
constexpr int kMaxScanJobs = 3;
cudaError_t launch_scan_multi(const ScanJob* jobs, int count, cudaStream_t s);
cudaError_t launch_chunk_end(const unsigned long long* offsets, uint32_t m, uint32_t begin,
                             unsigned long long capacity, Status* st, cudaStream_t s);
// list = sorted positions i (ascending) with begin <= qid[i] < end; uses
// flags/offs/sums as scratch.
cudaError_t launch_select(const uint32_t* qid, uint32_t m, uint32_t begin, uint32_t end,
                          uint32_t* flags, unsigned long long* offs, unsigned long long* sums,
                          uint32_t* list, Status* st, cudaStream_t s);

}  // namespace ddm
