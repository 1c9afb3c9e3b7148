// Host side of the C ABI (include/ddm.h): argument checks, device workspace,
// stream-ordered launches and the single status read-back per call.
#include <algorithm>
#include <utility>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "ddm_internal.cuh"

using namespace ddm;

namespace {
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void ddm::note_launches(unsigned count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct ddm_ctx {
  int device = 0;
  int sms = 0;
  uint64_t alloc_limit = 0;  // 0 = unlimited (testing aid)
  uint64_t allocated = 0;

  // Workspace comes from the context's own memory pool, allocated and freed
  // in stream order on the calling stream: growing a buffer never
  // synchronises the device (cudaMalloc / cudaFree would), so one context's
  // growth does not stall the work of others.  The pool keeps what is freed
  // (no release threshold) for the next growth.
  cudaMemPool_t pool = nullptr;
  cudaStream_t cur = nullptr;      // stream of the call in progress
  bool capturing = false;          // that stream is being captured into a graph
  // Calls may come on different streams: each call records `done` on its
  // stream when it has enqueued its work, and a call on another stream first
  // waits for it, so the context's buffers are never used by two streams at
  // once and a stream-ordered free never overtakes earlier work.
  cudaEvent_t done = nullptr;
  cudaStream_t last = nullptr;
  bool done_pending = false;

  Status* st_dev = nullptr;
  Status* st_host = nullptr;  // pinned mirror

  // sort scratch (shared by the subscription and the update sorts)
  DevBuf keys[2], vals[2], hist, lookback, counters;
  // tree
  DevBuf e, sid, nodes, tab;
  bool tables_on = true;        // rank tables of the leaves (ddm_set_tiling)
  // plan: sorted updates, per-update counts and offsets
  DevBuf qe, qid, counts, counts_pos, offsets, pos_offsets, sums, work;
  // range selection for ddm_write over a sub-range of updates
  DevBuf sel_offs, sel_list;
  // replay records of the count pass
  DevBuf rec, blk_next, blk_count, blk_pkt, pkt_first, pkt_nblk, pkt_off, blk_list,
      blk_counter;
  uint64_t replay_budget = 0;   // bytes; 0 = never record
  uint32_t rec_blocks = 0;      // blocks of the current arena
  // Blocks needed, packets and blocks held by the latest recorded count
  // pass, copied back by every plan without a host synchronisation (pinned;
  // read as a sizing hint for the next arena, possibly one plan stale).
  volatile uint32_t* rec_hint = nullptr;
  RecordArena arena{};          // arena of the current plan (max_blocks 0 = none)
  // batched instances
  DevBuf inst_s, inst_u, bglog2, bngroups, bgbase;
  // size classes of the tree order (d >= 2)
  DevBuf cls_hist, cls_off;
  DevBuf probe;                 // word polled by ddm_debug_wait_timeout
  DevBuf aos;                   // interleaved coordinates of the set being ordered
  BatchView bv{};               // count 0 = single problem
  // tuning knobs (ddm_set_tuning)
  int str_shift = 0;            // added to the re-sort group exponents
  uint32_t ctas_per_sm = 8;     // CTAs per SM of the packet kernels
  bool replay_on = true;        // record / replay write pass allowed
  uint32_t upd_base = 0;        // added to update ids in written pairs (ddm_set_update_id_base)
  // tiling (ddm_set_tiling): log2 of the queries per packet, and the number of
  // a packet's queries meeting a leaf from which the count pass swaps the loops
  uint32_t qpp_log2 = 5;
  uint32_t tmin = 12;

  bool built = false;
  bool attached = false;        // tree borrowed from another context (ddm_attach)
  bool swapped = false;         // one-shot call with DDM_SWAP_ROLES: tree over the updates
  uint64_t last_tests = 0;      // (query, leaf) tests of the last count pass read back
  TreeView tree{};
  bool planned = false;
  const float* ulo = nullptr;
  const float* uhi = nullptr;
  uint32_t m = 0;
  uint32_t flags = 0;
};

namespace {

// NVTX range around a phase of a call (tree build, plan, write pass, refit),
// so that a timeline tool shows the library's phases by name.  NVTX is
// header-only and costs nothing when no tool is attached.
class Phase {
 public:
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    ok_ = cudaGetDevice(&prev_) == cudaSuccess;
    if (ok_ && prev_ != dev) ok_ = cudaSetDevice(dev) == cudaSuccess;
    switched_ = ok_ && prev_ != dev;
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false, switched_ = false;
};

// Orders a call's work after the context's previous call (made on another
// stream) and marks its end; binds the call's stream for ensure().  A stream
// being captured into a graph is neither waited on nor recorded (its work runs
// only when the graph is launched); growth is refused while capturing.
class StreamUse {
 public:
  StreamUse(ddm_ctx* c, cudaStream_t s) : c_(c), s_(s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
      cudaGetLastError();
      st = cudaStreamCaptureStatusNone;
    }
    capturing_ = st != cudaStreamCaptureStatusNone;
    if (!capturing_ && c->done_pending && c->last != s) cudaStreamWaitEvent(s, c->done, 0);
    c->cur = s;
    c->capturing = capturing_;
  }
  ~StreamUse() {
    if (!capturing_ && cudaEventRecord(c_->done, s_) == cudaSuccess) {
      c_->done_pending = true;
      c_->last = s_;
    }
    cudaGetLastError();
    c_->capturing = false;
  }

 private:
  ddm_ctx* c_;
  cudaStream_t s_;
  bool capturing_ = false;
};

int ensure(ddm_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return DDM_OK;
  if (c->capturing) return DDM_ERR_NOMEM;  // a graph cannot own the workspace
  size_t want = bytes + bytes / 4;  // headroom against regrowth
  if (b.p) {
    cudaFreeAsync(b.p, c->cur);  // after the work already enqueued on this stream
    c->allocated -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  if (c->alloc_limit && c->allocated + want > c->alloc_limit) {
    want = bytes;
    if (c->allocated + want > c->alloc_limit) return DDM_ERR_NOMEM;
  }
  if (cudaMallocFromPoolAsync(&b.p, want, c->pool, c->cur) != cudaSuccess) {
    cudaGetLastError();  // clear the allocation error
    b.p = nullptr;
    return DDM_ERR_NOMEM;
  }
  b.cap = want;
  c->allocated += want;
  return DDM_OK;
}

// Interleaved copy of a set's coordinates for the gathers by id; NULL (the
// gathers then read the caller's rows) if it cannot be allocated.
float2* aos_buffer(ddm_ctx* c, int d, uint32_t cnt) {
  if (cnt == 0 || ensure(c, c->aos, sizeof(float2) * (size_t)d * cnt) != DDM_OK) return nullptr;
  return static_cast<float2*>(c->aos.p);
}

void release(DevBuf& b) {
  if (b.p) cudaFreeAsync(b.p, nullptr);
  b.p = nullptr;
  b.cap = 0;
}

#define DDM_TRY(expr)              \
  do {                             \
    int rc_ = (expr);              \
    if (rc_ != DDM_OK) return rc_; \
  } while (0)
#define DDM_CUDA(expr)                    \
  do {                                    \
    if ((expr) != cudaSuccess) {          \
      cudaGetLastError();                 \
      return DDM_ERR_CUDA;                \
    }                                     \
  } while (0)

bool set_ok(int d, const float* lo, const float* hi, uint32_t cnt) {
  if (cnt > DDM_MAX_EXTENTS) return false;
  if (cnt > 0 && (!lo || !hi)) return false;
  (void)d;
  return true;
}

int sync_status(ddm_ctx* c, cudaStream_t s) {
  DDM_CUDA(cudaMemcpyAsync(c->st_host, c->st_dev, sizeof(Status), cudaMemcpyDeviceToHost, s));
  DDM_CUDA(cudaStreamSynchronize(s));
  return DDM_OK;
}

int status_code(const Status& st) {
  if (st.err & kErrChecked) return DDM_ERR_INTERNAL;
  if (st.err & kErrTimeout) return DDM_ERR_TIMEOUT;
  if (st.err & kErrExtent) return DDM_ERR_EXTENT;
  if (st.err & kErrCapacity) return DDM_ERR_CAPACITY;
  return DDM_OK;
}

int ensure_sort(ddm_ctx* c, uint32_t cnt) {
  DDM_TRY(ensure(c, c->keys[0], sizeof(unsigned long long) * cnt));
  DDM_TRY(ensure(c, c->keys[1], sizeof(unsigned long long) * cnt));
  DDM_TRY(ensure(c, c->vals[0], sizeof(uint32_t) * cnt));
  DDM_TRY(ensure(c, c->vals[1], sizeof(uint32_t) * cnt));
  DDM_TRY(ensure(c, c->hist, sizeof(uint32_t) * 8 * 256));
  DDM_TRY(ensure(c, c->counters, sizeof(uint32_t) * 8));
  DDM_TRY(ensure(c, c->lookback, sizeof(uint32_t) * sort_lookback_words(cnt)));
  return DDM_OK;
}

// Radix sort of the keys/ids in buffer pair `cur` over `passes` 8-bit
// digits; `cur` is updated to the buffer pair holding the result.
int sort_pass(ddm_ctx* c, uint32_t cnt, int passes, int* cur, cudaStream_t s) {
  SortScratch sc;
  sc.keys[0] = static_cast<unsigned long long*>(c->keys[*cur].p);
  sc.keys[1] = static_cast<unsigned long long*>(c->keys[*cur ^ 1].p);
  sc.vals[0] = static_cast<uint32_t*>(c->vals[*cur].p);
  sc.vals[1] = static_cast<uint32_t*>(c->vals[*cur ^ 1].p);
  sc.hist = static_cast<uint32_t*>(c->hist.p);
  sc.lookback = static_cast<uint32_t*>(c->lookback.p);
  sc.counters = static_cast<uint32_t*>(c->counters.p);
  int out = 0;
  DDM_CUDA(launch_sort64(sc, cnt, passes, &out, c->st_dev, c->sms, s));
  *cur ^= out;
  return DDM_OK;
}

// Sort a set into the spatial order used by the tree: dimension-0 key first,
// then, for each further dimension with a group size, a stable re-sort by
// that dimension's lower bound inside aligned groups.  Validates the set on
// the way.  Returns the buffer pair whose vals hold the order.
// Bytes needed to hold values 0..v.
int key_bytes(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 8;
  }
  return b;
}

// Batched sets: the instance is the major sort key, and each instance's
// re-sort groups are sized from its own extent count.
struct BatchSet {
  const unsigned long long* off;  // [count + 1] positions of each instance
  uint32_t count;
  uint32_t* inst;                 // [cnt] instance of each position (filled here)
};

int order_set_batch(ddm_ctx* c, int d, const float* lo, const float* hi, uint32_t cnt,
                    const BatchSet& bs, float2* aos, int* cur, cudaStream_t s) {
  *cur = 0;
  DDM_TRY(ensure_sort(c, cnt));
  DDM_TRY(ensure(c, c->bglog2, sizeof(int) * (bs.count ? bs.count : 1)));
  DDM_TRY(ensure(c, c->bngroups, sizeof(uint32_t) * (bs.count ? bs.count : 1)));
  DDM_TRY(ensure(c, c->bgbase, sizeof(unsigned long long) * ((size_t)bs.count + 1)));
  DDM_TRY(ensure(c, c->sums, sizeof(unsigned long long) * ((size_t)cnt / kScanTile + (size_t)bs.count / kScanTile + 2)));
  DDM_CUDA(launch_fill_inst(bs.off, bs.count, cnt, bs.inst, c->sms, s));
  DDM_CUDA(launch_validate_batch(d, lo, hi, cnt, bs.inst,
                                 static_cast<unsigned long long*>(c->keys[0].p),
                                 static_cast<uint32_t*>(c->vals[0].p), aos, c->st_dev, c->sms, s));
  DDM_TRY(sort_pass(c, cnt, 3 + key_bytes(bs.count ? bs.count - 1 : 0), cur, s));
  for (int k = 1; k < d; ++k) {
    auto* gl = static_cast<int*>(c->bglog2.p);
    auto* ng = static_cast<uint32_t*>(c->bngroups.p);
    auto* gb = static_cast<unsigned long long*>(c->bgbase.p);
    DDM_CUDA(launch_batch_groups(bs.off, bs.count, d, k, c->str_shift, gl, ng, s));
    DDM_CUDA(launch_scan(ng, bs.count, gb, static_cast<unsigned long long*>(c->sums.p), nullptr, s));
    DDM_CUDA(launch_rekey_batch(static_cast<const uint32_t*>(c->vals[*cur].p), lo + (size_t)k * cnt,
                                cnt, bs.inst, bs.off, gl, gb,
                                static_cast<unsigned long long*>(c->keys[*cur].p), c->sms, s));
    // groups: at most one per instance without re-sort plus cnt / 64
    DDM_TRY(sort_pass(c, cnt, 3 + key_bytes((uint64_t)bs.count + cnt / 64), cur, s));
  }
  return DDM_OK;
}

// Tree order for d >= 2: sort by (size class, lower bound), then refine
// each class by the sort-tile-recursive re-sorts of its own size (the
// per-instance machinery of batched sets, with the classes as instances).
int order_set_classes(ddm_ctx* c, int d, const float* lo, const float* hi, uint32_t cnt,
                      float2* aos, int* cur, cudaStream_t s) {
  constexpr uint32_t kClasses = 256;
  *cur = 0;
  DDM_TRY(ensure_sort(c, cnt));
  DDM_TRY(ensure(c, c->cls_hist, sizeof(uint32_t) * kClasses));
  DDM_TRY(ensure(c, c->cls_off, sizeof(unsigned long long) * (kClasses + 1)));
  DDM_TRY(ensure(c, c->inst_s, sizeof(uint32_t) * cnt));
  DDM_TRY(ensure(c, c->bglog2, sizeof(int) * kClasses));
  DDM_TRY(ensure(c, c->bngroups, sizeof(uint32_t) * kClasses));
  DDM_TRY(ensure(c, c->bgbase, sizeof(unsigned long long) * (kClasses + 1)));
  DDM_TRY(ensure(c, c->sums, sizeof(unsigned long long) * 4));
  auto* hist = static_cast<uint32_t*>(c->cls_hist.p);
  auto* off = static_cast<unsigned long long*>(c->cls_off.p);
  auto* inst = static_cast<uint32_t*>(c->inst_s.p);
  auto* sums = static_cast<unsigned long long*>(c->sums.p);
  DDM_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kClasses, s));
  DDM_CUDA(launch_validate_class(d, lo, hi, cnt, static_cast<unsigned long long*>(c->keys[0].p),
                                 static_cast<uint32_t*>(c->vals[0].p), hist, aos, c->st_dev,
                                 c->sms, s));
  DDM_TRY(sort_pass(c, cnt, 4, cur, s));  // (class, 24-bit lower bound)
  DDM_CUDA(launch_scan(hist, kClasses, off, sums, nullptr, s));
  DDM_CUDA(launch_fill_inst(off, kClasses, cnt, inst, c->sms, s));
  for (int k = 1; k < d; ++k) {
    auto* gl = static_cast<int*>(c->bglog2.p);
    auto* ng = static_cast<uint32_t*>(c->bngroups.p);
    auto* gb = static_cast<unsigned long long*>(c->bgbase.p);
    DDM_CUDA(launch_batch_groups(off, kClasses, d, k, c->str_shift, gl, ng, s));
    DDM_CUDA(launch_scan(ng, kClasses, gb, sums, nullptr, s));
    DDM_CUDA(launch_rekey_batch(static_cast<const uint32_t*>(c->vals[*cur].p), lo + (size_t)k * cnt,
                                cnt, inst, off, gl, gb,
                                static_cast<unsigned long long*>(c->keys[*cur].p), c->sms, s));
    // groups: at most one per class without re-sort plus cnt / 64
    DDM_TRY(sort_pass(c, cnt, 3 + key_bytes((uint64_t)kClasses + cnt / 64), cur, s));
  }
  return DDM_OK;
}

int order_set(ddm_ctx* c, int d, const float* lo, const float* hi, uint32_t cnt, bool tree,
              float2* aos, int* cur, cudaStream_t s) {
  *cur = 0;
  DDM_TRY(ensure_sort(c, cnt));
  DDM_CUDA(launch_validate(d, lo, hi, cnt, static_cast<unsigned long long*>(c->keys[0].p),
                           static_cast<uint32_t*>(c->vals[0].p), tree ? 1 : 2, aos, c->st_dev,
                           c->sms, s));
  DDM_TRY(sort_pass(c, cnt, tree ? 8 : 3, cur, s));
  int glog2[DDM_MAX_DIMS];
  str_groups(cnt, d, glog2, c->str_shift);
  for (int k = 1; k < d; ++k) {
    if (!glog2[k]) continue;
    DDM_CUDA(launch_rekey(static_cast<const uint32_t*>(c->vals[*cur].p), lo + (size_t)k * cnt, cnt,
                          glog2[k], static_cast<unsigned long long*>(c->keys[*cur].p), c->sms, s));
    int gbits = 0;
    while (gbits < 32 && (((uint64_t)(cnt - 1) >> glog2[k]) >> gbits) != 0) ++gbits;
    DDM_TRY(sort_pass(c, cnt, 3 + (gbits + 7) / 8, cur, s));
  }
  return DDM_OK;
}

// Validate S, sort it into tree order and build the tree (steps run on `s`,
// no host synchronisation).
int build_async(ddm_ctx* c, int d, const float* slo, const float* shi, uint32_t n, cudaStream_t s,
                const BatchSet* bs = nullptr) {
  Phase phase("ddm build");
  c->built = false;
  c->attached = false;
  c->swapped = false;
  if (!bs) c->bv = BatchView{};
  c->planned = false;
  TreeView t{};
  t.d = d;
  t.n = n;
  if (n == 0) {
    c->tree = t;
    c->built = true;
    return DDM_OK;
  }
  tree_shape(n, &t.L, t.cnt, t.off, &t.total);
  DDM_TRY(ensure(c, c->e, sizeof(float2) * (size_t)d * n));
  DDM_TRY(ensure(c, c->sid, sizeof(uint32_t) * n));
  DDM_TRY(ensure(c, c->nodes, sizeof(float2) * (size_t)d * t.total));
  int cur = 0;
  float2* aos = aos_buffer(c, d, n);
  if (bs)
    DDM_TRY(order_set_batch(c, d, slo, shi, n, *bs, aos, &cur, s));
  else if (d >= 2)
    DDM_TRY(order_set_classes(c, d, slo, shi, n, aos, &cur, s));
  else
    DDM_TRY(order_set(c, d, slo, shi, n, true, aos, &cur, s));
  t.e = static_cast<const float2*>(c->e.p);
  t.sid = static_cast<const uint32_t*>(c->sid.p);
  t.nodes = static_cast<const float2*>(c->nodes.p);
  // Rank tables of the leaves (d <= 3): 544 bytes per leaf and dimension.
  // Optional: without room for them the swapped leaf test compares instead.
  t.tab = nullptr;
  if (d <= 3 && c->tables_on &&
      ensure(c, c->tab, sizeof(uint32_t) * 2u * kRankSlot * (size_t)d * t.cnt[1]) == DDM_OK)
    t.tab = static_cast<const uint32_t*>(c->tab.p);
  DDM_CUDA(launch_build(t, static_cast<const uint32_t*>(c->vals[cur].p), slo, shi, aos,
                        static_cast<float2*>(c->e.p), static_cast<uint32_t*>(c->sid.p),
                        static_cast<float2*>(c->nodes.p), const_cast<uint32_t*>(t.tab),
                        c->st_dev, s));
  c->tree = t;
  c->built = true;
  return DDM_OK;
}

// Grid size argument of the packet kernels (they launch 8 CTAs per "SM").
int packet_sms(const ddm_ctx* c) {
  const int v = (int)((uint64_t)c->sms * c->ctas_per_sm / 8u);
  return v > 0 ? v : 1;
}

// Packets of the count pass (and of its records) covering positions [0, m).
uint32_t packets_of(const ddm_ctx* c, uint32_t m) {
  return (uint32_t)(((uint64_t)m + (1u << c->qpp_log2) - 1u) >> c->qpp_log2);
}

QueryView query_view(ddm_ctx* c) {
  QueryView q{};
  q.m = c->m;
  q.qe = static_cast<const float2*>(c->qe.p);
  q.qid = static_cast<const uint32_t*>(c->qid.p);
  q.list = nullptr;
  q.first = 0;
  q.nq = c->m;
  q.qpp_log2 = c->qpp_log2;
  q.tmin = c->tmin;
  return q;
}

// Validate U, sort it, count per update, scan (no host synchronisation).
int plan_async(ddm_ctx* c, const float* ulo, const float* uhi, uint32_t m, uint32_t flags,
               bool record, cudaStream_t s, const BatchSet* bs = nullptr) {
  Phase phase("ddm plan");
  c->planned = false;
  const int d = c->tree.d;
  DDM_TRY(ensure(c, c->counts, sizeof(uint32_t) * (m ? m : 1)));
  DDM_TRY(ensure(c, c->counts_pos, sizeof(uint32_t) * (m ? m : 1)));
  DDM_TRY(ensure(c, c->offsets, sizeof(unsigned long long) * ((size_t)m + 1)));
  DDM_TRY(ensure(c, c->pos_offsets, sizeof(unsigned long long) * ((size_t)m + 1)));
  // tile sums of the three scans below, one region each
  const size_t upd_tiles = (size_t)m / kScanTile + 1;
  const size_t blk_tiles = (size_t)packets_of(c, m) * kRecChains / kScanTile + 1;
  DDM_TRY(ensure(c, c->sums, sizeof(unsigned long long) * (2 * upd_tiles + blk_tiles + 1)));
  DDM_TRY(ensure(c, c->work, sizeof(uint32_t)));
  DDM_TRY(ensure(c, c->qe, sizeof(float2) * (size_t)d * (m ? m : 1)));
  DDM_TRY(ensure(c, c->qid, sizeof(uint32_t) * (m ? m : 1)));
  auto* counts = static_cast<uint32_t*>(c->counts.p);
  auto* counts_pos = static_cast<uint32_t*>(c->counts_pos.p);
  auto* offsets = static_cast<unsigned long long*>(c->offsets.p);
  auto* pos_offsets = static_cast<unsigned long long*>(c->pos_offsets.p);
  c->m = m;
  c->arena = RecordArena{};
  if (record && c->replay_on && m > 0 && c->tree.n > 0 && c->replay_budget > 0) {
    const uint32_t packets = packets_of(c, m);
    // bytes per block: records (ten bytes each) and header, next/count/packet/list entries
    const uint64_t per_block = (uint64_t)kRecWords * sizeof(uint32_t) + 4 * sizeof(uint32_t);
    // Blocks the arena holds now, and what the latest recorded pass needed.
    uint64_t have = c->rec.cap / ((size_t)kRecWords * sizeof(uint32_t));
    for (const DevBuf* b : {&c->blk_next, &c->blk_count, &c->blk_pkt, &c->blk_list})
      have = std::min<uint64_t>(have, b->cap / sizeof(uint32_t));
    const uint32_t hint_blocks = c->rec_hint[0], hint_packets = c->rec_hint[1],
                   hint_max = c->rec_hint[2];
    uint64_t want = have;
    if (have == 0 || (hint_packets && hint_blocks > hint_max)) {
      // No arena yet, or the last pass ran out of it: size from that pass's
      // blocks per packet (plus 1/8 and some slack), else 2 per packet.  An
      // arena that sufficed is kept as it is: the blocks per packet depend on
      // how densely the updates cover the space, so extrapolating them from
      // one plan to the next would reallocate for nothing.
      const uint64_t need =
          hint_packets ? (uint64_t)((double)hint_blocks / (double)hint_packets * 1.125 *
                                    (double)packets) + 64
                       : 2ull * packets;
      want = std::max(have, need);
    }
    const uint64_t cap_blocks = c->replay_budget / per_block;
    if (want > cap_blocks) want = cap_blocks;
    if (want > 0xfffffff0ull) want = 0xfffffff0ull;
    if (want > 0 && ensure(c, c->rec, (size_t)want * kRecWords * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->blk_next, (size_t)want * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->blk_count, (size_t)want * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->blk_pkt, (size_t)want * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->blk_list, (size_t)want * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->pkt_first, (size_t)packets * kRecChains * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->pkt_nblk, (size_t)packets * kRecChains * sizeof(uint32_t)) == DDM_OK &&
        ensure(c, c->pkt_off, ((size_t)packets * kRecChains + 1) * sizeof(unsigned long long)) ==
            DDM_OK &&
        ensure(c, c->blk_counter, 4 * sizeof(uint32_t)) == DDM_OK) {
      c->arena.rec = static_cast<uint32_t*>(c->rec.p);
      c->arena.blk_next = static_cast<uint32_t*>(c->blk_next.p);
      c->arena.blk_count = static_cast<uint32_t*>(c->blk_count.p);
      c->arena.pkt_first = static_cast<uint32_t*>(c->pkt_first.p);
      c->arena.blk_pkt = static_cast<uint32_t*>(c->blk_pkt.p);
      c->arena.blk_list = static_cast<uint32_t*>(c->blk_list.p);
      c->arena.pkt_nblk = static_cast<uint32_t*>(c->pkt_nblk.p);
      c->arena.pkt_off = static_cast<unsigned long long*>(c->pkt_off.p);
      c->arena.blk_counter = static_cast<uint32_t*>(c->blk_counter.p);
      c->arena.max_blocks = (uint32_t)want;
      DDM_CUDA(cudaMemsetAsync(c->blk_counter.p, 0, 4 * sizeof(uint32_t), s));
    }
  }
  if (m > 0) {
    int cur = 0;
    float2* aos = aos_buffer(c, d, m);
    if (bs)
      DDM_TRY(order_set_batch(c, d, ulo, uhi, m, *bs, aos, &cur, s));
    else
      DDM_TRY(order_set(c, d, ulo, uhi, m, false, aos, &cur, s));
    DDM_CUDA(launch_gather(d, static_cast<const uint32_t*>(c->vals[cur].p), ulo, uhi, aos, m,
                           static_cast<float2*>(c->qe.p), static_cast<uint32_t*>(c->qid.p), c->sms,
                           s));
    if (c->tree.n > 0) {
      DDM_CUDA(launch_count(c->tree, query_view(c), c->bv, flags, counts, counts_pos, c->arena,
                            static_cast<uint32_t*>(c->work.p), c->st_dev, packet_sms(c), s));
    } else {
      DDM_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * m, s));
      DDM_CUDA(cudaMemsetAsync(counts_pos, 0, sizeof(uint32_t) * m, s));
    }
  }
  // offsets by plan position and by update id, and the record blocks' plan
  // order, in one launch sequence
  auto* sums = static_cast<unsigned long long*>(c->sums.p);
  ScanJob jobs[kMaxScanJobs] = {{counts_pos, m, pos_offsets, sums, nullptr},
                                {counts, m, offsets, sums + upd_tiles, c->st_dev}};
  int njobs = 2;
  if (c->arena.max_blocks)
    jobs[njobs++] = ScanJob{c->arena.pkt_nblk, packets_of(c, m) * kRecChains, c->arena.pkt_off,
                            sums + 2 * upd_tiles, nullptr};
  DDM_CUDA(launch_scan_multi(jobs, njobs, s));
  if (c->arena.max_blocks) DDM_CUDA(launch_block_list(c->arena, packets_of(c, m), s));
  if (c->arena.max_blocks)  // blocks needed, packets, blocks held: the next arena's sizing hint
    DDM_CUDA(cudaMemcpyAsync((void*)c->rec_hint, static_cast<uint32_t*>(c->blk_counter.p) + 1,
                             3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  c->ulo = ulo;
  c->uhi = uhi;
  c->flags = flags;
  c->planned = true;
  return DDM_OK;
}

// Write pass for updates with ids in [begin, end), laid out by update id.
// Global update ids (update-id base + local id) must fit 32 bits.
bool base_fits(const ddm_ctx* c) { return (uint64_t)c->upd_base + c->m <= (1ull << 32); }

int write_async(ddm_ctx* c, uint32_t begin, uint32_t end, ddm_pair* pairs, uint64_t capacity,
                cudaStream_t s, const uint32_t* qids = nullptr) {
  Phase phase("ddm write");
  if (!qids && !c->swapped && !c->bv.count && !base_fits(c)) return DDM_ERR_ARG;
  if (end > begin && c->tree.n > 0) {
    QueryView q = query_view(c);
    if (begin != 0 || end != c->m) {
      DDM_TRY(ensure(c, c->sel_offs, sizeof(unsigned long long) * ((size_t)c->m + 1)));
      DDM_TRY(ensure(c, c->sel_list, sizeof(uint32_t) * c->m));
      DDM_CUDA(launch_select(q.qid, c->m, begin, end, static_cast<uint32_t*>(c->counts.p),
                             static_cast<unsigned long long*>(c->sel_offs.p),
                             static_cast<unsigned long long*>(c->sums.p),
                             static_cast<uint32_t*>(c->sel_list.p), c->st_dev, s));
      q.list = static_cast<const uint32_t*>(c->sel_list.p);
      q.nq = end - begin;
    }
    WriteView w{};
    w.start = static_cast<const unsigned long long*>(c->offsets.p);
    w.by_pos = false;
    w.swap = c->swapped;
    w.qids = qids;
    w.qbase = (c->swapped || c->bv.count) ? 0u : c->upd_base;
    w.b_idx = begin;
    w.e_idx = end;
    w.pairs = pairs;
    w.capacity = capacity;
    auto* work = static_cast<uint32_t*>(c->work.p);
    if (c->arena.max_blocks) {
      const bool full = begin == 0 && end == c->m;
      DDM_CUDA(launch_replay(c->tree, query_view(c), c->bv, c->arena, w, 0, packets_of(c, c->m), 0, c->m,
                             !full, begin, end, work, c->st_dev, c->sms, s));
    }
    DDM_CUDA(launch_write(c->tree, q, c->bv, c->flags, w, c->arena, work, c->st_dev, packet_sms(c), s));
  } else {
    DDM_CUDA(cudaMemsetAsync(&c->st_dev->K, 0, sizeof(unsigned long long), s));
  }
  return DDM_OK;
}

// Write pass for the plan positions [pb, pe), laid out in plan order.
int write_ordered_async(ddm_ctx* c, uint32_t pb, uint32_t pe, ddm_pair* pairs, uint64_t capacity,
                        cudaStream_t s, uint32_t* ids = nullptr) {
  Phase phase("ddm write ordered");
  if (!ids && !base_fits(c)) return DDM_ERR_ARG;
  if (pe > pb && c->tree.n > 0) {
    QueryView q = query_view(c);
    q.first = pb;
    q.nq = pe - pb;
    WriteView w{};
    w.start = static_cast<const unsigned long long*>(c->pos_offsets.p);
    w.by_pos = true;
    w.qbase = c->upd_base;
    w.b_idx = pb;
    w.e_idx = pe;
    w.pairs = pairs;
    w.ids = ids;
    w.capacity = capacity;
    auto* work = static_cast<uint32_t*>(c->work.p);
    if (c->arena.max_blocks)
      DDM_CUDA(launch_replay(c->tree, q, c->bv, c->arena, w, pb >> c->qpp_log2, packets_of(c, pe), pb, pe, false, 0, 0,
                             work, c->st_dev, c->sms, s));
    DDM_CUDA(launch_write(c->tree, q, c->bv, c->flags, w, c->arena, work, c->st_dev, packet_sms(c), s));
  } else {
    DDM_CUDA(cudaMemsetAsync(&c->st_dev->K, 0, sizeof(unsigned long long), s));
  }
  return DDM_OK;
}

int reset_status(ddm_ctx* c, cudaStream_t s) {
  DDM_CUDA(cudaMemsetAsync(c->st_dev, 0, sizeof(Status), s));
  return DDM_OK;
}

}  // namespace

extern "C" {

const char* ddm_strerror(int code) {
  switch (code) {
    case DDM_OK: return "success";
    case DDM_ERR_ARG: return "invalid argument";
    case DDM_ERR_EXTENT: return "invalid extent (lo > hi or NaN)";
    case DDM_ERR_CAPACITY: return "pair buffer too small";
    case DDM_ERR_NOMEM: return "device memory allocation failed";
    case DDM_ERR_CUDA: return "CUDA error";
    case DDM_ERR_TIMEOUT: return "bounded device wait timed out";
    case DDM_ERR_STATE: return "tree or plan missing";
    case DDM_ERR_INTERNAL: return "an index failed its bounds check (checked build)";
    default: return "unknown error";
  }
}

int ddm_create(ddm_ctx** out, int device) {
  if (!out) return DDM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DDM_ERR_CUDA;
  }
  DeviceGuard g(device);
  if (!g.ok()) return DDM_ERR_CUDA;
  ddm_ctx* c = new (std::nothrow) ddm_ctx();
  if (!c) return DDM_ERR_NOMEM;
  c->device = device;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) c->replay_budget = total_b / 4;
    cudaGetLastError();
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  const uint64_t keep_all = ~0ull;
  if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, (void*)&keep_all) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&c->st_dev, sizeof(Status)) != cudaSuccess ||
      cudaMallocHost(&c->st_host, sizeof(Status)) != cudaSuccess ||
      cudaMallocHost((void**)&c->rec_hint, 3 * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    ddm_destroy(c);
    return DDM_ERR_NOMEM;
  }
  c->rec_hint[0] = c->rec_hint[1] = c->rec_hint[2] = 0;
  *out = c;
  return DDM_OK;
}

int ddm_destroy(ddm_ctx* c) {
  if (!c) return DDM_OK;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  for (DevBuf* b : {&c->keys[0], &c->keys[1], &c->vals[0], &c->vals[1], &c->hist, &c->lookback,
                    &c->counters, &c->e, &c->sid, &c->nodes, &c->tab, &c->qe, &c->qid, &c->counts,
                    &c->counts_pos, &c->offsets, &c->pos_offsets, &c->sums, &c->work,
                    &c->sel_offs, &c->sel_list, &c->rec, &c->blk_next, &c->blk_count,
                    &c->blk_pkt, &c->pkt_first, &c->pkt_nblk, &c->pkt_off,
                    &c->blk_list, &c->blk_counter, &c->inst_s, &c->inst_u, &c->bglog2,
                    &c->bngroups, &c->bgbase, &c->cls_hist, &c->cls_off, &c->probe, &c->aos})
    release(*b);
  cudaDeviceSynchronize();  // the stream-ordered frees above have run
  if (c->pool) cudaMemPoolDestroy(c->pool);
  if (c->done) cudaEventDestroy(c->done);
  if (c->st_dev) cudaFree(c->st_dev);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->rec_hint) cudaFreeHost((void*)c->rec_hint);
  delete c;
  return DDM_OK;
}

int ddm_set_replay_budget(ddm_ctx* c, uint64_t bytes) {
  if (!c) return DDM_ERR_ARG;
  c->replay_budget = bytes;
  return DDM_OK;
}

int ddm_set_tuning(ddm_ctx* c, int str_shift, uint32_t ctas_per_sm, uint32_t replay) {
  if (!c || str_shift < -4 || str_shift > 4 || ctas_per_sm < 1 || ctas_per_sm > 32)
    return DDM_ERR_ARG;
  c->str_shift = str_shift;
  c->ctas_per_sm = ctas_per_sm;
  c->replay_on = replay != 0;
  return DDM_OK;
}

int ddm_set_tiling(ddm_ctx* c, uint32_t queries_per_packet, uint32_t swap_min) {
  if (!c || (queries_per_packet != 16 && queries_per_packet != 32) || swap_min < 1 ||
      swap_min > 33)
    return DDM_ERR_ARG;
  const uint32_t lg = queries_per_packet == 16 ? 4u : 5u;
  if (lg != c->qpp_log2) c->planned = false;  // the plan's records use its packets
  c->qpp_log2 = lg;
  c->tmin = swap_min;
  return DDM_OK;
}

int ddm_set_update_id_base(ddm_ctx* c, uint32_t base) {
  if (!c) return DDM_ERR_ARG;
  c->upd_base = base;
  return DDM_OK;
}

int ddm_debug_wait_timeout(ddm_ctx* c, uint32_t polls, void* stream) {
  if (!c || polls == 0 || polls > (1u << 22)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(ensure(c, c->probe, sizeof(uint32_t)));
  DDM_CUDA(cudaMemsetAsync(c->probe.p, 0, sizeof(uint32_t), s));
  DDM_TRY(reset_status(c, s));
  DDM_CUDA(launch_debug_wait(static_cast<const uint32_t*>(c->probe.p), polls, c->st_dev, s));
  DDM_TRY(sync_status(c, s));
  return status_code(*c->st_host);
}

uint64_t ddm_debug_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int ddm_debug_set_alloc_limit(ddm_ctx* c, uint64_t bytes) {
  if (!c) return DDM_ERR_ARG;
  c->alloc_limit = bytes;
  return DDM_OK;
}

int ddm_build(ddm_ctx* c, int d, const float* slo, const float* shi, uint32_t n, void* stream) {
  if (!c || d < 1 || d > DDM_MAX_DIMS || !set_ok(d, slo, shi, n)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(build_async(c, d, slo, shi, n, s));
  DDM_TRY(sync_status(c, s));
  const int rc = status_code(*c->st_host);
  if (rc != DDM_OK) c->built = false;
  return rc;
}

int ddm_plan(ddm_ctx* c, const float* ulo, const float* uhi, uint32_t m, uint32_t flags,
             uint64_t* offsets, uint64_t* k_out, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built) return DDM_ERR_STATE;
  if (!set_ok(c->tree.d, ulo, uhi, m) || (flags & ~DDM_OPEN)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(plan_async(c, ulo, uhi, m, flags, true, s));
  if (offsets)
    DDM_CUDA(cudaMemcpyAsync(offsets, c->offsets.p, sizeof(unsigned long long) * ((size_t)m + 1),
                             cudaMemcpyDeviceToDevice, s));
  DDM_TRY(sync_status(c, s));
  c->last_tests = c->st_host->tests;
  if (k_out) *k_out = c->st_host->K;
  const int rc = status_code(*c->st_host);
  if (rc != DDM_OK) c->planned = false;
  return rc;
}

int ddm_write(ddm_ctx* c, uint32_t begin, uint32_t end, ddm_pair* pairs, uint64_t capacity,
              uint64_t* k_out, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (begin > end || end > c->m || (end > begin && !pairs)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(write_async(c, begin, end, pairs, capacity, s));
  DDM_TRY(sync_status(c, s));
  if (k_out) *k_out = c->st_host->K;
  return status_code(*c->st_host);
}

int ddm_chunk_end(ddm_ctx* c, uint32_t begin, uint64_t capacity, uint32_t* upd_end, void* stream) {
  if (!c || !upd_end) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (begin > c->m) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_CUDA(launch_chunk_end(static_cast<const unsigned long long*>(c->offsets.p), c->m, begin,
                            capacity, c->st_dev, s));
  DDM_TRY(sync_status(c, s));
  *upd_end = (uint32_t)c->st_host->aux;
  if (*upd_end == begin && begin < c->m) return DDM_ERR_CAPACITY;
  return DDM_OK;
}

int ddm_plan_async(ddm_ctx* c, const float* ulo, const float* uhi, uint32_t m, uint32_t flags,
                   void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built || c->bv.count) return DDM_ERR_STATE;
  if (!set_ok(c->tree.d, ulo, uhi, m) || (flags & ~DDM_OPEN)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(plan_async(c, ulo, uhi, m, flags, true, s));
  return DDM_OK;
}

int ddm_write_async(ddm_ctx* c, uint32_t begin, uint32_t end, ddm_pair* pairs, uint64_t capacity,
                    uint64_t* k_dev, uint32_t* err_dev, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (begin > end || end > c->m || (end > begin && !pairs && capacity > 0)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  // keep the plan's error bits; the write sets K (and the capacity bit)
  DDM_TRY(write_async(c, begin, end, pairs, capacity, s));
  if (k_dev)
    DDM_CUDA(cudaMemcpyAsync(k_dev, &c->st_dev->K, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (err_dev)
    DDM_CUDA(cudaMemcpyAsync(err_dev, &c->st_dev->err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  return DDM_OK;
}

int ddm_plan_stats(ddm_ctx* c, uint64_t* leaf_tests) {
  if (!c || !leaf_tests) return DDM_ERR_ARG;
  *leaf_tests = c->last_tests;
  return DDM_OK;
}

int ddm_match_moved(ddm_ctx* c, const float* lo, const float* hi, uint32_t k, const uint32_t* ids,
                    uint32_t flags, ddm_pair* pairs, uint64_t capacity, uint64_t* k_out,
                    void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built || c->bv.count) return DDM_ERR_STATE;
  if (!set_ok(c->tree.d, lo, hi, k) || (flags & ~(DDM_OPEN | DDM_SWAP_ROLES)) ||
      (k > 0 && !pairs && capacity > 0))
    return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(plan_async(c, lo, hi, k, flags & DDM_OPEN, true, s));
  const bool was = c->swapped;
  c->swapped = (flags & DDM_SWAP_ROLES) != 0;
  const int wrc = write_async(c, 0, k, pairs, capacity, s, ids);
  c->swapped = was;
  DDM_TRY(wrc);
  DDM_TRY(sync_status(c, s));
  c->last_tests = c->st_host->tests;
  if (k_out) *k_out = c->st_host->K;
  const int rc = status_code(*c->st_host);
  if (rc != DDM_OK) c->planned = false;
  return rc;
}

int ddm_pair_offsets_async(ddm_ctx* c, const uint64_t* upd_off, uint32_t count, uint64_t* pair_off,
                           void* stream) {
  if (!c || !upd_off || !pair_off) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  StreamUse use(c, static_cast<cudaStream_t>(stream));
  DDM_CUDA(launch_gather_offsets(static_cast<const unsigned long long*>(c->offsets.p), c->m,
                                 reinterpret_cast<const unsigned long long*>(upd_off), count,
                                 reinterpret_cast<unsigned long long*>(pair_off),
                                 static_cast<cudaStream_t>(stream)));
  return DDM_OK;
}

int ddm_write_ordered(ddm_ctx* c, uint32_t pos_begin, uint32_t pos_end, ddm_pair* pairs,
                      uint64_t capacity, uint64_t* k_out, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (pos_begin > pos_end || pos_end > c->m || (pos_end > pos_begin && !pairs)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(write_ordered_async(c, pos_begin, pos_end, pairs, capacity, s));
  DDM_TRY(sync_status(c, s));
  if (k_out) *k_out = c->st_host->K;
  return status_code(*c->st_host);
}

int ddm_write_ordered_ids(ddm_ctx* c, uint32_t pos_begin, uint32_t pos_end, uint32_t* sub_ids,
                          uint64_t capacity, uint64_t* k_out, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (pos_begin > pos_end || pos_end > c->m || (pos_end > pos_begin && !sub_ids)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(write_ordered_async(c, pos_begin, pos_end, nullptr, capacity, s, sub_ids));
  DDM_TRY(sync_status(c, s));
  if (k_out) *k_out = c->st_host->K;
  return status_code(*c->st_host);
}

int ddm_chunk_end_ordered(ddm_ctx* c, uint32_t pos_begin, uint64_t capacity, uint32_t* pos_end,
                          void* stream) {
  if (!c || !pos_end) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  if (pos_begin > c->m) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_CUDA(launch_chunk_end(static_cast<const unsigned long long*>(c->pos_offsets.p), c->m,
                            pos_begin, capacity, c->st_dev, s));
  DDM_TRY(sync_status(c, s));
  *pos_end = (uint32_t)c->st_host->aux;
  if (*pos_end == pos_begin && pos_begin < c->m) return DDM_ERR_CAPACITY;
  return DDM_OK;
}

int ddm_plan_order(ddm_ctx* c, uint32_t* order, uint64_t* order_offsets, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->planned) return DDM_ERR_STATE;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  if (order && c->m)
    DDM_CUDA(cudaMemcpyAsync(order, c->qid.p, sizeof(uint32_t) * c->m, cudaMemcpyDeviceToDevice, s));
  if (order_offsets)
    DDM_CUDA(cudaMemcpyAsync(order_offsets, c->pos_offsets.p,
                             sizeof(unsigned long long) * ((size_t)c->m + 1),
                             cudaMemcpyDeviceToDevice, s));
  return DDM_OK;
}

static int match_impl(ddm_ctx* c, int d, const float* ulo, const float* uhi, uint32_t m,
                      const float* slo, const float* shi, uint32_t n, uint32_t begin, uint32_t end,
                      uint32_t flags, ddm_pair* pairs, uint64_t capacity, uint64_t* k_out,
                      void* stream, bool write) {
  if (!c || d < 1 || d > DDM_MAX_DIMS || !set_ok(d, ulo, uhi, m) || !set_ok(d, slo, shi, n) ||
      (flags & ~(DDM_OPEN | DDM_SWAP_ROLES)) || begin > end || end > m)
    return DDM_ERR_ARG;
  const bool swap = (flags & DDM_SWAP_ROLES) != 0;
  if (swap && (begin != 0 || end != m)) return DDM_ERR_ARG;
  if (write && end > begin && !pairs && capacity > 0) return DDM_ERR_ARG;
  if (swap) {  // tree over the updates, one query per subscription
    std::swap(ulo, slo);
    std::swap(uhi, shi);
    std::swap(m, n);
    begin = 0;
    end = m;
  }
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  DDM_TRY(build_async(c, d, slo, shi, n, s));
  c->swapped = swap;
  DDM_TRY(plan_async(c, ulo, uhi, m, flags & DDM_OPEN, write, s));
  if (write) DDM_TRY(write_async(c, begin, end, pairs, capacity, s));
  DDM_TRY(sync_status(c, s));
  c->last_tests = c->st_host->tests;
  if (k_out) *k_out = c->st_host->K;
  const int rc = status_code(*c->st_host);
  // a swapped problem's tree and plan are not the caller's sets: no staged use
  if (swap || rc == DDM_ERR_EXTENT || rc == DDM_ERR_TIMEOUT) c->built = c->planned = false;
  return rc;
}

int ddm_count(ddm_ctx* c, int d, const float* ulo, const float* uhi, uint32_t m, const float* slo,
              const float* shi, uint32_t n, uint32_t flags, uint64_t* k_out, void* stream) {
  return match_impl(c, d, ulo, uhi, m, slo, shi, n, 0, m, flags, nullptr, 0, k_out, stream, false);
}

int ddm_match(ddm_ctx* c, int d, const float* ulo, const float* uhi, uint32_t m, const float* slo,
              const float* shi, uint32_t n, uint32_t flags, ddm_pair* pairs, uint64_t capacity,
              uint64_t* k_out, void* stream) {
  return match_impl(c, d, ulo, uhi, m, slo, shi, n, 0, m, flags, pairs, capacity, k_out, stream,
                    true);
}

int ddm_match_range(ddm_ctx* c, int d, const float* ulo, const float* uhi, uint32_t m,
                    const float* slo, const float* shi, uint32_t n, uint32_t begin, uint32_t end,
                    uint32_t flags, ddm_pair* pairs, uint64_t capacity, uint64_t* k_out,
                    void* stream) {
  return match_impl(c, d, ulo, uhi, m, slo, shi, n, begin, end, flags, pairs, capacity, k_out,
                    stream, true);
}

static int batch_impl(ddm_ctx* c, int d, uint32_t count, const float* ulo, const float* uhi,
                      const uint64_t* upd_off, uint32_t m, const float* slo, const float* shi,
                      const uint64_t* sub_off, uint32_t n, uint32_t flags, ddm_pair* pairs,
                      uint64_t capacity, uint64_t* pair_off, uint64_t* k_out, uint64_t* k_dev,
                      uint32_t* err_dev, void* stream, bool sync) {
  if (!c || d < 1 || d > DDM_MAX_DIMS || count == 0 || !upd_off || !sub_off || !set_ok(d, ulo, uhi, m) ||
      !set_ok(d, slo, shi, n) || (flags & ~DDM_OPEN) || (!pairs && capacity > 0))
    return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(ensure(c, c->inst_s, sizeof(uint32_t) * (n ? n : 1)));
  DDM_TRY(ensure(c, c->inst_u, sizeof(uint32_t) * (m ? m : 1)));
  DDM_TRY(reset_status(c, s));
  const auto* uoff = reinterpret_cast<const unsigned long long*>(upd_off);
  const auto* soff = reinterpret_cast<const unsigned long long*>(sub_off);
  BatchSet bs_s{soff, count, static_cast<uint32_t*>(c->inst_s.p)};
  BatchSet bs_u{uoff, count, static_cast<uint32_t*>(c->inst_u.p)};
  DDM_TRY(build_async(c, d, slo, shi, n, s, &bs_s));
  c->bv.count = count;
  c->bv.upd_off = uoff;
  c->bv.sub_off = soff;
  c->bv.q_inst = static_cast<const uint32_t*>(c->inst_u.p);
  DDM_TRY(plan_async(c, ulo, uhi, m, flags, true, s, &bs_u));
  DDM_TRY(write_async(c, 0, m, pairs, capacity, s));
  if (pair_off && m > 0)
    DDM_CUDA(launch_gather_offsets(static_cast<const unsigned long long*>(c->offsets.p), m, uoff,
                                   count, reinterpret_cast<unsigned long long*>(pair_off), s));
  else if (pair_off)
    DDM_CUDA(cudaMemsetAsync(pair_off, 0, sizeof(uint64_t) * ((size_t)count + 1), s));
  if (k_dev)
    DDM_CUDA(cudaMemcpyAsync(k_dev, &c->st_dev->K, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (err_dev)
    DDM_CUDA(cudaMemcpyAsync(err_dev, &c->st_dev->err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  // The tree and plan hold a batch: the single-problem staged calls must not use them.
  c->built = c->planned = false;
  if (!sync) return DDM_OK;
  DDM_TRY(sync_status(c, s));
  c->last_tests = c->st_host->tests;
  if (k_out) *k_out = c->st_host->K;
  return status_code(*c->st_host);
}

int ddm_batch_match(ddm_ctx* c, int d, uint32_t count, const float* upd_lo, const float* upd_hi,
                    const uint64_t* upd_off, uint32_t m_total, const float* sub_lo,
                    const float* sub_hi, const uint64_t* sub_off, uint32_t n_total, uint32_t flags,
                    ddm_pair* pairs, uint64_t capacity, uint64_t* pair_off, uint64_t* k_out,
                    void* stream) {
  return batch_impl(c, d, count, upd_lo, upd_hi, upd_off, m_total, sub_lo, sub_hi, sub_off,
                    n_total, flags, pairs, capacity, pair_off, k_out, nullptr, nullptr, stream, true);
}

int ddm_batch_match_async(ddm_ctx* c, int d, uint32_t count, const float* upd_lo,
                          const float* upd_hi, const uint64_t* upd_off, uint32_t m_total,
                          const float* sub_lo, const float* sub_hi, const uint64_t* sub_off,
                          uint32_t n_total, uint32_t flags, ddm_pair* pairs, uint64_t capacity,
                          uint64_t* pair_off, uint64_t* k_dev, uint32_t* err_dev, void* stream) {
  return batch_impl(c, d, count, upd_lo, upd_hi, upd_off, m_total, sub_lo, sub_hi, sub_off,
                    n_total, flags, pairs, capacity, pair_off, nullptr, k_dev, err_dev, stream,
                    false);
}

int ddm_refit(ddm_ctx* c, const float* sub_lo, const float* sub_hi, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built || c->attached || c->bv.count) return DDM_ERR_STATE;
  if (c->tree.n > 0 && (!sub_lo || !sub_hi)) return DDM_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  DDM_TRY(reset_status(c, s));
  c->planned = false;
  Phase phase("ddm refit");
  if (c->tree.n > 0) {
    float2* aos = aos_buffer(c, c->tree.d, c->tree.n);
    DDM_CUDA(launch_validate(c->tree.d, sub_lo, sub_hi, c->tree.n, nullptr, nullptr, 0, aos,
                             c->st_dev, c->sms, s));
    // Same order, new coordinates: gather through the tree's own id column and
    // recompute every node's per-dimension (minlower, maxupper).
    DDM_CUDA(launch_build(c->tree, c->tree.sid, sub_lo, sub_hi, aos, static_cast<float2*>(c->e.p),
                          static_cast<uint32_t*>(c->sid.p), static_cast<float2*>(c->nodes.p),
                          const_cast<uint32_t*>(c->tree.tab), c->st_dev, s));
  }
  DDM_TRY(sync_status(c, s));
  const int rc = status_code(*c->st_host);
  if (rc != DDM_OK) c->built = false;
  return rc;
}

int ddm_attach(ddm_ctx* c, const ddm_ctx* src) {
  if (!c || !src || c == src) return DDM_ERR_ARG;
  if (!src->built || src->bv.count) return DDM_ERR_STATE;
  if (c->device != src->device) return DDM_ERR_ARG;
  c->tree = src->tree;
  c->bv = BatchView{};
  c->built = true;
  c->attached = true;
  c->planned = false;
  return DDM_OK;
}

int ddm_tree_shape(ddm_ctx* c, int* levels, uint32_t* counts, uint32_t* total) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built) return DDM_ERR_STATE;
  const TreeView& t = c->tree;
  const int L = t.n ? t.L : 0;
  if (levels) *levels = L;
  uint32_t tot = 0;
  for (int l = 1; l <= L; ++l) {
    if (counts) counts[l - 1] = t.cnt[l];
    tot += t.cnt[l];
  }
  if (total) *total = tot;
  return DDM_OK;
}

int ddm_tree_export(ddm_ctx* c, uint32_t* order, float* node_lo, float* node_hi, void* stream) {
  if (!c) return DDM_ERR_ARG;
  if (!c->built) return DDM_ERR_STATE;
  if (c->tree.n == 0) return DDM_OK;
  DeviceGuard g(c->device);
  if (!g.ok()) return DDM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamUse use(c, s);
  if (order)
    DDM_CUDA(cudaMemcpyAsync(order, c->sid.p, sizeof(uint32_t) * c->tree.n,
                             cudaMemcpyDeviceToDevice, s));
  DDM_CUDA(launch_export_nodes(c->tree, node_lo, node_hi, s));
  return DDM_OK;
}

}  // extern "C"
