// Exclusive scan of the per-update match counts into 64-bit offsets.
//
// The intersection matrix M of Section III is sparse and is returned in
// compressed form: update j's matches occupy [offsets[j], offsets[j+1]) of
// the pair list, and offsets[m] = K (which can exceed 2^32).  Classic
// reduce-then-scan over tiles of 4096 counts: per-tile sums, one CTA scans
// the tile sums, then each tile scans its counts from its tile offset.  No
// kernel waits on another CTA.
#include <atomic>

#include "ddm_internal.cuh"

namespace ddm {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = kScanTile / kThreads;  // 16

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block-wide scan of one value per thread; returns the thread's
// exclusive prefix and the block total in *total.
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long wsum[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned long long incl = warp_incl_scan(v, lane);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  unsigned long long pre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kThreads / 32; ++i) {
    if (i < w) pre += wsum[i];
    tot += wsum[i];
  }
  __syncthreads();
  *total = tot;
  return pre + incl - v;
}

// Sum of tile `tile` of counts into sums[tile].
__device__ __forceinline__ void tile_sum(const uint32_t* __restrict__ counts, uint32_t m,
                                         uint32_t tile, unsigned long long* __restrict__ sums) {
  const size_t base = (size_t)tile * kScanTile;
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const size_t idx = base + (size_t)i * kThreads + threadIdx.x;  // coalesced
    if (idx < m) s += counts[idx];
  }
  unsigned long long tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[tile] = tot;
}

// One CTA: exclusive scan of the tile sums in place; total -> offsets[m], st->K.
__device__ __forceinline__ void scan_sums(unsigned long long* __restrict__ sums, uint32_t tiles,
                                          unsigned long long* __restrict__ offsets, uint32_t m,
                                          Status* __restrict__ st) {
  unsigned long long carry = 0;
  for (uint32_t c = 0; c < tiles; c += kThreads) {
    const uint32_t idx = c + threadIdx.x;
    const unsigned long long v = idx < tiles ? sums[idx] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan(v, &tot);
    if (idx < tiles) sums[idx] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    offsets[m] = carry;
    if (st) st->K = carry;
  }
}

// Offsets of tile `tile` from its scanned tile sum.  ONE: a single tile
// (m <= kScanTile) with no tile sums, which also writes the total to
// offsets[m] and st->K.
template <bool ONE>
__device__ __forceinline__ void scan_tile(const uint32_t* __restrict__ counts, uint32_t m,
                                          uint32_t tile,
                                          const unsigned long long* __restrict__ sums,
                                          unsigned long long* __restrict__ offsets,
                                          Status* __restrict__ st) {
  __shared__ uint32_t s_c[kScanTile];
  const size_t base = (size_t)tile * kScanTile;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const size_t idx = base + (size_t)i * kThreads + threadIdx.x;
    s_c[i * kThreads + threadIdx.x] = idx < m ? counts[idx] : 0u;
  }
  __syncthreads();
  // thread t scans items [t*16, t*16+16) of the tile
  unsigned long long local = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) local += s_c[threadIdx.x * kItems + i];
  unsigned long long tot;
  unsigned long long run = (ONE ? 0ull : sums[tile]) + block_excl_scan(local, &tot);
  if (ONE && threadIdx.x == 0) {
    offsets[m] = tot;
    if (st) st->K = tot;
  }
  unsigned long long out[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    out[i] = run;
    run += s_c[threadIdx.x * kItems + i];
  }
  // write back: reuse shared memory as 64-bit staging in two halves
  __syncthreads();
  unsigned long long* s_o = reinterpret_cast<unsigned long long*>(s_c);  // 2048 entries
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int lo_t = half * (kThreads / 2);
    if ((int)threadIdx.x >= lo_t && (int)threadIdx.x < lo_t + kThreads / 2) {
#pragma unroll
      for (int i = 0; i < kItems; ++i) s_o[(threadIdx.x - lo_t) * kItems + i] = out[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kScanTile / 2; q += kThreads) {
      const size_t idx = base + (size_t)half * (kScanTile / 2) + q;
      if (idx < m) offsets[idx] = s_o[q];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads)
k_tile_sums(const uint32_t* __restrict__ counts, uint32_t m, unsigned long long* __restrict__ sums) {
  tile_sum(counts, m, blockIdx.x, sums);
}

__global__ void __launch_bounds__(kThreads)
k_scan_sums(unsigned long long* __restrict__ sums, uint32_t tiles, unsigned long long* __restrict__ offsets,
            uint32_t m, Status* __restrict__ st) {
  scan_sums(sums, tiles, offsets, m, st);
}

template <bool ONE>
__global__ void __launch_bounds__(kThreads)
k_scan_tiles(const uint32_t* __restrict__ counts, uint32_t m, const unsigned long long* __restrict__ sums,
             unsigned long long* __restrict__ offsets, Status* __restrict__ st) {
  scan_tile<ONE>(counts, m, blockIdx.x, sums, offsets, st);
}

// Several independent scans in the same three launches: the CTAs of the
// per-tile kernels are numbered over the jobs' tiles one job after another
// (job j owns CTAs [tile0[j], tile0[j + 1])); the tile-sum scan runs one
// CTA per job.  ONE: every job is a single tile, one launch in all.
struct ScanJobs {
  ScanJob job[kMaxScanJobs];
  uint32_t tile0[kMaxScanJobs + 1];
  int count;
};

__device__ __forceinline__ int job_of(const ScanJobs& js, uint32_t cta) {
  int j = 0;
  while (j + 1 < js.count && cta >= js.tile0[j + 1]) ++j;
  return j;
}

__global__ void __launch_bounds__(kThreads) k_tile_sums_multi(const ScanJobs js) {
  const int j = job_of(js, blockIdx.x);
  tile_sum(js.job[j].counts, js.job[j].m, blockIdx.x - js.tile0[j], js.job[j].sums);
}

__global__ void __launch_bounds__(kThreads) k_scan_sums_multi(const ScanJobs js) {
  const ScanJob& jb = js.job[blockIdx.x];
  scan_sums(jb.sums, js.tile0[blockIdx.x + 1] - js.tile0[blockIdx.x], jb.offsets, jb.m, jb.st);
}

template <bool ONE>
__global__ void __launch_bounds__(kThreads) k_scan_tiles_multi(const ScanJobs js) {
  const int j = job_of(js, blockIdx.x);
  const ScanJob& jb = js.job[j];
  scan_tile<ONE>(jb.counts, jb.m, blockIdx.x - js.tile0[j], jb.sums, jb.offsets, jb.st);
}

// Largest e in [begin, m] with offsets[e] - offsets[begin] <= capacity.
__global__ void k_chunk_end(const unsigned long long* __restrict__ offsets, uint32_t m, uint32_t begin,
                            unsigned long long capacity, Status* __restrict__ st) {
  const unsigned long long b0 = offsets[begin];
  uint32_t lo = begin, hi = m;  // invariant: offsets[lo] - b0 <= capacity
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (offsets[mid] - b0 <= capacity) lo = mid; else hi = mid - 1;
  }
  st->aux = lo;
  st->K = offsets[lo] - b0;
}

__global__ void k_flags(const uint32_t* __restrict__ qid, uint32_t m, uint32_t begin, uint32_t end,
                        uint32_t* __restrict__ flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const uint32_t v = qid[i];
    flags[i] = (v >= begin && v < end) ? 1u : 0u;
  }
}

__global__ void k_compact(const uint32_t* __restrict__ flags, const unsigned long long* __restrict__ offs,
                          uint32_t m, uint32_t* __restrict__ list) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (flags[i]) list[offs[i]] = i;
}

}  // namespace

cudaError_t launch_select(const uint32_t* qid, uint32_t m, uint32_t begin, uint32_t end,
                          uint32_t* flags, unsigned long long* offs, unsigned long long* sums,
                          uint32_t* list, Status* st, cudaStream_t s) {
  (void)st;
  if (m == 0) return cudaSuccess;
  uint32_t blocks = (m + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_flags<<<blocks, 256, 0, s>>>(qid, m, begin, end, flags);
  cudaError_t e = launch_scan(flags, m, offs, sums, nullptr, s);
  if (e) return e;
  k_compact<<<blocks, 256, 0, s>>>(flags, offs, m, list);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* counts, uint32_t m, unsigned long long* offsets,
                        unsigned long long* block_sums, Status* st, cudaStream_t s) {
  const uint32_t tiles = (m + kScanTile - 1) / kScanTile;
  if (tiles == 1) {  // one CTA does it all
    k_scan_tiles<true><<<1, kThreads, 0, s>>>(counts, m, block_sums, offsets, st);
    note_launches(1);
    return cudaGetLastError();
  }
  if (tiles > 0) k_tile_sums<<<tiles, kThreads, 0, s>>>(counts, m, block_sums);
  k_scan_sums<<<1, kThreads, 0, s>>>(block_sums, tiles, offsets, m, st);
  if (tiles > 0)
    k_scan_tiles<false><<<tiles, kThreads, 0, s>>>(counts, m, block_sums, offsets, nullptr);
  note_launches(tiles > 0 ? 3u : 1u);
  return cudaGetLastError();
}

cudaError_t launch_scan_multi(const ScanJob* jobs, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxScanJobs) return cudaErrorInvalidValue;
  ScanJobs js = {};
  js.count = count;
  bool one = true;
  for (int j = 0; j < count; ++j) {
    js.job[j] = jobs[j];
    const uint32_t t = (jobs[j].m + kScanTile - 1) / kScanTile;
    one = one && t <= 1;
    js.tile0[j + 1] = js.tile0[j] + (t ? t : 1);  // an empty job keeps one CTA (writes offsets[0])
  }
  for (int j = count + 1; j <= kMaxScanJobs; ++j) js.tile0[j] = js.tile0[count];
  const uint32_t tiles = js.tile0[count];
  if (one) {
    k_scan_tiles_multi<true><<<tiles, kThreads, 0, s>>>(js);
    note_launches(1);
    return cudaGetLastError();
  }
  k_tile_sums_multi<<<tiles, kThreads, 0, s>>>(js);
  k_scan_sums_multi<<<count, kThreads, 0, s>>>(js);
  k_scan_tiles_multi<false><<<tiles, kThreads, 0, s>>>(js);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_chunk_end(const unsigned long long* offsets, uint32_t m, uint32_t begin,
                             unsigned long long capacity, Status* st, cudaStream_t s) {
  k_chunk_end<<<1, 1, 0, s>>>(offsets, m, begin, capacity, st);
  note_launches(1);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the offsets scan (ddm_scan_counts_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the
// offsets: a real-time loop that must not block in the allocator (cudaMalloc
// and cudaFree can synchronise the whole device), or a host that hands all
// device memory to its own pool.  This entry point runs the same three scan
// kernels as launch_scan, with the per-tile sums kept in a fixed device array
// instead of a context buffer.
//
// Limits and sharing: the array holds kNoallocTiles tile sums, so m may be
// at most DDM_NOALLOC_MAX_UPDATES (= kNoallocTiles * 4096); every GPU that
// loads the library holds the array (128 KiB) until the process exits.  All
// calls share it, so calls whose kernels overlap on the GPU (different
// streams, or different host threads) race and must be serialised by the
// caller.  Each call writes every tile sum it later reads, so nothing
// needs clearing between calls.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoallocTiles = DDM_NOALLOC_MAX_UPDATES / kScanTile;
static_assert(DDM_NOALLOC_MAX_UPDATES % kScanTile == 0, "limit must be whole tiles");

static __device__ __align__(256) unsigned long long g_noalloc_tile_sums[kNoallocTiles];

namespace {

// Device address of g_noalloc_tile_sums per device, looked up once per device
// (host code cannot use the symbol itself as a device pointer).  Two host
// threads that make their first call on a device at the same time both look
// the address up and store the same value; the atomics make that race benign.
constexpr int kMaxDevices = 64;
std::atomic<unsigned long long*> g_noalloc_ptr[kMaxDevices];

}  // namespace

}  // namespace ddm

extern "C" int ddm_scan_counts_noalloc(const uint32_t* counts, uint32_t m, uint64_t* offsets,
                                       void* stream) {
  using namespace ddm;
  if (!offsets || (m > 0 && !counts)) return DDM_ERR_ARG;
  if (m > DDM_NOALLOC_MAX_UPDATES) return DDM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return DDM_ERR_CUDA;
  }
  unsigned long long* sums = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!sums) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_tile_sums) != cudaSuccess || !p) {
      cudaGetLastError();
      return DDM_ERR_CUDA;
    }
    sums = static_cast<unsigned long long*>(p);
    g_noalloc_ptr[dev].store(sums, std::memory_order_release);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t tiles = (m + kScanTile - 1) / kScanTile;
  auto* off = reinterpret_cast<unsigned long long*>(offsets);
  if (tiles > 0) k_tile_sums<<<tiles, kThreads, 0, s>>>(counts, m, sums);
  k_scan_sums<<<1, kThreads, 0, s>>>(sums, tiles, off, m, nullptr);
  if (tiles > 0) k_scan_tiles<false><<<tiles, kThreads, 0, s>>>(counts, m, sums, off, nullptr);
  note_launches(tiles > 0 ? 3u : 1u);
  if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
  return DDM_OK;
}
