// Onesweep LSD radix sort of 64-bit keys with a 32-bit payload.
//
// Sorts the subscriptions into the interval tree order of Section IV (lower
// bound, then upper bound; the stable passes keep remaining ties in id
// order).  Design (after Adinets & Merrill, "Onesweep", 2022):
//   1. one histogram pass over the keys computes all eight 8-bit digit
//      histograms at once; a tiny kernel scans them into digit bases;
//   2. each digit pass is ONE kernel: a CTA takes the next tile (ticket from
//      an atomic counter, so every earlier tile is already resident), ranks
//      its keys per digit with warp match + per-warp counters, publishes its
//      per-digit counts, resolves its global per-digit offsets by decoupled
//      look-back over earlier tiles, and scatters through shared memory so
//      that global stores come out as runs of equal digits.
// Look-back waits are bounded: after kSpinLimit polls a CTA records
// kErrTimeout and carries on, so the kernel always terminates.
#include "ddm_internal.cuh"

namespace ddm {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPasses = 64 / kRadixBits;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = kSortTile / kThreads;  // 16 keys per thread
constexpr uint32_t kFlagAgg = 1u << 30;       // tile aggregate available
constexpr uint32_t kFlagInc = 2u << 30;       // inclusive prefix available
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

static_assert(kSortTile % kThreads == 0, "tile must split evenly over threads");

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded poll of a look-back word: returns it once any bit of `mask` is
// set, or 0 with *timed_out after `limit` polls (64 ns apart), so that no
// wait can outlive a predecessor that never publishes.
__device__ __forceinline__ uint32_t poll_flag(const uint32_t* p, uint32_t mask, uint32_t limit,
                                              bool* timed_out) {
  for (uint32_t spins = 0;; ++spins) {
    const uint32_t w = ld_relaxed(p);
    if (w & mask) return w;
    if (spins >= limit) {
      *timed_out = true;
      return 0u;
    }
    __nanosleep(64);
  }
}

// Test hook for the bounded waits: poll a word nothing sets.
__global__ void k_debug_wait(const uint32_t* __restrict__ word, uint32_t limit,
                             Status* __restrict__ st) {
  bool timed_out = false;
  poll_flag(word, kFlagMask, limit, &timed_out);
  if (timed_out && threadIdx.x == 0) atomicOr(&st->err, kErrTimeout);
}

// All eight digit histograms in one read of the keys.
__global__ void __launch_bounds__(kThreads)
k_histogram(const unsigned long long* __restrict__ keys, uint32_t n, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kPasses * kRadix];
  for (int t = threadIdx.x; t < kPasses * kRadix; t += kThreads) h[t] = 0;
  __syncthreads();
  const uint32_t stride = gridDim.x * kThreads;
  for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
    const unsigned long long k = keys[i];
#pragma unroll
    for (int p = 0; p < kPasses; ++p)
      atomicAdd(&h[p * kRadix + (uint32_t)((k >> (p * kRadixBits)) & (kRadix - 1))], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kPasses * kRadix; t += kThreads)
    if (h[t]) atomicAdd(&hist[t], h[t]);
}

// Exclusive scan of each pass's 256-bin histogram, in place (one CTA per pass).
__global__ void __launch_bounds__(kRadix) k_hist_scan(uint32_t* __restrict__ hist) {
  __shared__ uint32_t warp_tot[kRadix / 32];
  uint32_t* h = hist + blockIdx.x * kRadix;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t v = h[t];
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int i = 0; i < w; ++i) pre += warp_tot[i];
  h[t] = pre + x - v;
}

struct OnesweepSmem {
  uint32_t whist[kWarps][kRadix];  // per-warp digit counts, then per-warp exclusive offsets
  uint32_t lstart[kRadix];         // tile-local start of each digit
  uint32_t gbase[kRadix];          // global position of local slot 0 of each digit
  uint32_t wtot[kRadix / 32];
  uint32_t tile;
  unsigned long long keys[kSortTile];
  uint32_t vals[kSortTile];
};

// Three resident CTAs per SM (registers capped at 80, a few spilled): measured
// faster than two CTAs at 128 registers.
__global__ void __launch_bounds__(kThreads, 3)
k_onesweep(const unsigned long long* __restrict__ in_keys, const uint32_t* __restrict__ in_vals,
           unsigned long long* __restrict__ out_keys, uint32_t* __restrict__ out_vals, uint32_t n,
           int shift, const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ lookback,
           uint32_t* __restrict__ counter, Status* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  OnesweepSmem& sm = *reinterpret_cast<OnesweepSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) sm.tile = atomicAdd(counter, 1u);
  for (int t = tid; t < kWarps * kRadix; t += kThreads) (&sm.whist[0][0])[t] = 0;
  __syncthreads();
  const uint32_t tile = sm.tile;
  const size_t tile_base = (size_t)tile * kSortTile;
  const uint32_t tile_valid = (uint32_t)min((size_t)kSortTile, (size_t)n - tile_base);

  // Load: warp w owns keys [w*512, w*512+512) of the tile; item i of a lane
  // is key w*512 + i*32 + lane, so (warp, item, lane) is input order.
  unsigned long long key[kItems];
  uint32_t val[kItems], dig[kItems], rank[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
    if (local < tile_valid) {
      key[i] = in_keys[tile_base + local];
      val[i] = in_vals[tile_base + local];
      dig[i] = (uint32_t)(key[i] >> shift) & (kRadix - 1);
    } else {
      key[i] = 0;
      val[i] = 0;
      dig[i] = kRadix;  // sentinel: not counted
    }
  }

  // Rank within the warp, item by item: lanes sharing a digit are found with
  // match.any; the lowest such lane bumps the warp's counter for the digit.
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t peers = __match_any_sync(0xffffffffu, dig[i]);
    uint32_t before = 0;
    if (dig[i] < kRadix) before = sm.whist[warp][dig[i]];
    rank[i] = before + __popc(peers & lt);
    __syncwarp();
    if (dig[i] < kRadix && (peers & lt) == 0) sm.whist[warp][dig[i]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // Thread t owns digit t: per-warp exclusive offsets and the tile count.
  uint32_t count = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = sm.whist[w][tid];
    sm.whist[w][tid] = count;
    count += c;
  }
  uint32_t* my_slot = lookback + (size_t)tile * kRadix + tid;
  st_relaxed(my_slot, (tile == 0 ? kFlagInc : kFlagAgg) | count);

  // Tile-local exclusive scan of the digit counts.
  uint32_t x = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm.wtot[warp] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < warp; ++w) pre += sm.wtot[w];
  const uint32_t lstart = pre + x - count;
  sm.lstart[tid] = lstart;

  // Decoupled look-back over earlier tiles for digit `tid`.
  uint32_t excl = 0;
  if (tile > 0) {
    uint32_t p = tile - 1;
    for (;;) {
      bool timed_out = false;
      const uint32_t w = poll_flag(lookback + (size_t)p * kRadix + tid, kFlagMask, kSpinLimit,
                                   &timed_out);
      if (timed_out) {
        atomicOr(&st->err, kErrTimeout);
        break;
      }
      excl += w & kValMask;
      if ((w & kFlagMask) == kFlagInc || p == 0) break;
      --p;
    }
    st_relaxed(my_slot, kFlagInc | (excl + count));
  }
  sm.gbase[tid] = digit_base[tid] + excl - lstart;  // modular: gbase + slot is exact
  __syncthreads();

  // Scatter into shared memory in (digit, input order) order ...
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (dig[i] < kRadix) {
      const uint32_t slot = sm.lstart[dig[i]] + sm.whist[warp][dig[i]] + rank[i];
      sm.keys[slot] = key[i];
      sm.vals[slot] = val[i];
    }
  }
  __syncthreads();
  // ... and out to global memory, consecutive threads taking consecutive slots.
  for (uint32_t s = tid; s < tile_valid; s += kThreads) {
    const unsigned long long k = sm.keys[s];
    const uint32_t g = sm.gbase[(uint32_t)(k >> shift) & (kRadix - 1)] + s;
    if (DDM_IN_BOUNDS(g < n, st)) {
      out_keys[g] = k;
      out_vals[g] = sm.vals[s];
    }
  }
}

// Small arrays (n <= kSmallTile): one CTA of 512 threads runs every digit
// pass in shared memory -- the same stable ranking as k_onesweep (warp match
// + per-warp counters, warps in order), with the tile's own digit offsets in
// place of the look-back -- so the whole sort is one launch.
constexpr int kSmallThreads = 512;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr uint32_t kSmallTile = kSmallThreads * kItems;  // 8192

struct SmallSortSmem {
  uint32_t whist[kSmallWarps][kRadix];
  uint32_t wtot[kRadix / 32];
  uint32_t lstart[kRadix];
  unsigned long long keys[kSmallTile];
  uint32_t vals[kSmallTile];
};

__global__ void __launch_bounds__(kSmallThreads, 1)
k_sort_small(const unsigned long long* __restrict__ in_keys, const uint32_t* __restrict__ in_vals,
             unsigned long long* __restrict__ out_keys, uint32_t* __restrict__ out_vals,
             uint32_t n, int passes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSortSmem& sm = *reinterpret_cast<SmallSortSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  unsigned long long key[kItems];
  uint32_t val[kItems], rank[kItems];
  // item i of lane l in warp w is element w*512 + i*32 + l (input order)
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
    key[i] = local < n ? in_keys[local] : 0ull;
    val[i] = local < n ? in_vals[local] : 0u;
  }
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kRadixBits;
    for (int t = tid; t < kSmallWarps * kRadix; t += kSmallThreads) (&sm.whist[0][0])[t] = 0;
    __syncthreads();
    uint32_t dig[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
      dig[i] = local < n ? (uint32_t)(key[i] >> shift) & (kRadix - 1) : kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[i]);
      uint32_t before = 0;
      if (dig[i] < kRadix) before = sm.whist[warp][dig[i]];
      rank[i] = before + __popc(peers & lt);
      __syncwarp();
      if (dig[i] < kRadix && (peers & lt) == 0) sm.whist[warp][dig[i]] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (tid < kRadix) {  // thread t owns digit t: per-warp offsets, tile offsets
      uint32_t count = 0;
#pragma unroll
      for (int w = 0; w < kSmallWarps; ++w) {
        const uint32_t c = sm.whist[w][tid];
        sm.whist[w][tid] = count;
        count += c;
      }
      uint32_t x = count;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) sm.wtot[warp] = x;
      sm.lstart[tid] = x - count;  // within-warp part; warp prefix added below
    }
    __syncthreads();
    if (tid < kRadix) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += sm.wtot[w];
      sm.lstart[tid] += pre;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (dig[i] < kRadix) {
        const uint32_t slot = sm.lstart[dig[i]] + sm.whist[warp][dig[i]] + rank[i];
        sm.keys[slot] = key[i];
        sm.vals[slot] = val[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
      if (local < n) {
        key[i] = sm.keys[local];
        val[i] = sm.vals[local];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
    if (local < n) {
      out_keys[local] = key[i];
      out_vals[local] = val[i];
    }
  }
}

}  // namespace

cudaError_t launch_debug_wait(const uint32_t* word, uint32_t limit, Status* st, cudaStream_t s) {
  k_debug_wait<<<1, 32, 0, s>>>(word, limit, st);
  note_launches(1);
  return cudaGetLastError();
}

size_t sort_lookback_words(uint32_t n) {
  const size_t tiles = ((size_t)n + kSortTile - 1) / kSortTile;
  return (size_t)kPasses * tiles * kRadix;
}

cudaError_t launch_sort64(SortScratch sc, uint32_t n, int passes, int* out_buf, Status* st,
                          int sms, cudaStream_t s) {
  *out_buf = 0;
  if (n <= 1 || passes <= 0) return cudaSuccess;
  if (passes > kPasses) passes = kPasses;
  if (n <= kSmallTile) {  // one CTA, every pass in shared memory
    const size_t smem = sizeof(SmallSortSmem);
    cudaError_t e = cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    const int out = passes & 1;
    k_sort_small<<<1, kSmallThreads, smem, s>>>(sc.keys[0], sc.vals[0], sc.keys[out], sc.vals[out],
                                                n, passes);
    note_launches(1);
    *out_buf = out;
    return cudaGetLastError();
  }
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * kPasses * kRadix, s))) return e;
  if ((e = cudaMemsetAsync(sc.counters, 0, sizeof(uint32_t) * kPasses, s))) return e;
  if ((e = cudaMemsetAsync(sc.lookback, 0, sizeof(uint32_t) * (size_t)passes * tiles * kRadix, s)))
    return e;
  uint32_t hb = (n + kThreads * 16 - 1) / (kThreads * 16);
  if (hb > (uint32_t)sms * 4u) hb = (uint32_t)sms * 4u;
  k_histogram<<<hb, kThreads, 0, s>>>(sc.keys[0], n, sc.hist);
  k_hist_scan<<<kPasses, kRadix, 0, s>>>(sc.hist);
  const size_t smem = sizeof(OnesweepSmem);
  if ((e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)))
    return e;
  for (int p = 0; p < passes; ++p) {
    const int src = p & 1;
    k_onesweep<<<tiles, kThreads, smem, s>>>(sc.keys[src], sc.vals[src], sc.keys[src ^ 1],
                                             sc.vals[src ^ 1], n, p * kRadixBits,
                                             sc.hist + p * kRadix,
                                             sc.lookback + (size_t)p * tiles * kRadix,
                                             sc.counters + p, st);
  }
  note_launches(2u + (unsigned)passes);
  *out_buf = passes & 1;
  return cudaGetLastError();
}

}  // namespace ddm
