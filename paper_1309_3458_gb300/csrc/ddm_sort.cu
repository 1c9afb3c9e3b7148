// LSD radix sort of 64-bit keys with a 32-bit payload.
//
// Sorts the subscriptions into the interval tree order of Section IV (lower
// bound, then upper bound; the stable passes keep remaining ties in id
// order), and the updates and the re-sorts into locality orders.  Three
// forms by size, each a stable sort over 8-bit digits:
//   * up to 16 tiles of 2,048 keys: one thread-block cluster keeps the keys
//     in distributed shared memory for every pass (k_sort_cluster);
//   * up to one resident tile per SM: one cooperative launch runs every pass,
//     the tiles exchanging digit counts across bounded grid barriers
//     (k_sort_grid);
//   * beyond (and under stream capture): onesweep, after Adinets & Merrill
//     ("Onesweep", 2022): one histogram pass over the keys computes all eight
//     8-bit digit histograms at once, a tiny kernel scans them into digit
//     bases, and each digit pass is ONE kernel: a CTA takes the next tile
//     (ticket from an atomic counter, so every earlier tile is already
//     resident), ranks its keys per digit with a warp match (one ballot per
//     digit bit) and per-warp counters, publishes its per-digit counts,
//     resolves its global per-digit offsets by decoupled look-back over
//     earlier tiles, and scatters through shared memory so that global
//     stores come out as runs of equal digits.  Under stream capture, sets of
//     up to 8,192 keys take one CTA instead (k_sort_small).
// Every wait is bounded: after kSpinLimit polls a CTA records kErrTimeout and
// carries on (look-back) or returns (grid barrier), so the kernels always
// terminate.
#include <algorithm>
#include <atomic>

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

// Lanes of the warp holding the same digit (0..256, 256 = no key): one
// ballot per digit bit.  Measured: the 8,192-key single-CTA sort took 59
// instead of 88 us with this in place of match.any, which the SM's warps
// issue one at a time.
__device__ __forceinline__ uint32_t same_digit_lanes(uint32_t dig) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b <= kRadixBits; ++b) {
    const uint32_t bit = (dig >> b) & 1u;
    const uint32_t votes = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? votes : ~votes;
  }
  return peers;
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

  // Rank within the warp, item by item: lanes sharing a digit are found by
  // ballots; the lowest such lane bumps the warp's counter for the digit.
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t peers = same_digit_lanes(dig[i]);
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

// Ranking of one tile of 512 * ITEMS keys held in registers by 512 threads
// (item i of lane l in warp w is the tile's element w*32*ITEMS + i*32 + l):
// the same stable ranking as k_onesweep (warp match + per-warp counters,
// warps in order).  Afterwards whist[w][dg] is warp w's first slot within
// digit dg, lstart[dg] the digit's first slot in the tile, and the returned
// count (threads < 256, digit = thread) the tile's keys with that digit.
constexpr int kSmallThreads = 512;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr uint32_t kSmallTile = kSmallThreads * kItems;  // 8192

struct RankSmem {
  uint32_t whist[kSmallWarps][kRadix];
  uint32_t wtot[kRadix / 32];
  uint32_t lstart[kRadix];
};

template <int ITEMS>
__device__ __forceinline__ uint32_t rank_tile(RankSmem& sm, const unsigned long long (&key)[ITEMS],
                                              uint32_t (&dig)[ITEMS], uint32_t (&rank)[ITEMS],
                                              uint32_t valid, int shift) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  for (int t = tid; t < kSmallWarps * kRadix; t += kSmallThreads) (&sm.whist[0][0])[t] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t local = warp * (ITEMS * 32) + i * 32 + lane;
    dig[i] = local < valid ? (uint32_t)(key[i] >> shift) & (kRadix - 1) : kRadix;
    const uint32_t peers = same_digit_lanes(dig[i]);
    uint32_t before = 0;
    if (dig[i] < kRadix) before = sm.whist[warp][dig[i]];
    rank[i] = before + __popc(peers & lt);
    __syncwarp();
    if (dig[i] < kRadix && (peers & lt) == 0) sm.whist[warp][dig[i]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  uint32_t count = 0;
  if (tid < kRadix) {  // thread t owns digit t: per-warp offsets, tile offsets
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
  return count;
}

// Small arrays (n <= kSmallTile): one CTA of 512 threads runs every digit
// pass in shared memory, with the tile's own digit offsets in place of the
// look-back, so the whole sort is one launch.
struct SmallSortSmem {
  RankSmem r;
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
  unsigned long long key[kItems];
  uint32_t val[kItems], dig[kItems], rank[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t local = warp * (kItems * 32) + i * 32 + lane;
    key[i] = local < n ? in_keys[local] : 0ull;
    val[i] = local < n ? in_vals[local] : 0u;
  }
  for (int p = 0; p < passes; ++p) {
    rank_tile<kItems>(sm.r, key, dig, rank, n, p * kRadixBits);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (dig[i] < kRadix) {
        const uint32_t slot = sm.r.lstart[dig[i]] + sm.r.whist[warp][dig[i]] + rank[i];
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

// Mid-size arrays (up to kGridMaxTiles tiles of 512 * ITEMS keys, all CTAs
// resident): one cooperative launch runs every pass.  CTA g holds tile g in
// registers and ranks it as k_sort_small does; the tiles then exchange their
// digit counts through global memory across a grid barrier, each CTA takes
// its digit offsets from the counts (no look-back chain), scatters, and a
// second barrier ends the pass.  Tiles come in groups of kGridGroup: a tile
// adds its counts into its group's sums (global atomics) and stores them,
// 16-bit and packed two to a word, in its own row; a digit's total is the
// sum of the group sums and the part before tile g the sums of the groups
// before g's plus the rows of g's group before it -- at most 12 + 15 reads
// per digit instead of one per tile.  The group sums are double-buffered by
// pass parity, and each pass clears the buffer of the next.  Smaller tiles
// (fewer items per thread) spread a set over more SMs: each pass's ranking
// and scatter shrink with the tile, the two barriers do not.
constexpr uint32_t kGridMaxTiles = 192;
constexpr uint32_t kGridGroup = 16;
constexpr uint32_t kGridGroups = kGridMaxTiles / kGridGroup;  // 12
// Scratch words of a cooperative sort: the per-tile rows, the group sums of
// both parities and the barrier counter (the last two zeroed before each
// launch).
constexpr size_t kGridRowWords = (size_t)kGridMaxTiles * (kRadix / 2);
constexpr size_t kGridSumWords = 2 * (size_t)kGridGroups * kRadix;
constexpr size_t kGridScratchWords = kGridRowWords + kGridSumWords + 32;

template <int ITEMS>
struct GridSortSmem {
  RankSmem r;
  uint32_t gbase[kRadix];
  uint32_t dtot[kRadix / 32];
  int abort;
  int pad[3];
  unsigned long long keys[kSmallThreads * ITEMS];
  uint32_t vals[kSmallThreads * ITEMS];
};

// Grid-wide barrier for a cooperative launch (all CTAs resident).  `bar` is
// zeroed before the launch and only grows; barrier number b completes when
// it reaches gridDim.x * b.  The wait is bounded: after kSpinLimit polls
// the CTA records kErrTimeout and the kernel returns false to every thread
// of it, so every CTA ends (those left waiting time out in turn).
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t target, Status* st,
                                             int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    bool timed_out = false;
    for (uint32_t spins = 0;; ++spins) {
      uint32_t v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (spins >= kSpinLimit) {
        timed_out = true;
        break;
      }
      __nanosleep(32);
    }
    if (timed_out) {
      atomicOr(&st->err, kErrTimeout);
      *s_abort = 1;
    }
    __threadfence();
  }
  __syncthreads();
  return *s_abort == 0;
}

template <int ITEMS>
__global__ void __launch_bounds__(kSmallThreads, 1)
k_sort_grid(unsigned long long* __restrict__ keys0, uint32_t* __restrict__ vals0,
            unsigned long long* __restrict__ keys1, uint32_t* __restrict__ vals1, uint32_t n,
            int passes, uint32_t* __restrict__ table, uint32_t* __restrict__ bar,
            Status* __restrict__ st) {
  constexpr uint32_t kTile = kSmallThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GridSortSmem<ITEMS>& sm = *reinterpret_cast<GridSortSmem<ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blockIdx.x, tiles = gridDim.x;
  const size_t base = (size_t)tile * kTile;
  const uint32_t valid = (uint32_t)min((size_t)kTile, (size_t)n - base);
  if (tid == 0) sm.abort = 0;
  uint32_t barriers = 0;
  unsigned long long key[ITEMS];
  uint32_t val[ITEMS], dig[ITEMS], rank[ITEMS];
  for (int p = 0; p < passes; ++p) {
    const unsigned long long* ik = (p & 1) ? keys1 : keys0;
    const uint32_t* iv = (p & 1) ? vals1 : vals0;
    unsigned long long* ok = (p & 1) ? keys0 : keys1;
    uint32_t* ov = (p & 1) ? vals0 : vals1;
    // written by other CTAs of this launch: read through L2, not L1
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t local = warp * (ITEMS * 32) + i * 32 + lane;
      key[i] = local < valid ? __ldcg(ik + base + local) : 0ull;
      val[i] = local < valid ? __ldcg(iv + base + local) : 0u;
    }
    const int shift = p * kRadixBits;
    const uint32_t count = rank_tile<ITEMS>(sm.r, key, dig, rank, valid, shift);
    uint32_t* gsum = table + kGridRowWords + (size_t)(p & 1) * kGridGroups * kRadix;
    if (tid < kRadix) {  // this tile's counts: its row (two 16-bit digits per word), its group's sums
      const uint32_t next = __shfl_down_sync(0xffffffffu, count, 1);
      if ((tid & 1) == 0) __stcg(table + (size_t)tile * (kRadix / 2) + tid / 2, count | (next << 16));
      if (count) atomicAdd(&gsum[(tile / kGridGroup) * kRadix + tid], count);
    }
    if (!grid_barrier(bar, tiles * ++barriers, st, &sm.abort)) return;
    {  // clear the next pass's group sums (last read in the previous pass)
      uint32_t* other = table + kGridRowWords + (size_t)((p + 1) & 1) * kGridGroups * kRadix;
      for (uint32_t q = tile * kSmallThreads + tid; q < kGridGroups * kRadix; q += tiles * kSmallThreads)
        other[q] = 0u;
    }
    if (tid < kRadix) {  // digit tid: its total, and the part before this tile
      const uint32_t groups = (tiles + kGridGroup - 1) / kGridGroup, mine = tile / kGridGroup;
      uint32_t tot = 0, pre = 0;
      for (uint32_t g = 0; g < groups; ++g) {
        const uint32_t c = __ldcg(gsum + g * kRadix + tid);
        tot += c;
        pre += g < mine ? c : 0u;
      }
      for (uint32_t t = mine * kGridGroup; t < tile; ++t)
        pre += (__ldcg(table + (size_t)t * (kRadix / 2) + tid / 2) >> ((tid & 1) * 16)) & 0xffffu;
      // exclusive scan of the digit totals: the digit's first position
      uint32_t x = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) sm.dtot[warp] = x;
      sm.gbase[tid] = x - tot + pre - sm.r.lstart[tid];
    }
    __syncthreads();
    if (tid < kRadix) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += sm.dtot[w];
      sm.gbase[tid] += pre;  // modular: gbase + slot is exact
    }
    // stage the tile in (digit, input order) order ...
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (dig[i] < kRadix) {
        const uint32_t slot = sm.r.lstart[dig[i]] + sm.r.whist[warp][dig[i]] + rank[i];
        sm.keys[slot] = key[i];
        sm.vals[slot] = val[i];
      }
    }
    __syncthreads();
    // ... and out, consecutive threads taking consecutive slots
    for (uint32_t q = tid; q < valid; q += kSmallThreads) {
      const unsigned long long k = sm.keys[q];
      const uint32_t g = sm.gbase[(uint32_t)(k >> shift) & (kRadix - 1)] + q;
      if (DDM_IN_BOUNDS(g < n, st)) {
        ok[g] = k;
        ov[g] = sm.vals[q];
      }
    }
    if (p + 1 < passes && !grid_barrier(bar, tiles * ++barriers, st, &sm.abort)) return;
  }
}

// Small sets (up to kClusterMax tiles of 512 * ITEMS keys): one thread-block
// cluster holds the whole set in shared memory.  Each pass ranks a tile as
// k_sort_grid does, writes its digit counts into every CTA's count table
// (distributed shared memory), and after a cluster barrier scatters its
// keys straight into the shared-memory tiles of their next owners; a second
// cluster barrier ends the pass, and only the last pass writes to global
// memory.  Both barriers are the hardware cluster barrier (no polling), and
// no key goes through L2 between passes.
constexpr uint32_t kClusterMax = 16;

template <int ITEMS>
struct ClusterSortSmem {
  RankSmem r;
  uint32_t gbase[kRadix];
  uint32_t dtot[kRadix / 32];
  uint32_t table[kClusterMax][kRadix];  // row j: CTA j's digit counts
  unsigned long long tile_k[kSmallThreads * ITEMS];  // this CTA's keys of the next pass
  uint32_t tile_v[kSmallThreads * ITEMS];
  unsigned long long stage_k[kSmallThreads * ITEMS];  // this pass's keys in digit order
  uint32_t stage_v[kSmallThreads * ITEMS];
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of `p` (this CTA's shared memory) in CTA `cta`'s shared memory.
__device__ __forceinline__ uint32_t remote_smem(const void* p, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(cta));
  return r;
}
__device__ __forceinline__ void st_remote(uint32_t a, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_remote(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

template <int ITEMS>
__global__ void __launch_bounds__(kSmallThreads, 1)
k_sort_cluster(const unsigned long long* __restrict__ in_k, const uint32_t* __restrict__ in_v,
               unsigned long long* __restrict__ out_k, uint32_t* __restrict__ out_v, uint32_t n,
               int passes) {
  constexpr uint32_t kTile = kSmallThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ClusterSortSmem<ITEMS>& sm = *reinterpret_cast<ClusterSortSmem<ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t me = cluster_rank(), ctas = gridDim.x;  // the grid is one cluster
  const uint32_t base = me * kTile;
  const uint32_t valid = min(kTile, n - base);
  unsigned long long key[ITEMS];
  uint32_t val[ITEMS], dig[ITEMS], rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t local = warp * (ITEMS * 32) + i * 32 + lane;
    key[i] = local < valid ? in_k[base + local] : 0ull;
    val[i] = local < valid ? in_v[base + local] : 0u;
  }
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kRadixBits;
    const uint32_t count = rank_tile<ITEMS>(sm.r, key, dig, rank, valid, shift);
    if (tid < kRadix)
      for (uint32_t j = 0; j < ctas; ++j) st_remote(remote_smem(&sm.table[me][tid], j), count);
    cluster_sync_all();  // every table complete; every CTA holds its keys in registers
    if (tid < kRadix) {  // the digit's first position, plus the CTAs before this one
      uint32_t tot = 0, pre = 0;
      for (uint32_t j = 0; j < ctas; ++j) {
        const uint32_t c = sm.table[j][tid];
        tot += c;
        pre += j < me ? c : 0u;
      }
      uint32_t x = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) sm.dtot[warp] = x;
      sm.gbase[tid] = x - tot + pre - sm.r.lstart[tid];
    }
    __syncthreads();
    if (tid < kRadix) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += sm.dtot[w];
      sm.gbase[tid] += pre;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (dig[i] < kRadix) {
        const uint32_t slot = sm.r.lstart[dig[i]] + sm.r.whist[warp][dig[i]] + rank[i];
        sm.stage_k[slot] = key[i];
        sm.stage_v[slot] = val[i];
      }
    }
    __syncthreads();
    const bool last = p + 1 == passes;
    // consecutive threads take consecutive slots: runs of one digit land in
    // consecutive positions of one owner
    for (uint32_t q = tid; q < valid; q += kSmallThreads) {
      const unsigned long long k = sm.stage_k[q];
      const uint32_t g = sm.gbase[(uint32_t)(k >> shift) & (kRadix - 1)] + q;
      if (!DDM_IN_BOUNDS(g < n, nullptr)) continue;
      if (last) {
        out_k[g] = k;
        out_v[g] = sm.stage_v[q];
      } else {
        const uint32_t owner = g / kTile, at = g % kTile;
        st_remote(remote_smem(&sm.tile_k[at], owner), k);
        st_remote(remote_smem(&sm.tile_v[at], owner), sm.stage_v[q]);
      }
    }
    if (last) break;
    cluster_sync_all();  // every key of the next pass is in its owner's tile
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t local = warp * (ITEMS * 32) + i * 32 + lane;
      key[i] = local < valid ? sm.tile_k[local] : 0ull;
      val[i] = local < valid ? sm.tile_v[local] : 0u;
    }
  }
}

// Largest cluster (CTAs) k_sort_cluster<ITEMS> can run on the current
// device: 16 (non-portable), else 8, else 0.
template <int ITEMS>
int cluster_sort_ctas() {
  static std::atomic<int> best[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  int b = best[dev].load(std::memory_order_relaxed);
  if (b == 0) {
    b = -1;
    const size_t smem = sizeof(ClusterSortSmem<ITEMS>);
    if (cudaFuncSetAttribute(k_sort_cluster<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess &&
        cudaFuncSetAttribute(k_sort_cluster<ITEMS>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kSmallThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_sort_cluster<ITEMS>, &cfg) == cudaSuccess &&
            clusters > 0) {
          b = c;
          break;
        }
      }
    }
    cudaGetLastError();
    best[dev].store(b, std::memory_order_relaxed);
  }
  return b < 0 ? 0 : b;
}

// One cluster launch of k_sort_cluster<ITEMS> if the set fits one cluster:
// *done = true then (or an error), else nothing is enqueued.
template <int ITEMS>
cudaError_t try_sort_cluster(SortScratch sc, uint32_t n, int passes, cudaStream_t s, bool* done) {
  *done = false;
  constexpr uint32_t kTile = kSmallThreads * ITEMS;
  const uint32_t ctas = (n + kTile - 1) / kTile;
  if (ctas > (uint32_t)cluster_sort_ctas<ITEMS>()) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = sizeof(ClusterSortSmem<ITEMS>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int out = passes & 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_sort_cluster<ITEMS>, sc.keys[0], sc.vals[0],
                                     sc.keys[out], sc.vals[out], n, passes);
  if (e == cudaSuccess) {
    note_launches(1);
    *done = true;
  }
  return e;
}

// Co-resident CTAs of k_sort_grid<ITEMS> on the current device, capped at
// kGridMaxTiles (0: not usable).
template <int ITEMS>
int grid_sort_tiles(int sms) {
  static std::atomic<int> per_sm[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  int b = per_sm[dev].load(std::memory_order_relaxed);
  if (b == 0) {
    const size_t smem = sizeof(GridSortSmem<ITEMS>);
    if (cudaFuncSetAttribute(k_sort_grid<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sort_grid<ITEMS>, kSmallThreads, smem)) {
      cudaGetLastError();
      b = 0;
    }
    per_sm[dev].store(b > 0 ? b : -1, std::memory_order_relaxed);
  }
  if (b < 0) return 0;
  return (int)std::min<long long>((long long)b * sms, kGridMaxTiles);
}

// One cooperative launch of k_sort_grid<ITEMS> if the set fits its resident
// grid: *done = true then (or an error), else nothing is enqueued.
template <int ITEMS>
cudaError_t try_sort_grid(SortScratch sc, uint32_t n, int passes, Status* st, int sms,
                          cudaStream_t s, bool* done) {
  *done = false;
  constexpr uint32_t kTile = kSmallThreads * ITEMS;
  const uint32_t tiles = (n + kTile - 1) / kTile;
  if (tiles > (uint32_t)grid_sort_tiles<ITEMS>(sms)) return cudaSuccess;
  cudaError_t e;
  // both parities' group sums and the barrier counter start at zero
  uint32_t* sums = sc.lookback + kGridRowWords;
  if ((e = cudaMemsetAsync(sums, 0, sizeof(uint32_t) * (kGridSumWords + 1), s))) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = sizeof(GridSortSmem<ITEMS>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_sort_grid<ITEMS>, sc.keys[0], sc.vals[0], sc.keys[1], sc.vals[1],
                         n, passes, sc.lookback, sums + kGridSumWords, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {  // fewer SMs available than counted
    cudaGetLastError();
    return cudaSuccess;
  }
  if (e == cudaSuccess) {
    note_launches(1);
    *done = true;
  }
  return e;
}

}  // namespace

cudaError_t launch_debug_wait(const uint32_t* word, uint32_t limit, Status* st, cudaStream_t s) {
  k_debug_wait<<<1, 32, 0, s>>>(word, limit, st);
  note_launches(1);
  return cudaGetLastError();
}

size_t sort_lookback_words(uint32_t n) {
  const size_t tiles = ((size_t)n + kSortTile - 1) / kSortTile;
  // the onesweep look-back words, or the cooperative sort's rows, group sums and counter
  return std::max((size_t)kPasses * tiles * kRadix, kGridScratchWords);
}

cudaError_t launch_sort64(SortScratch sc, uint32_t n, int passes, int* out_buf, Status* st,
                          int sms, cudaStream_t s) {
  *out_buf = 0;
  if (n <= 1 || passes <= 0) return cudaSuccess;
  if (passes > kPasses) passes = kPasses;
  cudaError_t e;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap))) return e;
  // Up to 16 tiles of 2,048 keys: one cluster, keys kept on chip; else one
  // cooperative launch when every tile can be resident at once, with the
  // smallest tile that allows it.  Measured (8 passes, one GB300): 5,000
  // keys 33 us in a cluster, 53 cooperative, 51 in one CTA; 25,000 keys 41,
  // 57 (2,048-key tiles) and 100 (8,192-key tiles); 250,000 keys 76
  // cooperative.  Not under stream capture: the single-CTA or multi-launch
  // form is recorded instead.
  if (cap == cudaStreamCaptureStatusNone) {
    bool done = false;
    if ((e = try_sort_cluster<4>(sc, n, passes, s, &done)) || done) {
      *out_buf = passes & 1;
      return e;
    }
    if ((e = try_sort_grid<4>(sc, n, passes, st, sms, s, &done)) || done) {
      *out_buf = passes & 1;
      return e;
    }
    if ((e = try_sort_grid<8>(sc, n, passes, st, sms, s, &done)) || done) {
      *out_buf = passes & 1;
      return e;
    }
    if ((e = try_sort_grid<16>(sc, n, passes, st, sms, s, &done)) || done) {
      *out_buf = passes & 1;
      return e;
    }
  }
  if (n <= kSmallTile) {  // one CTA, every pass in shared memory
    const size_t smem = sizeof(SmallSortSmem);
    if ((e = cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    const int out = passes & 1;
    k_sort_small<<<1, kSmallThreads, smem, s>>>(sc.keys[0], sc.vals[0], sc.keys[out], sc.vals[out],
                                                n, passes);
    note_launches(1);
    *out_buf = out;
    return cudaGetLastError();
  }
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
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
