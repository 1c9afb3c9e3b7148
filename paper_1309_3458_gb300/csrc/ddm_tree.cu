// Implicit interval tree build (Section IV, Interval-Tree-Create of Alg. 5).
//
// The paper stores the subscriptions in an augmented AVL tree ordered by
// lower bound, each node keeping maxupper and minlower of its subtree, and
// notes that any interval tree may stand in for it.  The GPU keeps the order
// and the two subtree bounds in a flattened, pointer-free form:
//
//   * the sorted subscriptions themselves are the leaves;
//   * a level-l node g covers the sorted positions [g*32^l, (g+1)*32^l) and
//     stores (minlower, maxupper) of that range -- for every dimension, so
//     that the d-dimensional test of Section III-A prunes whole subtrees;
//   * the top level has at most 32 nodes, so one warp tests it in one step.
//
// The bounds are min/max reductions done with warp shuffles (32 children
// per warp), level by level from the leaves up.  The element order comes
// from ddm_layout.cu / ddm_sort.cu: dimension-0 (lower, upper, id), refined
// inside aligned groups by the lower bound of the other dimensions (for
// d > 1 within size classes of the extents); the bounds are computed from
// the coordinates, so any order gives a correct tree.
#include <cfloat>
#include <cmath>

#include "ddm_internal.cuh"

namespace ddm {
namespace {

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sorts the warp's 32 keys ascending (bitonic network over shuffles; ties by
// lane) and writes them and their prefix masks into one rank-table slot of
// kRankSlot words: slot[j] = the j-th smallest key, slot[35 + c] = the bits
// of the lanes holding the c smallest keys (c = 0..32; words 32..35 are 0).
__device__ __forceinline__ void rank_slot(float key, int lane, uint32_t* __restrict__ slot) {
  uint32_t idx = (uint32_t)lane;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const float ok = __shfl_xor_sync(0xffffffffu, key, j);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, idx, j);
      const bool mine_less = key < ok || (key == ok && idx < oi);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      if (keep_min != mine_less) {
        key = ok;
        idx = oi;
      }
    }
  }
  uint32_t m = 1u << idx;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, m, o);
    if (lane >= o) m |= y;
  }
  slot[lane] = __float_as_uint(key);
  slot[36 + lane] = m;
  if (lane < 4) slot[32 + lane] = 0u;
}

// Gather the sorted SoA layout and build levels 1 and 2.  One CTA of 1024
// threads covers 1024 sorted positions: one warp per level-1 node, and the
// CTA's 32 level-1 nodes form level-2 node blockIdx.x.  With `tab` (d <= 3)
// it also writes every leaf's rank tables: per dimension k, its 32 lower
// bounds (slot 2k) and 32 upper bounds (slot 2k + 1) sorted, with prefix
// masks, padding positions holding +inf.
__global__ void __launch_bounds__(1024)
k_gather_build(TreeView t, const uint32_t* __restrict__ sorted_ids, const float* __restrict__ lo,
               const float* __restrict__ hi, const float2* __restrict__ aos,
               float2* __restrict__ e, uint32_t* __restrict__ sid, float2* __restrict__ nodes,
               uint32_t* __restrict__ tab, Status* __restrict__ st) {
  __shared__ float s_min[DDM_MAX_DIMS][32], s_max[DDM_MAX_DIMS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t n = t.n;
  const uint32_t i = blockIdx.x * 1024u + threadIdx.x;
  const bool valid = i < n;
  uint32_t id = 0;
  bool valid_id = valid;
  if (valid) {
    id = sorted_ids[i];
    valid_id = DDM_IN_BOUNDS(id < n, st);
    if (!valid_id) id = 0;
    sid[i] = id;
  }
  const uint32_t g = blockIdx.x * 32u + w;
  const bool gvalid = g < t.cnt[1];
  for (int k = 0; k < t.d; ++k) {
    float a = FLT_MAX, b = -FLT_MAX;
    if (valid) {
      if (aos) {
        const float2 v = aos[(size_t)id * t.d + k];
        a = v.x;
        b = v.y;
      } else {
        a = lo[(size_t)k * n + id];
        b = hi[(size_t)k * n + id];
      }
      e[(size_t)k * n + i] = make_float2(a, b);
    }
    const float mn = warp_min(valid ? a : INFINITY);
    const float mx = warp_max(valid ? b : -INFINITY);
    if (tab && gvalid) {  // warp-uniform
      uint32_t* slot = tab + ((size_t)g * 2u * (uint32_t)t.d + 2u * (uint32_t)k) * kRankSlot;
      rank_slot(valid ? a : INFINITY, lane, slot);
      rank_slot(valid ? b : INFINITY, lane, slot + kRankSlot);
    }
    if (lane == 0) {
      if (gvalid) nodes[(size_t)k * t.total + t.off[1] + g] = make_float2(mn, mx);
      s_min[k][w] = gvalid ? mn : INFINITY;
      s_max[k][w] = gvalid ? mx : -INFINITY;
    }
  }
  if (t.L < 2) return;
  __syncthreads();
  if (w < t.d) {
    const float mn = warp_min(s_min[w][lane]);
    const float mx = warp_max(s_max[w][lane]);
    if (lane == 0) nodes[(size_t)w * t.total + t.off[2] + blockIdx.x] = make_float2(mn, mx);
  }
}

// Levels 3..L (at most n / 32768 nodes): one CTA walks up level by level.
__global__ void __launch_bounds__(1024) k_build_upper(TreeView t, float2* __restrict__ nodes) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l = 3; l <= t.L; ++l) {
    const uint32_t child_cnt = t.cnt[l - 1];
    for (uint32_t g = w; g < t.cnt[l]; g += 32) {
      const uint32_t c = g * 32u + lane;
      for (int k = 0; k < t.d; ++k) {
        const float2* child = nodes + (size_t)k * t.total + t.off[l - 1];
        const float2 v = c < child_cnt ? child[c] : make_float2(INFINITY, -INFINITY);
        const float mn = warp_min(v.x);
        const float mx = warp_max(v.y);
        if (lane == 0) nodes[(size_t)k * t.total + t.off[l] + g] = make_float2(mn, mx);
      }
    }
    __syncthreads();
  }
}

__global__ void k_export_nodes(const float2* __restrict__ nodes, size_t total,
                               float* __restrict__ node_lo, float* __restrict__ node_hi) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = nodes[i];
    if (node_lo) node_lo[i] = v.x;
    if (node_hi) node_hi[i] = v.y;
  }
}

}  // namespace

void tree_shape(uint32_t n, int* L, uint32_t* cnt, uint32_t* off, uint32_t* total) {
  for (int l = 0; l <= kMaxLevels; ++l) cnt[l] = off[l] = 0;
  int lv = 1;
  cnt[1] = (n + kFan - 1) / kFan;
  while (cnt[lv] > (uint32_t)kFan) {
    cnt[lv + 1] = (cnt[lv] + kFan - 1) / kFan;
    ++lv;
  }
  uint32_t acc = 0;
  for (int l = 1; l <= lv; ++l) {
    off[l] = acc;
    acc += cnt[l];
  }
  *L = lv;
  *total = acc;
}

// Group exponents of the per-dimension re-sorts (str_group_log2), kept
// strictly decreasing so that every re-sort refines the previous groups.
void str_groups(uint32_t n, int d, int* glog2, int shift) {
  for (int k = 0; k < DDM_MAX_DIMS; ++k) glog2[k] = 0;
  int prev = 64;
  for (int k = 1; k < d; ++k) {
    const int g = str_group_log2(n, d, k, shift);
    if (g > 0 && g < prev) {
      glog2[k] = g;
      prev = g;
    }
  }
}

cudaError_t launch_build(const TreeView& t, const uint32_t* sorted_ids, const float* lo,
                         const float* hi, const float2* aos, float2* e, uint32_t* sid,
                         float2* nodes, uint32_t* tab, Status* st, cudaStream_t s) {
  if (t.n == 0) return cudaSuccess;
  const uint32_t blocks = (t.n + 1023) / 1024;
  k_gather_build<<<blocks, 1024, 0, s>>>(t, sorted_ids, lo, hi, aos, e, sid, nodes, tab, st);
  if (t.L >= 3) k_build_upper<<<1, 1024, 0, s>>>(t, nodes);
  note_launches(t.L >= 3 ? 2u : 1u);
  return cudaGetLastError();
}

cudaError_t launch_export_nodes(const TreeView& t, float* node_lo, float* node_hi, cudaStream_t s) {
  const size_t total = (size_t)t.total * t.d;
  if (total == 0 || (!node_lo && !node_hi)) return cudaSuccess;
  const size_t blocks = (total + 255) / 256;
  k_export_nodes<<<blocks < 1024 ? (unsigned)blocks : 1024u, 256, 0, s>>>(t.nodes, total, node_lo,
                                                                       node_hi);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ddm
