// Input validation, sort keys and gathers of the structure-of-arrays layout.
//
// Every extent must have lo <= hi with no NaN in every dimension (the
// paper's segments [low, high], Section III-A); a violation raises
// kErrExtent.  For the subscription set of a d = 1 tree the same pass emits
// the 64-bit sort key of the interval tree order of Section IV -- lower
// bound, ties broken by upper bound -- as (key(lo0) << 32 | key(hi0)), and
// the identity id payload, so a stable radix sort leaves remaining ties in id
// order.  Every other order (d > 1 trees, the updates) is a locality order:
// its keys hold the top 24 bits of key(lo) below a class, group or instance.
//
// For d > 1 the order is then refined one dimension at a time: inside
// aligned groups of consecutive positions the extents are re-sorted by their
// lower bound in the next dimension (k_rekey builds (group, key(lo_k))
// keys).  Each group stays a contiguous range of the dimension-0 order, so
// the top of the tree still follows the paper's lower-bound order, while the
// small subtrees near the leaves become compact in every dimension.  For the
// tree with d > 1 the subscriptions are first grouped by size class
// (k_validate_class: class, then lower bound), and every class is refined
// with groups sized for it (k_batch_groups / k_rekey_batch, the machinery of
// batched sets with the classes as instances).
#include "ddm_internal.cuh"

namespace ddm {
namespace {

constexpr int kThreads = 256;
// Locality keys (every sort but the d = 1 tree's): the top 24 bits of the
// order-preserving float key -- sign, exponent and 15 mantissa bits, about
// 3e-5 relative -- below a group / class / instance number.  Such an order
// is a heuristic (any order gives the same pairs), and dropping the low
// byte saves one radix pass per sort.
constexpr int kLocalityBits = 24;
constexpr int kLocalityDrop = 32 - kLocalityBits;

__global__ void __launch_bounds__(kThreads)
k_validate(int d, const float* __restrict__ lo, const float* __restrict__ hi, uint32_t cnt,
           unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals, int key_mode,
           float2* __restrict__ aos, Status* __restrict__ st) {
  bool bad = false;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    // Row loads are coalesced: consecutive lanes read consecutive floats.
    for (int k = 0; k < d; ++k) {
      const float a = __ldg(lo + (size_t)k * cnt + i);
      const float b = __ldg(hi + (size_t)k * cnt + i);
      bad |= !(a <= b);  // false for NaN as well as for lo > hi
      if (aos) aos[(size_t)i * d + k] = make_float2(a, b);
    }
    if (keys) {
      const float a = __ldg(lo + i), b = __ldg(hi + i);
      keys[i] = key_mode == 1 ? ((unsigned long long)float_key(a) << 32) | float_key(b)
                              : (unsigned long long)(float_key(a) >> kLocalityDrop);
      vals[i] = i;
    }
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->err, kErrExtent);
}

__global__ void __launch_bounds__(kThreads)
k_rekey(const uint32_t* __restrict__ vals, const float* __restrict__ lo_k, uint32_t cnt, int glog2,
        unsigned long long* __restrict__ keys) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride)
    keys[i] = ((unsigned long long)(i >> glog2) << kLocalityBits) |
              (float_key(__ldg(lo_k + vals[i])) >> kLocalityDrop);
}

__global__ void __launch_bounds__(kThreads)
k_gather(int d, const uint32_t* __restrict__ vals, const float* __restrict__ lo,
         const float* __restrict__ hi, const float2* __restrict__ aos, uint32_t cnt,
         float2* __restrict__ qe, uint32_t* __restrict__ qid) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    const uint32_t id = vals[i];
    qid[i] = id;
    for (int k = 0; k < d; ++k)
      qe[(size_t)k * cnt + i] = aos ? aos[(size_t)id * d + k]
                                    : make_float2(__ldg(lo + (size_t)k * cnt + id),
                                                  __ldg(hi + (size_t)k * cnt + id));
  }
}

// Validation plus the first sort key of the tree order for d >= 2: the size
// class of the extent -- the binary exponent of its largest side (the float
// exponent field) -- then the dimension-0 lower bound and, in the low 24
// bits, the top of the upper bound.  Sorting by class first keeps extents of
// similar size together, so that one long extent does not widen the boxes
// of a leaf of short ones; the order is a heuristic (node bounds come from
// the coordinates whatever the order).  hist[class] counts the extents.
__global__ void __launch_bounds__(kThreads)
k_validate_class(int d, const float* __restrict__ lo, const float* __restrict__ hi, uint32_t cnt,
                 unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals,
                 uint32_t* __restrict__ hist, float2* __restrict__ aos, Status* __restrict__ st) {
  __shared__ uint32_t s_h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_h[i] = 0u;
  __syncthreads();
  bool bad = false;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    float side = 0.0f;
    for (int k = 0; k < d; ++k) {
      const float a = __ldg(lo + (size_t)k * cnt + i);
      const float b = __ldg(hi + (size_t)k * cnt + i);
      bad |= !(a <= b);
      side = fmaxf(side, b - a);
      if (aos) aos[(size_t)i * d + k] = make_float2(a, b);
    }
    const uint32_t cls = (__float_as_uint(side) >> 23) & 0xffu;
    keys[i] = ((unsigned long long)cls << kLocalityBits) |
              (float_key(__ldg(lo + i)) >> kLocalityDrop);
    vals[i] = i;
    atomicAdd(&s_h[cls], 1u);
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->err, kErrExtent);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

// Instance (batched set, or size class) of every position: the b with
// off[b] <= i < off[b+1], by binary search over the offsets, so that one
// very large instance is filled by the whole grid.
__global__ void __launch_bounds__(kThreads)
k_fill_inst(const unsigned long long* __restrict__ off, uint32_t count, uint32_t total,
            uint32_t* __restrict__ inst) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    uint32_t lo = 0, hi = count;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (off[mid] <= i) lo = mid; else hi = mid;
    }
    inst[i] = lo;
  }
}

__global__ void __launch_bounds__(kThreads)
k_validate_batch(int d, const float* __restrict__ lo, const float* __restrict__ hi, uint32_t cnt,
                 const uint32_t* __restrict__ inst, unsigned long long* __restrict__ keys,
                 uint32_t* __restrict__ vals, float2* __restrict__ aos, Status* __restrict__ st) {
  bool bad = false;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    for (int k = 0; k < d; ++k) {
      const float a = __ldg(lo + (size_t)k * cnt + i);
      const float b = __ldg(hi + (size_t)k * cnt + i);
      bad |= !(a <= b);
      if (aos) aos[(size_t)i * d + k] = make_float2(a, b);
    }
    keys[i] = ((unsigned long long)inst[i] << kLocalityBits) |
              (float_key(__ldg(lo + i)) >> kLocalityDrop);
    vals[i] = i;
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->err, kErrExtent);
}

__global__ void k_batch_groups(const unsigned long long* __restrict__ off, uint32_t count, int d,
                               int k, int shift, int* __restrict__ glog2,
                               uint32_t* __restrict__ ngroups) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t n = (uint32_t)(off[i + 1] - off[i]);
    // strictly smaller than the previous dimension's groups, as in str_groups
    int g = str_group_log2(n, d, k, shift);
    for (int j = 1; j < k && g > 0; ++j) {
      const int gp = str_group_log2(n, d, j, shift);
      if (gp > 0 && g >= gp) g = 0;
    }
    glog2[i] = g;
    // g == 0 (no re-sort): the whole instance is one group whose keys are
    // all equal, so the stable sort keeps it in place.  With g >= 6 every
    // instance has at most n / 64 + 1 groups.
    ngroups[i] = g > 0 ? ((n + (1u << g) - 1) >> g) : (n > 0 ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(kThreads)
k_rekey_batch(const uint32_t* __restrict__ vals, const float* __restrict__ lo_k, uint32_t cnt,
              const uint32_t* __restrict__ inst, const unsigned long long* __restrict__ off,
              const int* __restrict__ glog2, const unsigned long long* __restrict__ gbase,
              unsigned long long* __restrict__ keys) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    const uint32_t b = inst[i];
    const int g = glog2[b];
    if (g == 0) {  // one group, equal keys: the instance keeps its order
      keys[i] = gbase[b] << kLocalityBits;
      continue;
    }
    const unsigned long long local = i - off[b];
    const unsigned long long group = gbase[b] + (local >> g);
    keys[i] = (group << kLocalityBits) | (float_key(__ldg(lo_k + vals[i])) >> kLocalityDrop);
  }
}

uint32_t grid_for(uint32_t cnt, int sms) {
  uint32_t blocks = (cnt + kThreads - 1) / kThreads;
  const uint32_t cap = (uint32_t)sms * 8u;
  return blocks > cap ? cap : (blocks ? blocks : 1);
}

}  // namespace

cudaError_t launch_rekey(const uint32_t* vals, const float* lo_k, uint32_t cnt, int glog2,
                         unsigned long long* keys, int sms, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_rekey<<<grid_for(cnt, sms), kThreads, 0, s>>>(vals, lo_k, cnt, glog2, keys);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather(int d, const uint32_t* vals, const float* lo, const float* hi,
                          const float2* aos, uint32_t cnt, float2* qe, uint32_t* qid, int sms,
                          cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_gather<<<grid_for(cnt, sms), kThreads, 0, s>>>(d, vals, lo, hi, aos, cnt, qe, qid);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_validate_class(int d, const float* lo, const float* hi, uint32_t cnt,
                                  unsigned long long* keys, uint32_t* vals, uint32_t* hist,
                                  float2* aos, Status* st, int sms, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_validate_class<<<grid_for(cnt, sms), kThreads, 0, s>>>(d, lo, hi, cnt, keys, vals, hist, aos,
                                                           st);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill_inst(const unsigned long long* off, uint32_t count, uint32_t total,
                             uint32_t* inst, int sms, cudaStream_t s) {
  if (count == 0 || total == 0) return cudaSuccess;
  k_fill_inst<<<grid_for(total, sms), kThreads, 0, s>>>(off, count, total, inst);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_validate_batch(int d, const float* lo, const float* hi, uint32_t cnt,
                                  const uint32_t* inst, unsigned long long* keys, uint32_t* vals,
                                  float2* aos, Status* st, int sms, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_validate_batch<<<grid_for(cnt, sms), kThreads, 0, s>>>(d, lo, hi, cnt, inst, keys, vals, aos,
                                                           st);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_groups(const unsigned long long* off, uint32_t count, int d, int k,
                                int shift, int* glog2, uint32_t* ngroups, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t blocks = (count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024;
  k_batch_groups<<<blocks, 256, 0, s>>>(off, count, d, k, shift, glog2, ngroups);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rekey_batch(const uint32_t* vals, const float* lo_k, uint32_t cnt,
                               const uint32_t* inst, const unsigned long long* off,
                               const int* glog2, const unsigned long long* gbase,
                               unsigned long long* keys, int sms, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_rekey_batch<<<grid_for(cnt, sms), kThreads, 0, s>>>(vals, lo_k, cnt, inst, off, glog2, gbase,
                                                        keys);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_validate(int d, const float* lo, const float* hi, uint32_t cnt,
                            unsigned long long* keys, uint32_t* vals, int key_mode, float2* aos,
                            Status* st, int sms, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  k_validate<<<grid_for(cnt, sms), kThreads, 0, s>>>(d, lo, hi, cnt, keys, vals, key_mode, aos,
                                                     st);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ddm
