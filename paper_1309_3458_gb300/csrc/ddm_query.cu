// Interval-Query (Alg. 4) for every update extent: warp-cooperative tree
// walk over packets of 32 queries.
//
// The paper's query descends only into subtrees that can hold a match: it
// prunes when maxupper < q.lower or minlower > q.upper and otherwise visits
// the children in order, testing each stored interval with Intersect-1D
// (Alg. 1).  Queries are independent (Section IV, "Parallelizing ITM"), so
// the GPU runs 32 of them per warp:
//
//   * the updates are sorted with the same spatial order as the tree (see
//     ddm_layout.cu), so the 32 queries of a packet lie close together;
//   * the warp walks the flattened 32-ary tree depth-first with the packet's
//     bounding box: one lane per child, one coalesced load of the children's
//     per-dimension (minlower, maxupper), one ballot, a 32-bit mask of
//     surviving children per level;
//   * at a leaf (32 consecutive subscriptions) the packet's queries whose own
//     box meets the leaf's box are tested one after the other: every lane
//     holds one subscription and applies the segment test of Alg. 1 in every
//     dimension (the reduction of Section III-A), and a ballot yields that
//     query's matches in the leaf.
//
// The count pass adds up matches per update; the write pass stores
// (update, subscription) pairs from each update's output offset.  Both walk
// the same leaves in the same order, so the write pass reproduces the
// counted pairs exactly, in tree order.  Predicates are combined with
// bitwise ANDs so the per-query test has no branches.
#include <cfloat>

#include "ddm_internal.cuh"

namespace ddm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <bool OPEN>
__device__ __forceinline__ bool le(float a, float b) {
  return OPEN ? (a < b) : (a <= b);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

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

// D > 0: compile-time dimension count; D == 0: runtime d (up to 8).
template <int D, bool OPEN, bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_packets(TreeView t, QueryView q, uint32_t* __restrict__ counts, uint32_t* __restrict__ counts_pos,
          WriteView w, uint32_t* __restrict__ work, Status* __restrict__ st) {
  constexpr int DM = D > 0 ? D : DDM_MAX_DIMS;
  const int d = D > 0 ? D : t.d;
  __shared__ float2 s_q[kWarps][DM][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const size_t n = t.n, total = t.total, m = q.m;

  unsigned long long base0 = 0;
  if (WRITE) {
    base0 = w.start[w.b_idx];
    const unsigned long long need = w.start[w.e_idx] - base0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->K = need;
      if (need > w.capacity) atomicOr(&st->err, kErrCapacity);
    }
    if (need > w.capacity) return;
  }

  const uint32_t npk = (q.nq + 31u) >> 5;
  for (;;) {
    uint32_t p = 0;
    if (lane == 0) p = atomicAdd(work, 1u);
    p = __shfl_sync(0xffffffffu, p, 0);
    if (p >= npk) break;

    // ---- the packet: up to 32 queries, one per lane ----
    const uint32_t idx = p * 32u + lane;
    const bool valid = idx < q.nq;
    uint32_t pos = 0, Q = 0;
    if (valid) {
      pos = q.list ? q.list[idx] : q.first + idx;
      Q = q.qid[pos];
    }
    float ql[DM], qh[DM], gl[DM], gh[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
      if (k < d) {
        const float2 v = valid ? q.qe[k * m + pos] : make_float2(INFINITY, -INFINITY);
        ql[k] = v.x;
        qh[k] = v.y;
        s_q[wib][k][lane] = v;
        gl[k] = warp_min(v.x);  // packet bounding box
        gh[k] = warp_max(v.y);
      }
    }
    uint32_t cnt = 0;
    unsigned long long out = 0;
    if (WRITE && valid) out = w.start[w.by_pos ? pos : Q] - base0;
    __syncwarp();

    // Test the 32 level-1 nodes (leaves) from g1 on against the packet box,
    // then run the packet's queries over each surviving leaf.
    auto leaves = [&](uint32_t g1) {
      const uint32_t c = g1 + lane;
      const bool cv = c < t.cnt[1];
      float bl[DM], bh[DM];
      bool ok = cv;
#pragma unroll
      for (int k = 0; k < DM; ++k) {
        if (k < d) {
          const float2 v = cv ? t.nodes[k * total + t.off[1] + c] : make_float2(INFINITY, -INFINITY);
          bl[k] = v.x;
          bh[k] = v.y;
          ok = ok & le<OPEN>(v.x, gh[k]) & le<OPEN>(gl[k], v.y);
        }
      }
      uint32_t lm = __ballot_sync(0xffffffffu, ok);
      while (lm) {
        const int cl = __ffs(lm) - 1;
        lm &= lm - 1u;
        // queries of the packet whose box meets this leaf's box
        bool qok = valid;
#pragma unroll
        for (int k = 0; k < DM; ++k) {
          if (k < d) {
            const float a = __shfl_sync(0xffffffffu, bl[k], cl);
            const float b = __shfl_sync(0xffffffffu, bh[k], cl);
            qok = qok & le<OPEN>(a, qh[k]) & le<OPEN>(ql[k], b);
          }
        }
        uint32_t qm = __ballot_sync(0xffffffffu, qok);
        if (qm == 0u) continue;
        const uint32_t i = (g1 + cl) * 32u + lane;
        const bool iv = i < n;
        float2 ev[DM];
#pragma unroll
        for (int k = 0; k < DM; ++k)
          if (k < d) ev[k] = iv ? t.e[k * n + i] : make_float2(INFINITY, -INFINITY);
        uint32_t my_sid = 0;
        if (WRITE && iv) my_sid = t.sid[i];
        while (qm) {
          const int qq = __ffs(qm) - 1;
          qm &= qm - 1u;
          bool hit = iv;
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            if (k < d) {
              const float2 b = s_q[wib][k][qq];
              hit = hit & le<OPEN>(ev[k].x, b.y) & le<OPEN>(b.x, ev[k].y);
            }
          }
          const uint32_t hb = __ballot_sync(0xffffffffu, hit);
          if (WRITE) {
            const unsigned long long o = __shfl_sync(0xffffffffu, out, qq);
            const uint32_t Qq = __shfl_sync(0xffffffffu, Q, qq);
            if (hit) {
              const unsigned long long at = o + __popc(hb & lt);
              if (at < w.capacity) {
                ddm_pair pr;
                pr.upd = Qq;
                pr.sub = my_sid;
                w.pairs[at] = pr;
              }
            }
            if (lane == qq) out = o + __popc(hb);
          } else {
            if (lane == qq) cnt += __popc(hb);
          }
        }
      }
    };

    if (t.L == 1) {
      leaves(0);
    } else {
      // Depth-first walk over levels L..2; mask[l] holds the surviving, not
      // yet visited nodes among the 32 level-l nodes starting at base[l].
      uint32_t mask[kMaxLevels + 1], base[kMaxLevels + 1];
      int lvl = t.L;
      {
        const bool cv = (uint32_t)lane < t.cnt[lvl];
        bool ok = cv;
#pragma unroll
        for (int k = 0; k < DM; ++k) {
          if (k < d) {
            const float2 v = cv ? t.nodes[k * total + t.off[lvl] + lane]
                                : make_float2(INFINITY, -INFINITY);
            ok = ok & le<OPEN>(v.x, gh[k]) & le<OPEN>(gl[k], v.y);
          }
        }
        mask[lvl] = __ballot_sync(0xffffffffu, ok);
        base[lvl] = 0;
      }
      for (;;) {
        const uint32_t mk = mask[lvl];
        if (mk == 0u) {
          if (lvl == t.L) break;
          ++lvl;
          continue;
        }
        mask[lvl] = mk & (mk - 1u);
        const uint32_t g = base[lvl] + (uint32_t)(__ffs(mk) - 1);
        if (lvl == 2) {
          leaves(g * 32u);
        } else {
          const uint32_t ch = g * 32u + lane;
          const bool cv = ch < t.cnt[lvl - 1];
          bool ok = cv;
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            if (k < d) {
              const float2 v = cv ? t.nodes[k * total + t.off[lvl - 1] + ch]
                                  : make_float2(INFINITY, -INFINITY);
              ok = ok & le<OPEN>(v.x, gh[k]) & le<OPEN>(gl[k], v.y);
            }
          }
          --lvl;
          mask[lvl] = __ballot_sync(0xffffffffu, ok);
          base[lvl] = g * 32u;
        }
      }
    }
    if (!WRITE && valid) {
      counts[Q] = cnt;
      if (counts_pos) counts_pos[pos] = cnt;
    }
  }
}

template <bool WRITE>
cudaError_t launch_packets(const TreeView& t, const QueryView& q, uint32_t flags, uint32_t* counts,
                           uint32_t* counts_pos, const WriteView& w, uint32_t* work, Status* st,
                           int sms, cudaStream_t s) {
  if (q.nq == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
  if (e) return e;
  const bool open = (flags & DDM_OPEN) != 0;
  const uint32_t packets = (q.nq + 31) / 32;
  uint32_t blocks = (packets + kWarps - 1) / kWarps;
  const uint32_t cap = (uint32_t)sms * 8u;
  if (blocks > cap) blocks = cap;
#define DDM_LAUNCH(DD, OP) \
  k_packets<DD, OP, WRITE><<<blocks, kThreads, 0, s>>>(t, q, counts, counts_pos, w, work, st)
  switch (t.d) {
    case 1: open ? DDM_LAUNCH(1, true) : DDM_LAUNCH(1, false); break;
    case 2: open ? DDM_LAUNCH(2, true) : DDM_LAUNCH(2, false); break;
    case 3: open ? DDM_LAUNCH(3, true) : DDM_LAUNCH(3, false); break;
    default: open ? DDM_LAUNCH(0, true) : DDM_LAUNCH(0, false); break;
  }
#undef DDM_LAUNCH
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_count(const TreeView& t, const QueryView& q, uint32_t flags, uint32_t* counts,
                         uint32_t* counts_pos, uint32_t* work, int sms, cudaStream_t s) {
  WriteView w{};
  return launch_packets<false>(t, q, flags, counts, counts_pos, w, work, nullptr, sms, s);
}

cudaError_t launch_write(const TreeView& t, const QueryView& q, uint32_t flags, const WriteView& w,
                         uint32_t* work, Status* st, int sms, cudaStream_t s) {
  return launch_packets<true>(t, q, flags, nullptr, nullptr, w, work, st, sms, s);
}

}  // namespace ddm
