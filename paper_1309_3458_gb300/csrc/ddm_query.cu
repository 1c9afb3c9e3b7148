// Interval-Query (Alg. 4) for every update extent: warp-cooperative tree
// walk over packets of 32 queries.
//
// The paper's query descends only into subtrees that can hold a match: it
// prunes when maxupper < q.lower or minlower > q.upper and otherwise visits
// the children in order, testing each stored interval with Intersect-1D
// (Alg. 1).  Queries are independent (Section IV, "Parallelizing ITM"), so
// the GPU runs 32 of them per warp:
//
//   * the updates are sorted by lower bound with the same sort-tile-recursive
//     refinement as the tree (ddm_api.cu, order_set; the tree's size classes
//     are not applied to queries), so the 32 queries of a packet lie close
//     together;
//   * the warp walks the flattened 32-ary tree depth-first with the packet's
//     bounding box: one lane per child, one coalesced load of the children's
//     per-dimension (minlower, maxupper), one ballot, a 32-bit mask of
//     surviving children per level;
//   * at a leaf (32 consecutive subscriptions) the packet's queries whose own
//     box meets the leaf's box are tested one after the other: every lane
//     holds one subscription and applies the segment test of Alg. 1 in every
//     dimension (the reduction of Section III-A), and a ballot yields that
//     query's matches in the leaf; when many of them meet the leaf, the
//     roles swap (lane = query): for d <= 3 each lane finds its query's
//     matches from the leaf's rank tables -- per dimension the leaf's lower
//     and upper bounds sorted, with the mask of positions holding the c
//     smallest -- by one binary search per bound, the same set as the
//     segment tests since {lo_k <= q.hi_k} is a prefix of the sorted lower
//     bounds and {hi_k >= q.lo_k} the complement of a prefix of the sorted
//     upper bounds; for d > 3 by a loop over the leaf's subscriptions.
//
// The count pass adds up matches per update and leaves replay records; the
// write pass (k_replay) expands the records into (update, subscription)
// pairs from each update's output offset, or, if the record arena ran out,
// walks the tree again (k_packets with WRITE), visiting the same leaves in
// the same order -- either way the pairs come out exactly as counted, in
// tree order.  The write pass can also store only each pair's subscription
// id (the compressed form of the intersection matrix, Section III), or the
// pairs with their fields exchanged when the roles are swapped.  For d <= 3
// the count pass's leaf tests are hand-written PTX: the 2d segment
// comparisons chain one predicate (setp with .and) into a vote or a
// predicated or, with no branch and no integer form of the predicate; other
// paths combine the comparisons with bitwise ANDs, also without branches.
#include <cfloat>
#include <type_traits>

#include "ddm_internal.cuh"

namespace ddm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Without rank tables (d > 3, or no room for them) the swapped leaf test
// compares the leaf's 32 subscriptions one by one, which pays only from about
// this many queries on a leaf.
constexpr uint32_t kCompareSwapMin = 24;
// Resident 256-thread blocks per SM the packet kernels are compiled for.
#ifndef DDM_PACKET_MIN_BLOCKS
#define DDM_PACKET_MIN_BLOCKS 4
#endif

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

// Ballot of the d-dimensional segment test (Alg. 1 in every dimension,
// Section III-A) of this lane's subscription e against one query, for
// d = 1..3: one predicate chained through 2d compare-and-accumulate setp
// instructions and one vote, with no integer form of the predicate.  b0 / b1
// hold the query's (lo, hi) pairs of dimensions (0, 1) and 2.  A padding lane
// carries NaN bounds, which fail every comparison.
#define DDM_SEG_BALLOT(CMP)                                                              \
  template <int D>                                                                        \
  __device__ __forceinline__ uint32_t seg_ballot_##CMP(const float2* e, float4 b0, float4 b1) { \
    uint32_t hb;                                                                          \
    if (D == 1) {                                                                         \
      asm("{\n\t.reg .pred p;\n\t"                                                       \
          "setp." #CMP ".f32 p, %1, %2;\n\t"                                              \
          "setp." #CMP ".and.f32 p, %3, %4, p;\n\t"                                       \
          "vote.sync.ballot.b32 %0, p, 0xffffffff;\n\t}"                                  \
          : "=r"(hb) : "f"(e[0].x), "f"(b0.y), "f"(b0.x), "f"(e[0].y));                   \
    } else if (D == 2) {                                                                  \
      asm("{\n\t.reg .pred p;\n\t"                                                       \
          "setp." #CMP ".f32 p, %1, %2;\n\t"                                              \
          "setp." #CMP ".and.f32 p, %3, %4, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %5, %6, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %7, %8, p;\n\t"                                       \
          "vote.sync.ballot.b32 %0, p, 0xffffffff;\n\t}"                                  \
          : "=r"(hb) : "f"(e[0].x), "f"(b0.y), "f"(b0.x), "f"(e[0].y),                    \
            "f"(e[1].x), "f"(b0.w), "f"(b0.z), "f"(e[1].y));                               \
    } else {                                                                              \
      asm("{\n\t.reg .pred p;\n\t"                                                       \
          "setp." #CMP ".f32 p, %1, %2;\n\t"                                              \
          "setp." #CMP ".and.f32 p, %3, %4, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %5, %6, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %7, %8, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %9, %10, p;\n\t"                                      \
          "setp." #CMP ".and.f32 p, %11, %12, p;\n\t"                                     \
          "vote.sync.ballot.b32 %0, p, 0xffffffff;\n\t}"                                  \
          : "=r"(hb) : "f"(e[0].x), "f"(b0.y), "f"(b0.x), "f"(e[0].y),                    \
            "f"(e[1].x), "f"(b0.w), "f"(b0.z), "f"(e[1].y),                               \
            "f"(e[2].x), "f"(b1.y), "f"(b1.x), "f"(e[2].y));                               \
    }                                                                                     \
    return hb;                                                                            \
  }
DDM_SEG_BALLOT(le)  // closed segments
DDM_SEG_BALLOT(lt)  // the strict test of Alg. 1
#undef DDM_SEG_BALLOT

// The same test with the roles swapped (lane = query, one subscription b of
// the leaf broadcast from shared memory, for d = 1..3): `bit` is or-ed into
// acc when the lane's query [ql, qh] meets b in every dimension.
#define DDM_SEG_OR(CMP)                                                                    \
  template <int D>                                                                          \
  __device__ __forceinline__ void seg_or_##CMP(uint32_t& acc, uint32_t bit, float4 b0,      \
                                               float4 b1, const float* ql, const float* qh) { \
    if (D == 1) {                                                                           \
      asm("{\n\t.reg .pred p;\n\t"                                                         \
          "setp." #CMP ".f32 p, %2, %3;\n\t"                                                \
          "setp." #CMP ".and.f32 p, %4, %5, p;\n\t"                                         \
          "@p or.b32 %0, %0, %1;\n\t}"                                                      \
          : "+r"(acc) : "r"(bit), "f"(b0.x), "f"(qh[0]), "f"(ql[0]), "f"(b0.y));            \
    } else if (D == 2) {                                                                    \
      asm("{\n\t.reg .pred p;\n\t"                                                         \
          "setp." #CMP ".f32 p, %2, %3;\n\t"                                                \
          "setp." #CMP ".and.f32 p, %4, %5, p;\n\t"                                         \
          "setp." #CMP ".and.f32 p, %6, %7, p;\n\t"                                         \
          "setp." #CMP ".and.f32 p, %8, %9, p;\n\t"                                         \
          "@p or.b32 %0, %0, %1;\n\t}"                                                      \
          : "+r"(acc) : "r"(bit), "f"(b0.x), "f"(qh[0]), "f"(ql[0]), "f"(b0.y),             \
            "f"(b0.z), "f"(qh[1]), "f"(ql[1]), "f"(b0.w));                                  \
    } else {                                                                                \
      asm("{\n\t.reg .pred p;\n\t"                                                         \
          "setp." #CMP ".f32 p, %2, %3;\n\t"                                                \
          "setp." #CMP ".and.f32 p, %4, %5, p;\n\t"                                         \
          "setp." #CMP ".and.f32 p, %6, %7, p;\n\t"                                         \
          "setp." #CMP ".and.f32 p, %8, %9, p;\n\t"                                         \
          "setp." #CMP ".and.f32 p, %10, %11, p;\n\t"                                       \
          "setp." #CMP ".and.f32 p, %12, %13, p;\n\t"                                       \
          "@p or.b32 %0, %0, %1;\n\t}"                                                      \
          : "+r"(acc) : "r"(bit), "f"(b0.x), "f"(qh[0]), "f"(ql[0]), "f"(b0.y),             \
            "f"(b0.z), "f"(qh[1]), "f"(ql[1]), "f"(b0.w),                                    \
            "f"(b1.x), "f"(qh[2]), "f"(ql[2]), "f"(b1.y));                                   \
    }                                                                                       \
  }
DDM_SEG_OR(le)
DDM_SEG_OR(lt)
#undef DDM_SEG_OR

// D > 0: compile-time dimension count; D == 0: runtime d (up to 8).
// BATCH: every query matches only its instance's subscription positions, and
// pairs carry instance-local ids.
template <int D, bool OPEN, bool WRITE, bool BATCH>
__global__ void __launch_bounds__(kThreads, DDM_PACKET_MIN_BLOCKS)
k_packets(TreeView t, QueryView q, BatchView bv, uint32_t* __restrict__ counts,
          uint32_t* __restrict__ counts_pos, RecordArena ra, WriteView w,
          uint32_t* __restrict__ work, Status* __restrict__ st) {
  constexpr int DM = D > 0 ? D : DDM_MAX_DIMS;
  constexpr int DP = (DM + 1) / 2;  // dimension pairs: one 128-bit shared load each
  // Per query a row of RW float4: its bounds, dimension pairs first, and one
  // word for its hit mask in the leaf being tested (in the unused half of the
  // last pair for odd DM, else in a float4 of its own).
  constexpr int RW = (DM & 1) ? DP : DP + 1;
  constexpr int HB = (DM & 1) ? 4 * (DP - 1) + 2 : 4 * DP;  // hit-mask word within a row
  const int d = D > 0 ? D : t.d;
  __shared__ float4 s_q[kWarps][32][RW];
  __shared__ uint32_t s_list[WRITE ? 1 : kWarps][32];  // count pass: rows of a leaf's queries
  __shared__ float4 s_e[WRITE ? 1 : kWarps][32][DP];  // count pass: a leaf's subscriptions
  // count pass, d <= 3: a leaf's rank tables (2d slots of kRankSlot words)
  constexpr int TW = (!WRITE && D >= 1 && D <= 3) ? 2 * D * (int)kRankSlot : 4;
  __shared__ __align__(16) uint32_t s_tab[kWarps][TW];
  __shared__ uint2 s_rng[kWarps][BATCH ? 32 : 1];  // per query: its instance's positions
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const size_t n = t.n, total = t.total, m = q.m;

  unsigned long long base0 = 0;
  if (WRITE) {
    if (records_complete(ra)) return;  // the replay kernel writes this range
    base0 = w.start[w.b_idx];
    const unsigned long long need = w.start[w.e_idx] - base0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->K = need;
      if (need > w.capacity) atomicOr(&st->err, kErrCapacity);
    }
    if (need > w.capacity) return;
  }

  const uint32_t qpp = 1u << q.qpp_log2;  // queries per packet: 16 or 32
  const uint32_t npk = (q.nq + qpp - 1u) >> q.qpp_log2;
  for (;;) {
    uint32_t p = 0;
    if (lane == 0) p = atomicAdd(work, 1u);
    p = __shfl_sync(0xffffffffu, p, 0);
    if (p >= npk) break;

    // ---- the packet: up to qpp queries, one per lane ----
    const uint32_t idx = (p << q.qpp_log2) + lane;
    const bool valid = (uint32_t)lane < qpp && idx < q.nq;
    uint32_t pos = 0, Q = 0;
    if (valid) {
      pos = q.list ? q.list[idx] : q.first + idx;
      Q = q.qid[pos];
    }
    // Position range of the subscriptions this query may match, and the
    // update id written into pairs (instance-local when batched).
    uint32_t r_lo = 0, r_hi = (uint32_t)n, Qout = WRITE ? Q + w.qbase : Q;
    if (WRITE && w.qids && valid) Qout = w.qids[Q];
    if (BATCH && valid) {
      const uint32_t b = bv.q_inst[pos];
      r_lo = (uint32_t)bv.sub_off[b];
      r_hi = (uint32_t)bv.sub_off[b + 1];
      Qout = Q - (uint32_t)bv.upd_off[b];
    }
    uint32_t g_lo = 0, g_hi = (uint32_t)n;  // union of the packet's ranges
    if (BATCH) {
      g_lo = __reduce_min_sync(0xffffffffu, valid ? r_lo : 0xffffffffu);
      g_hi = __reduce_max_sync(0xffffffffu, valid ? r_hi : 0u);
      s_rng[wib][lane] = make_uint2(r_lo, r_hi);
    }
    float ql[DM], qh[DM], gl[DM], gh[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
      if (k < d) {
        const float2 v = valid ? q.qe[k * m + pos] : make_float2(INFINITY, -INFINITY);
        ql[k] = v.x;
        qh[k] = v.y;
        gl[k] = warp_min(v.x);  // packet bounding box
        gh[k] = warp_max(v.y);
      }
    }
#pragma unroll
    for (int k2 = 0; k2 < DP; ++k2) {
      const int a = 2 * k2, b = 2 * k2 + 1;
      if (a < d)
        s_q[wib][lane][k2] = make_float4(ql[a], qh[a], b < d ? ql[b] : 0.f, b < d ? qh[b] : 0.f);
    }
    uint32_t cnt = 0, ntests = 0;
    unsigned long long out = 0;
    if (WRITE && valid) out = w.start[w.by_pos ? pos : Q] - base0;
    __syncwarp();

    // Records of the count pass: one per (query, leaf) with hits, written
    // leaf by leaf with one coalesced store.  After the arena runs out the
    // packet stops writing but keeps counting the blocks it would need.
    const bool recording = !WRITE && ra.max_blocks > 0;
    bool rec_write = recording;
    uint32_t cur0 = kNoBlock, cur1 = kNoBlock, fill0 = kRecBlock, fill1 = kRecBlock;
    uint32_t nblk0 = 0, nblk1 = 0;
    uint32_t blk_cnt = 0;  // this query's matches before its chain's current block
    // Test the 32 level-1 nodes (leaves) from g1 on against the packet box,
    // then run the packet's queries over each surviving leaf.
    auto leaves = [&](uint32_t g1) {
      const uint32_t c = g1 + lane;
      const bool cv = c < t.cnt[1];
      float bl[DM], bh[DM];
      bool ok = cv;
      if (BATCH) ok = ok && c * 32u < g_hi && c * 32u + 32u > g_lo;
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
        if (BATCH) qok = qok && (g1 + cl) * 32u < r_hi && (g1 + cl) * 32u + 32u > r_lo;
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
        if (!WRITE) ntests += __popc(qm);
        const uint32_t i = (g1 + cl) * 32u + lane;
        const bool iv = i < n;
        uint32_t my_hb = 0;  // count pass: this lane's query's hit mask in the leaf
        bool by_rank = false;
        if constexpr (!WRITE && D >= 1 && D <= 3) by_rank = t.tab && __popc(qm) >= q.tmin;
        if (by_rank) {
          // Rank tables (lane = query): per dimension k, the leaf positions
          // with lo_k <= q.hi_k are those of the c smallest lower bounds, c
          // found by a 6-step search in the sorted bounds; those with
          // hi_k >= q.lo_k are all but the c' smallest upper bounds below
          // q.lo_k.  The hit mask is their intersection over the dimensions:
          // the segment test of Alg. 1 in every dimension (Section III-A),
          // for all 32 subscriptions at once.
          const float4* src = reinterpret_cast<const float4*>(
              t.tab + (size_t)(g1 + cl) * (2u * D) * kRankSlot);
          float4* dst = reinterpret_cast<float4*>(&s_tab[wib][0]);
          constexpr int NV = 2 * D * (int)kRankSlot / 4;
#pragma unroll
          for (int j = lane; j < NV; j += 32) dst[j] = __ldg(src + j);
          __syncwarp();
          uint32_t hbm = __ballot_sync(0xffffffffu, iv);  // padding positions of the last leaf
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const uint32_t* sl = &s_tab[wib][2 * k * kRankSlot];
            const uint32_t* sh = sl + kRankSlot;
            const float xh = qh[k], xl = ql[k];
            uint32_t c = 0u, c2 = 0u;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
              c += le<OPEN>(__uint_as_float(sl[c + step - 1]), xh) ? (uint32_t)step : 0u;
              c2 += !le<OPEN>(xl, __uint_as_float(sh[c2 + step - 1])) ? (uint32_t)step : 0u;
            }
            c += le<OPEN>(__uint_as_float(sl[c]), xh) ? 1u : 0u;
            c2 += !le<OPEN>(xl, __uint_as_float(sh[c2])) ? 1u : 0u;
            hbm &= sl[35 + c] & ~sh[35 + c2];
          }
          __syncwarp();
          if (BATCH) {  // only this query's instance: positions [r_lo, r_hi)
            const uint32_t base = (g1 + cl) * 32u;
            const uint32_t a = r_lo > base ? min(r_lo - base, 32u) : 0u;
            const uint32_t b = r_hi > base ? min(r_hi - base, 32u) : 0u;
            const uint32_t upto_b = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
            const uint32_t upto_a = a >= 32u ? 0xffffffffu : ((1u << a) - 1u);
            hbm &= upto_b & ~upto_a;
          }
          my_hb = ((qm >> lane) & 1u) ? hbm : 0u;
        } else {
          float2 ev[DM];
  #pragma unroll
          for (int k = 0; k < DM; ++k)
            if (k < d) ev[k] = iv ? t.e[k * n + i] : make_float2(NAN, NAN);  // fails every test
          uint32_t my_sid = 0;
          if (WRITE && iv) my_sid = t.sid[i];
          if (!WRITE && __popc(qm) >= max(q.tmin, kCompareSwapMin)) {
            // Swapped loops: stage the leaf's subscriptions, then every lane
            // tests its own query against all 32 of them (the same segment
            // tests of Alg. 1 in every dimension, in the opposite order).
  #pragma unroll
            for (int k2 = 0; k2 < DP; ++k2) {
              if (2 * k2 < d)
                s_e[wib][lane][k2] = make_float4(ev[2 * k2].x, ev[2 * k2].y,
                                                 2 * k2 + 1 < d ? ev[2 * k2 + 1].x : 0.f,
                                                 2 * k2 + 1 < d ? ev[2 * k2 + 1].y : 0.f);
            }
            __syncwarp();
            uint32_t hbm = 0;
            if constexpr (D >= 1 && D <= 3) {
  #pragma unroll
              for (int e = 0; e < 32; ++e) {
                const float4 b0 = s_e[wib][e][0], b1 = D == 3 ? s_e[wib][e][DP - 1] : b0;
                if (OPEN)
                  seg_or_lt<D>(hbm, 1u << e, b0, b1, ql, qh);
                else
                  seg_or_le<D>(hbm, 1u << e, b0, b1, ql, qh);
              }
            } else {  // runtime d (up to 8)
  #pragma unroll 8
              for (int e = 0; e < 32; ++e) {
                bool hit = true;
  #pragma unroll
                for (int k2 = 0; k2 < DP; ++k2) {
                  if (2 * k2 < d) {
                    const float4 b = s_e[wib][e][k2];
                    hit = hit & le<OPEN>(b.x, qh[2 * k2]) & le<OPEN>(ql[2 * k2], b.y);
                    if (2 * k2 + 1 < d)
                      hit = hit & le<OPEN>(b.z, qh[2 * k2 + 1]) & le<OPEN>(ql[2 * k2 + 1], b.w);
                  }
                }
                hbm |= (hit ? 1u : 0u) << e;
              }
            }
            __syncwarp();
            hbm &= __ballot_sync(0xffffffffu, iv);  // padding lanes of the last leaf
            if (BATCH) {  // only this query's instance: positions [r_lo, r_hi)
              const uint32_t base = (g1 + cl) * 32u;
              const uint32_t a = r_lo > base ? min(r_lo - base, 32u) : 0u;
              const uint32_t b = r_hi > base ? min(r_hi - base, 32u) : 0u;
              const uint32_t upto_b = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
              const uint32_t upto_a = a >= 32u ? 0xffffffffu : ((1u << a) - 1u);
              hbm &= upto_b & ~upto_a;
            }
            my_hb = ((qm >> lane) & 1u) ? hbm : 0u;
            qm = 0u;
          }
          if (!WRITE && qm) {
            // Queries of the leaf as a list of row offsets (in float4 units);
            // two per iteration, each the segment tests of Alg. 1 in every
            // dimension and one ballot, its hit mask stored into its row (every
            // lane stores the same word).
            const bool mine = (qm >> lane) & 1u;
            const uint32_t nq = __popc(qm);
            if (mine) s_list[wib][__popc(qm & lt)] = (uint32_t)(lane * RW);
            __syncwarp();
            const float4* rows = &s_q[wib][0][0];
            uint32_t* hbw = reinterpret_cast<uint32_t*>(&s_q[wib][0][0]);
            auto test = [&](uint32_t r) {
              if constexpr (D >= 1 && D <= 3 && !BATCH) {
                const float4 b0 = rows[r], b1 = D == 3 ? rows[r + 1] : b0;
                hbw[4 * r + HB] = OPEN ? seg_ballot_lt<D>(ev, b0, b1) : seg_ballot_le<D>(ev, b0, b1);
                return;
              }
              bool hit = iv;
              if (BATCH) {
                const uint2 rg = s_rng[wib][r / RW];
                hit = hit & (i >= rg.x) & (i < rg.y);
              }
  #pragma unroll
              for (int k2 = 0; k2 < DP; ++k2) {
                if (2 * k2 < d) {
                  const float4 b = rows[r + k2];
                  hit = hit & le<OPEN>(ev[2 * k2].x, b.y) & le<OPEN>(b.x, ev[2 * k2].y);
                  if (2 * k2 + 1 < d)
                    hit = hit & le<OPEN>(ev[2 * k2 + 1].x, b.w) & le<OPEN>(b.z, ev[2 * k2 + 1].y);
                }
              }
              hbw[4 * r + HB] = __ballot_sync(0xffffffffu, hit);
            };
            uint32_t j = 0;
            for (; j + 2u <= nq; j += 2u) {
              const uint2 rr = *reinterpret_cast<const uint2*>(&s_list[wib][j]);
              test(rr.x);
              test(rr.y);
            }
            if (j < nq) test(s_list[wib][j]);
            __syncwarp();
            my_hb = mine ? hbw[4 * lane * RW + HB] : 0u;
            qm = 0u;
          }
          while (qm) {
            const int qq = __ffs(qm) - 1;
            qm &= qm - 1u;
            bool hit = iv;
            uint32_t sub_base = 0;
            if (BATCH) {
              const uint2 rg = s_rng[wib][qq];
              hit = hit & (i >= rg.x) & (i < rg.y);
              sub_base = rg.x;
            }
  #pragma unroll
            for (int k2 = 0; k2 < DP; ++k2) {
              if (2 * k2 < d) {
                const float4 b = s_q[wib][qq][k2];
                hit = hit & le<OPEN>(ev[2 * k2].x, b.y) & le<OPEN>(b.x, ev[2 * k2].y);
                if (2 * k2 + 1 < d)
                  hit = hit & le<OPEN>(ev[2 * k2 + 1].x, b.w) & le<OPEN>(b.z, ev[2 * k2 + 1].y);
              }
            }
            const uint32_t hb = __ballot_sync(0xffffffffu, hit);
            if (WRITE) {
              const unsigned long long o = __shfl_sync(0xffffffffu, out, qq);
              const uint32_t Qq = __shfl_sync(0xffffffffu, Qout, qq);
              if (hit) {
                const unsigned long long at = o + __popc(hb & lt);
                if (at < w.capacity) {
                  if (w.ids) {
                    w.ids[at] = my_sid - sub_base;
                  } else {
                    ddm_pair pr;
                    pr.upd = Qq;
                    pr.sub = my_sid - sub_base;
                    if (w.swap) pr = ddm_pair{pr.sub, pr.upd};
                    w.pairs[at] = pr;
                  }
                }
              }
              if (lane == qq) out = o + __popc(hb);
            } else {
              if (lane == qq) my_hb = hb;
            }
          }
        }
        if (recording) {
          // Records of lanes 0-15 go to chain 0, of lanes 16-31 to chain 1
          // (kRecChains == 2); both in one store step, each lane at its
          // chain's fill position plus its rank among its chain's records.
          static_assert(kRecChains == 2, "two record chains per packet");
          const uint32_t rm = __ballot_sync(0xffffffffu, my_hb != 0u);
          const uint32_t k0 = __popc(rm & 0xffffu), k1 = __popc(rm >> 16);
          if (rm && (fill0 + k0 > kRecBlock || fill1 + k1 > kRecBlock)) {
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
              const uint32_t kc = ch ? k1 : k0;
              uint32_t& fl = ch ? fill1 : fill0;
              uint32_t& cb = ch ? cur1 : cur0;
              if (kc == 0u || fl + kc <= kRecBlock) continue;  // the leaf's records start a new block
              if (ch) ++nblk1; else ++nblk0;
              if (rec_write) {
                uint32_t b = 0;
                if (lane == 0) b = atomicAdd(&ra.blk_counter[0], 1u);
                b = __shfl_sync(0xffffffffu, b, 0);
                if (b >= ra.max_blocks) {
                  rec_write = false;  // arena exhausted: the write pass walks instead
                } else {
                  if (lane == 0) {
                    if (cb == kNoBlock) {
                      ra.pkt_first[(size_t)p * 2u + ch] = b;
                    } else {
                      ra.blk_next[cb] = b;
                      ra.blk_count[cb] = fl;
                    }
                    ra.blk_pkt[b] = p;
                  }
                  // header: the chain's queries' matches before this leaf
                  if ((uint32_t)(lane >> 4) == (uint32_t)ch) {
                    ra.rec[(size_t)b * kRecWords + 2u * kRecBlock + kRecBlock / 2u + (lane & 15)] = cnt;
                    blk_cnt = cnt;
                  }
                  cb = b;
                }
              }
              fl = 0;
            }
          }
          if (rec_write && my_hb != 0u) {
            const bool hi = lane >= 16;
            const uint32_t at = (hi ? fill1 + __popc(rm & lt & 0xffff0000u) : fill0 + __popc(rm & lt));
            if (DDM_IN_BOUNDS(at < kRecBlock && (hi ? cur1 : cur0) < ra.max_blocks, st)) {
              uint32_t* r = ra.rec + (size_t)(hi ? cur1 : cur0) * kRecWords;
              r[at] = ((g1 + cl) << 5) | (uint32_t)lane;
              r[kRecBlock + at] = my_hb;
              // this query's matches before the leaf, from the block's start
              reinterpret_cast<uint16_t*>(r + 2u * kRecBlock)[at] = (uint16_t)(cnt - blk_cnt);
            }
          }
          fill0 += k0;
          fill1 += k1;
        }
        if (!WRITE) cnt += __popc(my_hb);
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
        if (BATCH) {
          const unsigned long long span = 1ull << (kLog2Fan * lvl);
          ok = ok && (unsigned long long)lane * span < g_hi &&
               ((unsigned long long)lane + 1) * span > g_lo;
        }
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
          if (BATCH) {
            const unsigned long long span = 1ull << (kLog2Fan * (lvl - 1));
            ok = ok && (unsigned long long)ch * span < g_hi &&
                 ((unsigned long long)ch + 1) * span > g_lo;
          }
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
    if (!WRITE && valid && DDM_IN_BOUNDS(Q < m, st)) {
      counts[Q] = cnt;
      if (counts_pos) counts_pos[pos] = cnt;
    }
    if (!WRITE && st && lane == 0 && ntests) atomicAdd(&st->tests, (unsigned long long)ntests);
    if (recording && lane == 0) {
      if (rec_write) {
        if (cur0 == kNoBlock) {
          ra.pkt_first[(size_t)p * 2u] = kNoBlock;
        } else {
          ra.blk_next[cur0] = kNoBlock;
          ra.blk_count[cur0] = fill0;
        }
        if (cur1 == kNoBlock) {
          ra.pkt_first[(size_t)p * 2u + 1u] = kNoBlock;
        } else {
          ra.blk_next[cur1] = kNoBlock;
          ra.blk_count[cur1] = fill1;
        }
      }
      ra.pkt_nblk[(size_t)p * 2u] = rec_write ? nblk0 : 0u;
      ra.pkt_nblk[(size_t)p * 2u + 1u] = rec_write ? nblk1 : 0u;
      if (nblk0 + nblk1) atomicAdd(&ra.blk_counter[1], nblk0 + nblk1);
    }
  }
}

// Plan-order list of record blocks: one thread per chain copies it (chains of
// a packet in lane order, packets in plan order).
__global__ void k_block_list(RecordArena ra, uint32_t packets) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // sizing hint for the next arena
    ra.blk_counter[2] = packets;
    ra.blk_counter[3] = ra.max_blocks;
  }
  if (!records_complete(ra)) return;
  const uint32_t chains = packets * kRecChains;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < chains;
       p += gridDim.x * blockDim.x) {
    unsigned long long at = ra.pkt_off[p];
    for (uint32_t b = ra.pkt_first[p]; b != kNoBlock; b = ra.blk_next[b]) ra.blk_list[at++] = b;
  }
}

// L2 eviction-priority hints (PTX createpolicy / .L2::cache_hint): the pairs
// and the records stream through L2 once and are marked evict-first, so that
// they do not push the subscription ids (reused by every record that names
// their leaf) out of L2; the id loads are marked evict-last.
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_hinted(const uint32_t* a, unsigned long long policy) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(policy));
  return v;
}
__device__ __forceinline__ uint32_t ld_hinted(const uint16_t* a, unsigned long long policy) {
  unsigned short v;
  asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(policy));
  return v;
}
__device__ __forceinline__ void st_hinted(ddm_pair* a, ddm_pair v, unsigned long long policy) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(a), "r"(v.upd),
               "r"(v.sub), "l"(policy)
               : "memory");
}

__device__ __forceinline__ void st_hinted(uint32_t* a, uint32_t v, unsigned long long policy) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(policy) : "memory");
}

// Write pass from the records of the count pass.  Work unit: one record
// block (up to 512 records of one packet), taken from the plan-order block
// list, so uneven packets spread over the whole GPU.  A warp loads the
// block's packet queries (their output offsets) and takes the records 32 at
// a time (the next 32 are loaded while these expand), one per lane: each lane
// works out where its record's pairs go (its query's offset, plus the block
// header's count of the query's matches before the block, plus the record's
// own count of them since) and leaves (leaf, hit mask, update id, position)
// in shared memory.  The warp then expands the 32
// records one after another with lane = leaf slot, each record's fields read
// by one broadcast from shared memory: the lanes whose bit is set in the hit
// mask load their subscription ids (one 128-byte load for the whole leaf) and
// store their pairs at the record's position plus their rank among the set
// bits -- one contiguous run of the output per record.  A group of records
// (ReplayShape) is in flight at a time (their id loads issued before their
// stores).  Positions
// are relative to the range's first pair; with fewer than 2^32 pairs in the
// range (WIDE false) they are 32-bit.  OUT fixes the output form at compile
// time: kOutPairs {update, subscription}; kOutSwapped the same with the
// fields exchanged (roles swapped: the tree holds the updates); kOutIds the
// compressed output, only each pair's subscription id (4 bytes) at the
// pair's position.
constexpr int kOutPairs = 0, kOutSwapped = 1, kOutIds = 2;
// Resident CTAs per SM and records expanded per group (their id loads issued
// before their stores) of the replay kernel, by output form.  Pairs (8-byte
// stores): two CTAs of eight warps with sixteen records in flight each (128
// registers, no spill) beat four CTAs with eight (64 registers, spilling):
// 131.9 against 147.4 ms per step on the clustered d = 3 workload; one CTA,
// or four records per group, was slower.  Subscription ids (4-byte stores)
// go the other way: four CTAs with eight records take 122.3 ms, three 138.0,
// two 178.7.
//
// The ids form also expands differently (dense): per round of 32 records, a
// scan of their hit counts turns the hit bits into a list of pairs, and each
// lane then writes one id of the list (one load and one 32-lane store per 32
// ids) -- 115.1 instead of 122.1 ms; for pairs that form is slower (147.6 at
// three CTAs, 168.8 at two).
template <int OUT>
struct ReplayShape {
  static constexpr int ctas = OUT == 2 ? 4 : 2;
  static constexpr int group = OUT == 2 ? 8 : 16;
  static constexpr bool dense = OUT == 2;
  // a round of 32 records is expanded in whole groups
  static_assert(32 % group == 0, "records in flight must divide a round of 32");
};
template <bool FILTER_ID, bool WIDE, bool BATCH, int OUT>
__global__ void __launch_bounds__(kThreads, ReplayShape<OUT>::ctas)
k_replay(TreeView t, QueryView q, BatchView bv, RecordArena ra, WriteView w, uint32_t p0,
         uint32_t p1, uint32_t pb, uint32_t pe, uint32_t idb, uint32_t ide,
         uint32_t* __restrict__ work, Status* __restrict__ st) {
  using Cursor = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  // Per record: leaf, hit mask, update id, and the output position of its first
  // pair (32-bit positions, not batched: one 128-bit load per record) or else
  // the subscription id base, the position then in s_at.
  __shared__ uint4 s_rec[kWarps][32];
  __shared__ Cursor s_at[kWarps][32];
  constexpr bool kDense = ReplayShape<OUT>::dense;
  // dense expansion: each round's pairs as a list of (record, leaf slot)
  __shared__ uint32_t s_pre[kDense ? kWarps : 1][32];
  __shared__ uint16_t s_list[kDense ? kWarps : 1][kDense ? 1024 : 2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t below = (1u << lane) - 1u;  // lanes below this one
  const uint32_t lanebit = 1u << lane;
  if (!records_complete(ra)) return;  // the walking write pass handles this range
  const unsigned long long base0 = w.start[w.b_idx];
  const unsigned long long need = w.start[w.e_idx] - base0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->K = need;
    if (need > w.capacity) atomicOr(&st->err, kErrCapacity);
  }
  // Pair positions are bounded by construction: a record's pairs go to its
  // update's offset plus the matches the count pass had found before it, and
  // the update's count is the sum of its records' popcounts, so all writes
  // stay below need <= capacity.
  if (need > w.capacity) return;
  if (!WIDE && need > 0xffffffffull) return;  // host picks WIDE for such ranges
  ddm_pair* __restrict__ pairs = w.pairs;
  uint32_t* __restrict__ ids = w.ids;
  const uint32_t* __restrict__ sid = t.sid;
  const unsigned long long keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
  const unsigned long long i0 = ra.pkt_off[(size_t)p0 * kRecChains],
                           i1 = ra.pkt_off[(size_t)p1 * kRecChains];
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = i0 + atomicAdd(work, 1u);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= i1) break;
    const uint32_t blk = ra.blk_list[i];
    const uint32_t p = ra.blk_pkt[blk];
    const uint32_t pos = (p << q.qpp_log2) + lane;
    bool valid = (uint32_t)lane < (1u << q.qpp_log2) && pos >= pb && pos < pe;
    uint32_t Q = 0;
    if (valid) Q = q.qid[pos];
    if (FILTER_ID) valid = valid && Q >= idb && Q < ide;
    Cursor out = 0;
    if (valid) out = (Cursor)(w.start[w.by_pos ? pos : Q] - base0);
    uint32_t Qout = Q + w.qbase, sub_base = 0;
    if (w.qids && valid) Qout = w.qids[Q];
    if (BATCH && valid) {
      const uint32_t b = bv.q_inst[pos];
      Qout = Q - (uint32_t)bv.upd_off[b];
      sub_base = (uint32_t)bv.sub_off[b];
    }
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    if (vmask == 0u) continue;
    const uint32_t nrec = ra.blk_count[blk];
    const uint32_t* rec = ra.rec + (size_t)blk * kRecWords;
    const uint16_t* rel = reinterpret_cast<const uint16_t*>(rec + 2u * kRecBlock);
    uint32_t nx = 0u, nhb = 0u, nrel = 0u;
    if (lane < nrec) {
      nx = ld_hinted(&rec[lane], stream);
      nhb = ld_hinted(&rec[kRecBlock + lane], stream);
      nrel = ld_hinted(&rel[lane], stream);
    }
    // the block header: lane j holds the matches query j of the chain had
    // before the block
    const uint32_t hdr =
        lane < (int)kRecHdr ? ld_hinted(&rec[2u * kRecBlock + kRecBlock / 2u + lane], stream) : 0u;
    for (uint32_t r0 = 0; r0 < nrec; r0 += 32u) {
      const uint32_t x = nx, xrel = nrel;
      uint32_t hb = nhb;
      nx = nhb = nrel = 0u;  // lanes past the block's last record hold x = hb = 0
      if (r0 + 32u + lane < nrec) {
        nx = ld_hinted(&rec[r0 + 32u + lane], stream);
        nhb = ld_hinted(&rec[kRecBlock + r0 + 32u + lane], stream);
        nrel = ld_hinted(&rel[r0 + 32u + lane], stream);
      }
      const int qq = (int)(x & 31u);
      // the query's matches before this record: header + the record's count
      const uint32_t bef = __shfl_sync(0xffffffffu, hdr, qq & (int)(kRecHdr - 1)) + xrel;
      if (!((vmask >> qq) & 1u)) hb = 0u;  // also clears lanes past nrec (x = hb = 0)
      const Cursor o = __shfl_sync(0xffffffffu, out, qq) + (Cursor)bef;
      const uint32_t Qq = __shfl_sync(0xffffffffu, Qout, qq);
      const uint32_t sb = BATCH ? __shfl_sync(0xffffffffu, sub_base, qq) : 0u;
      __syncwarp();  // the previous round has read s_rec / s_at
      constexpr bool kPacked = !WIDE && !BATCH;  // position fits the record's fourth word
      s_rec[wib][lane] = make_uint4(x >> 5, hb, Qq, kPacked ? (uint32_t)o : sb);
      if (!kPacked) s_at[wib][lane] = o;
      if constexpr (kDense) {
        // The round's pairs, numbered record by record: an exclusive scan of
        // the records' hit counts gives each record's first pair; the hit
        // bits become a list of (record, leaf slot) in that numbering
        // (lane = leaf slot); then every lane takes one pair of the list at
        // a time: one id load and one store per 32 pairs.
        const uint32_t c = __popc(hb);
        uint32_t incl = c;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, dd);
          if (lane >= dd) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        s_pre[wib][lane] = incl - c;
        __syncwarp();
#pragma unroll 8
        for (int u = 0; u < 32; ++u) {
          const uint32_t h = s_rec[wib][u].y;
          if (h & lanebit)
            s_list[wib][s_pre[wib][u] + __popc(h & below)] = (uint16_t)(((uint32_t)u << 5) | (uint32_t)lane);
        }
        __syncwarp();
#pragma unroll 2
        for (uint32_t ti = lane; ti < total; ti += 32u) {
          const uint32_t ent = s_list[wib][ti];
          const uint32_t r = ent >> 5, slot = ent & 31u;
          const uint4 R = s_rec[wib][r];
          const Cursor at = (kPacked ? (Cursor)R.w : s_at[wib][r]) + (Cursor)(ti - s_pre[wib][r]);
          if (!DDM_IN_BOUNDS(R.x * 32u + slot < t.n && (unsigned long long)at < need, st)) continue;
          const uint32_t sv = ld_hinted(sid + R.x * 32u + slot, keep);
          const uint32_t sub = sv - (kPacked ? 0u : R.w);
          if (OUT == kOutIds) {
            st_hinted(ids + (unsigned long long)at, sub, stream);
          } else {
            ddm_pair pr;
            pr.upd = OUT == kOutSwapped ? sub : R.z;
            pr.sub = OUT == kOutSwapped ? R.z : sub;
            st_hinted(pairs + (unsigned long long)at, pr, stream);
          }
        }
        continue;
      }
      __syncwarp();
#pragma unroll 1
      constexpr int G = ReplayShape<OUT>::group;
      for (int g = 0; g < 32; g += G) {
        uint4 rr[G];
        uint32_t sv[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
          rr[u] = s_rec[wib][g + u];
          sv[u] = 0u;
          if ((rr[u].y & lanebit) && DDM_IN_BOUNDS(rr[u].x * 32u + (uint32_t)lane < t.n, st))
            sv[u] = ld_hinted(sid + rr[u].x * 32u + (uint32_t)lane, keep);
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
          if (rr[u].y & lanebit) {
            const Cursor at = kPacked ? (Cursor)rr[u].w : s_at[wib][g + u];
            const unsigned long long slot = (unsigned long long)(at + (Cursor)__popc(rr[u].y & below));
            if (!DDM_IN_BOUNDS(slot < need, st)) continue;
            const uint32_t sub = sv[u] - (kPacked ? 0u : rr[u].w);
            if (OUT == kOutIds) {
              st_hinted(ids + slot, sub, stream);
            } else {
              ddm_pair pr;
              pr.upd = OUT == kOutSwapped ? sub : rr[u].z;
              pr.sub = OUT == kOutSwapped ? rr[u].z : sub;
              st_hinted(pairs + slot, pr, stream);
            }
          }
        }
      }
    }
  }
}

template <bool WRITE, bool BATCH>
void dispatch_packets(int d, bool open, uint32_t blocks, cudaStream_t s, const TreeView& t,
                      const QueryView& q, const BatchView& bv, uint32_t* counts,
                      uint32_t* counts_pos, const RecordArena& ra, const WriteView& w,
                      uint32_t* work, Status* st) {
#define DDM_LAUNCH(DD, OP)                                                              \
  k_packets<DD, OP, WRITE, BATCH><<<blocks, kThreads, 0, s>>>(t, q, bv, counts, counts_pos, \
                                                               ra, w, work, st)
  switch (d) {
    case 1: open ? DDM_LAUNCH(1, true) : DDM_LAUNCH(1, false); break;
    case 2: open ? DDM_LAUNCH(2, true) : DDM_LAUNCH(2, false); break;
    case 3: open ? DDM_LAUNCH(3, true) : DDM_LAUNCH(3, false); break;
    default: open ? DDM_LAUNCH(0, true) : DDM_LAUNCH(0, false); break;
  }
#undef DDM_LAUNCH
}

template <bool WRITE>
cudaError_t launch_packets(const TreeView& t, const QueryView& q, const BatchView& bv,
                           uint32_t flags, uint32_t* counts, uint32_t* counts_pos,
                           const RecordArena& ra, const WriteView& w, uint32_t* work, Status* st,
                           int sms, cudaStream_t s) {
  if (q.nq == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
  if (e) return e;
  const bool open = (flags & DDM_OPEN) != 0;
  const uint32_t packets = (q.nq + (1u << q.qpp_log2) - 1u) >> q.qpp_log2;
  uint32_t blocks = (packets + kWarps - 1) / kWarps;
  const uint32_t cap = (uint32_t)sms * 8u;
  if (blocks > cap) blocks = cap;
  if (bv.count)
    dispatch_packets<WRITE, true>(t.d, open, blocks, s, t, q, bv, counts, counts_pos, ra, w, work,
                                  st);
  else
    dispatch_packets<WRITE, false>(t.d, open, blocks, s, t, q, bv, counts, counts_pos, ra, w,
                                   work, st);
  note_launches(1);
  return cudaGetLastError();
}

template <bool FILTER_ID, bool BATCH>
void dispatch_replay(bool wide, uint32_t sms, cudaStream_t s, const TreeView& t,
                     const QueryView& q, const BatchView& bv, const RecordArena& ra,
                     const WriteView& w, uint32_t p0, uint32_t p1, uint32_t pb, uint32_t pe,
                     uint32_t idb, uint32_t ide, uint32_t* work, Status* st) {
#define DDM_REPLAY(F, WD, OUT)                                                              \
  k_replay<F, WD, BATCH, OUT><<<sms * ReplayShape<OUT>::ctas, kThreads, 0, s>>>(t, q, bv, ra, w, p0, p1, pb, pe, idb, \
                                                          ide, work, st)
  // Compressed output and swapped roles: whole single problems only (checked
  // by launch_replay), so those forms exist for that case alone.
  if constexpr (!FILTER_ID && !BATCH) {
    if (w.ids) {
      wide ? DDM_REPLAY(false, true, kOutIds) : DDM_REPLAY(false, false, kOutIds);
      return;
    }
    if (w.swap) {
      wide ? DDM_REPLAY(false, true, kOutSwapped) : DDM_REPLAY(false, false, kOutSwapped);
      return;
    }
  }
  wide ? DDM_REPLAY(FILTER_ID, true, kOutPairs) : DDM_REPLAY(FILTER_ID, false, kOutPairs);
#undef DDM_REPLAY
}

__global__ void k_gather_offsets(const unsigned long long* __restrict__ offsets, uint32_t m,
                                 const unsigned long long* __restrict__ upd_off, uint32_t count,
                                 unsigned long long* __restrict__ pair_off) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += gridDim.x * blockDim.x) {
    const unsigned long long u = upd_off[i];
    pair_off[i] = offsets[u < m ? u : m];
  }
}

}  // namespace

cudaError_t launch_count(const TreeView& t, const QueryView& q, const BatchView& bv,
                         uint32_t flags, uint32_t* counts, uint32_t* counts_pos,
                         const RecordArena& ra, uint32_t* work, Status* st, int sms,
                         cudaStream_t s) {
  WriteView w{};
  return launch_packets<false>(t, q, bv, flags, counts, counts_pos, ra, w, work, st, sms, s);
}

cudaError_t launch_write(const TreeView& t, const QueryView& q, const BatchView& bv,
                         uint32_t flags, const WriteView& w, const RecordArena& ra,
                         uint32_t* work, Status* st, int sms, cudaStream_t s) {
  return launch_packets<true>(t, q, bv, flags, nullptr, nullptr, ra, w, work, st, sms, s);
}

cudaError_t launch_block_list(const RecordArena& ra, uint32_t packets, cudaStream_t s) {
  if (packets == 0 || ra.max_blocks == 0) return cudaSuccess;
  uint32_t blocks = (packets + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_block_list<<<blocks, 256, 0, s>>>(ra, packets);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_replay(const TreeView& t, const QueryView& q, const BatchView& bv,
                          const RecordArena& ra, const WriteView& w, uint32_t p0, uint32_t p1,
                          uint32_t pb, uint32_t pe, bool id_filter, uint32_t idb, uint32_t ide,
                          uint32_t* work, Status* st, int sms, cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  if ((w.ids || w.swap) && (id_filter || bv.count)) return cudaErrorInvalidValue;  // see dispatch_replay
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
  if (e) return e;
  // Cursors fit 32 bits when the range's pairs do; the capacity bounds them.
  const bool wide = w.capacity > 0xffffffffull;
  if (id_filter) {
    if (bv.count)
      dispatch_replay<true, true>(wide, (uint32_t)sms, s, t, q, bv, ra, w, p0, p1, pb, pe, idb, ide, work, st);
    else
      dispatch_replay<true, false>(wide, (uint32_t)sms, s, t, q, bv, ra, w, p0, p1, pb, pe, idb, ide, work, st);
  } else {
    if (bv.count)
      dispatch_replay<false, true>(wide, (uint32_t)sms, s, t, q, bv, ra, w, p0, p1, pb, pe, idb, ide, work, st);
    else
      dispatch_replay<false, false>(wide, (uint32_t)sms, s, t, q, bv, ra, w, p0, p1, pb, pe, idb, ide, work, st);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_offsets(const unsigned long long* offsets, uint32_t m,
                                  const unsigned long long* upd_off, uint32_t count,
                                  unsigned long long* pair_off, cudaStream_t s) {
  const uint32_t blocks = (count + 256) / 256 < 1024 ? (count + 256) / 256 : 1024;
  k_gather_offsets<<<blocks, 256, 0, s>>>(offsets, m, upd_off, count, pair_off);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ddm
