/*
 * CPU oracle for Data Distribution Management matching
 * (Marzolla, D'Angelo, Mandrioli, "A Parallel Data Distribution Management
 * Algorithm", DS-RT 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the library's
 * product path never does.  It shares no code, header or constant with the
 * CUDA path.
 *
 * Problem (Section III): subscription extents S_1..S_n and update extents
 * U_1..U_m, each a d-rectangle; report every pair (S_i, U_j) whose
 * intersection is non-empty.  Ids are 0-based input indices here (the paper
 * numbers from 1).
 *
 * Coordinates arrive as float32 in structure-of-arrays layout: row k
 * (dimension k) of a set with c extents starts at offset k*c.  All
 * arithmetic below is comparisons, carried out on values widened to double
 * (exact for float32 inputs, so no rounding enters).
 *
 * Readings of the paper taken here:
 *  - Closed vs open segments.  Alg. 1 writes strict comparisons, while the
 *    segments are written as closed intervals [low, high].  The default rule
 *    is closed (x.low <= y.high and y.low <= x.high); flag OPEN selects the
 *    literal strict test of Alg. 1.
 *  - Under the closed rule the right-subtree descent of Alg. 4 becomes
 *    q.upper >= x.in.lower (equal lower keys may sit in the right subtree).
 *  - Tree order (Section IV): by lower bound, ties by upper bound; remaining
 *    ties by id (the paper is silent; this only fixes an order).
 *
 * Parity: pinned.  BF and ITM are checked against each other, against
 * closed-form lattice counts, against the worked example of Fig. 1 and
 * against BITS counting (Section II) by the CPU test suite.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OPEN 1u

/* ------------------------------------------------------------------ */
/* Alg. 1, Intersect-1D                                                */
/* ------------------------------------------------------------------ */
static int intersect_1d(double xlo, double xhi, double ylo, double yhi, int open)
{
    if (open)
        return xlo < yhi && ylo < xhi;          /* the strict test of Alg. 1 */
    return xlo <= yhi && ylo <= xhi;            /* closed segments */
}

/* Section III-A: two d-rectangles intersect iff all their projections do. */
static int intersect_d(int d,
                       const float *alo, const float *ahi, uint64_t astride, uint64_t ai,
                       const float *blo, const float *bhi, uint64_t bstride, uint64_t bi,
                       int open)
{
    for (int k = 0; k < d; ++k) {
        if (!intersect_1d(alo[k * astride + ai], ahi[k * astride + ai],
                          blo[k * bstride + bi], bhi[k * bstride + bi], open))
            return 0;
    }
    return 1;
}

int oracle_intersect_1d(double xlo, double xhi, double ylo, double yhi, uint32_t flags)
{
    return intersect_1d(xlo, xhi, ylo, yhi, (flags & ORACLE_OPEN) != 0);
}

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014), used only
 * to give each update an order-independent digest of its matched ids. */
uint64_t oracle_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* Alg. 2, Brute Force, extended to d dimensions (Section III-A).      */
/* The pair test of every (S_i, U_j) is independent; the loop runs     */
/* over updates outside so that each update's pairs come out together, */
/* in ascending subscription id.                                       */
/* ------------------------------------------------------------------ */
uint64_t oracle_bf(int d,
                   const float *upd_lo, const float *upd_hi, uint32_t m,
                   const float *sub_lo, const float *sub_hi, uint32_t n,
                   uint32_t flags,
                   uint32_t *counts,                  /* [m] or NULL */
                   uint64_t *digests,                 /* [m] or NULL */
                   uint32_t *out_upd, uint32_t *out_sub, uint64_t cap)
{
    const int open = (flags & ORACLE_OPEN) != 0;
    uint64_t K = 0;
    for (uint32_t j = 0; j < m; ++j) {
        uint32_t c = 0;
        uint64_t dig = 0;
        for (uint32_t i = 0; i < n; ++i) {
            if (intersect_d(d, sub_lo, sub_hi, n, i, upd_lo, upd_hi, m, j, open)) {
                if (out_upd && K < cap) {
                    out_upd[K] = j;
                    out_sub[K] = i;
                }
                ++K;
                ++c;
                dig += oracle_mix64(i);
            }
        }
        if (counts) counts[j] = c;
        if (digests) digests[j] = dig;
    }
    return K;
}

/* ------------------------------------------------------------------ */
/* Interval tree (Section IV): augmented AVL tree.                     */
/* Each node holds one interval x.in (dimension 0 of a subscription),  */
/* plus maxupper / minlower of the subtree rooted at it.               */
/* ------------------------------------------------------------------ */
typedef struct {
    double lo, hi;          /* x.in */
    uint32_t id;            /* x.in.id */
    double maxupper, minlower;
    int32_t left, right;    /* -1 = null */
    int32_t height;
} it_node;

typedef struct {
    it_node *v;
    int32_t root;
    uint32_t size;
} it_tree;

static int32_t h_of(const it_tree *t, int32_t x) { return x < 0 ? 0 : t->v[x].height; }

/* Recompute the augmented fields of x from its interval and children. */
static void it_fix(it_tree *t, int32_t x)
{
    it_node *p = &t->v[x];
    double mu = p->hi, ml = p->lo;
    int32_t hl = h_of(t, p->left), hr = h_of(t, p->right);
    if (p->left >= 0) {
        if (t->v[p->left].maxupper > mu) mu = t->v[p->left].maxupper;
        if (t->v[p->left].minlower < ml) ml = t->v[p->left].minlower;
    }
    if (p->right >= 0) {
        if (t->v[p->right].maxupper > mu) mu = t->v[p->right].maxupper;
        if (t->v[p->right].minlower < ml) ml = t->v[p->right].minlower;
    }
    p->maxupper = mu;
    p->minlower = ml;
    p->height = 1 + (hl > hr ? hl : hr);
}

static int32_t rot_right(it_tree *t, int32_t y)
{
    int32_t x = t->v[y].left;
    t->v[y].left = t->v[x].right;
    t->v[x].right = y;
    it_fix(t, y);
    it_fix(t, x);
    return x;
}

static int32_t rot_left(it_tree *t, int32_t x)
{
    int32_t y = t->v[x].right;
    t->v[x].right = t->v[y].left;
    t->v[y].left = x;
    it_fix(t, x);
    it_fix(t, y);
    return y;
}

/* Key order: lower bound, then upper bound, then id. */
static int key_less(const it_node *a, const it_node *b)
{
    if (a->lo < b->lo) return 1;
    if (b->lo < a->lo) return 0;
    if (a->hi < b->hi) return 1;
    if (b->hi < a->hi) return 0;
    return a->id < b->id;
}

/* Usual AVL insertion; augmented fields are refreshed on the way back to the
 * root and through every rotation, so they stay exact (Section IV). */
static int32_t it_insert(it_tree *t, int32_t x, int32_t z)
{
    if (x < 0) return z;
    if (key_less(&t->v[z], &t->v[x]))
        t->v[x].left = it_insert(t, t->v[x].left, z);
    else
        t->v[x].right = it_insert(t, t->v[x].right, z);
    it_fix(t, x);
    int32_t bal = h_of(t, t->v[x].left) - h_of(t, t->v[x].right);
    if (bal > 1) {
        if (h_of(t, t->v[t->v[x].left].left) < h_of(t, t->v[t->v[x].left].right))
            t->v[x].left = rot_left(t, t->v[x].left);
        return rot_right(t, x);
    }
    if (bal < -1) {
        if (h_of(t, t->v[t->v[x].right].right) < h_of(t, t->v[t->v[x].right].left))
            t->v[x].right = rot_right(t, t->v[x].right);
        return rot_left(t, x);
    }
    return x;
}

/* Interval-Tree-Create (Alg. 5): n insertions of dimension-0 segments. */
static int it_create(it_tree *t, const float *lo0, const float *hi0, uint32_t n)
{
    t->v = (it_node *)malloc((size_t)(n ? n : 1) * sizeof(it_node));
    if (!t->v) return -1;
    t->root = -1;
    t->size = n;
    for (uint32_t i = 0; i < n; ++i) {
        it_node *p = &t->v[i];
        p->lo = lo0[i];
        p->hi = hi0[i];
        p->id = i;
        p->left = p->right = -1;
        p->height = 1;
        p->maxupper = p->hi;
        p->minlower = p->lo;
        t->root = it_insert(t, t->root, (int32_t)i);
    }
    return 0;
}

typedef struct {
    int d, open;
    const float *ulo, *uhi; uint32_t m; uint32_t j;   /* the query U_j */
    const float *slo, *shi; uint32_t n;
    uint32_t count;
    uint64_t digest;
    uint32_t *out_sub; uint64_t cap; uint64_t K;      /* optional pair list */
} it_query;

/* Interval-Query (Alg. 4), written as an iterative in-order walk with an
 * explicit stack.  Every prune below follows from the segment test of
 * Section III-A on dimension 0 and from what a subtree's augmented fields
 * bound:
 *  - every interval s stored under a node x has s.hi <= x.maxupper and
 *    s.lo >= x.minlower;
 *  - s meets the query [ql, qh] (closed rule) only if s.hi >= ql and
 *    s.lo <= qh, so no interval under x can meet it when x.maxupper < ql or
 *    x.minlower > qh (these bounds are conservative for the open rule too);
 *  - the tree is ordered by lower bound, so every interval in x's right
 *    subtree has s.lo >= x.lo: when x.lo > qh (closed) or x.lo >= qh (open)
 *    that subtree cannot hold a match.
 * The walk reports the surviving intervals in tree order (left subtree,
 * node, right subtree).  An interval that meets the query on dimension 0
 * is then tested on dimensions 1..d-1 before it is reported. */
#define IT_STACK_MAX 128   /* AVL height <= 1.45 log2(n + 2) < 64 for n < 2^32 */

static int subtree_may_meet(const it_node *x, double ql, double qh)
{
    return !(x->maxupper < ql) && !(x->minlower > qh);
}

static int right_may_meet(const it_node *x, double qh, int open)
{
    return open ? (qh > x->lo) : (qh >= x->lo);
}

/* Dimensions 1..d-1 of subscription `sid` against the query U_j. */
static int other_dims_meet(const it_query *q, uint32_t sid)
{
    for (int k = 1; k < q->d; ++k) {
        const uint64_t si = (uint64_t)k * q->n + sid, uj = (uint64_t)k * q->m + q->j;
        if (!intersect_1d(q->slo[si], q->shi[si], q->ulo[uj], q->uhi[uj], q->open))
            return 0;
    }
    return 1;
}

static void it_report(it_query *q, uint32_t sid)
{
    if (q->out_sub && q->K < q->cap) q->out_sub[q->K] = sid;
    ++q->K;
    ++q->count;
    q->digest += oracle_mix64(sid);
}

static void it_query_walk(const it_tree *t, it_query *q)
{
    const double ql = q->ulo[q->j], qh = q->uhi[q->j];
    int32_t stack[IT_STACK_MAX];
    int top = 0;
    int32_t x = t->root;
    for (;;) {
        /* go down the left spine of every subtree that may hold a match */
        while (x >= 0 && subtree_may_meet(&t->v[x], ql, qh)) {
            if (top == IT_STACK_MAX) abort();   /* unreachable for an AVL tree */
            stack[top++] = x;
            x = t->v[x].left;
        }
        if (top == 0) break;
        const it_node *p = &t->v[stack[--top]];
        if (intersect_1d(p->lo, p->hi, ql, qh, q->open) && other_dims_meet(q, p->id))
            it_report(q, p->id);
        x = right_may_meet(p, qh, q->open) ? p->right : -1;
    }
}

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* IntTree-Matching (Alg. 5) with per-update counts and digests; the loop
 * over updates is split across threads as in the paper's parallel ITM
 * (Section IV, "Parallelizing ITM"): every query only reads the tree.
 * seconds (optional, 2 entries) receives the wall time of the tree build
 * and of the queries. */
uint64_t oracle_itm_count(int d,
                          const float *upd_lo, const float *upd_hi, uint32_t m,
                          const float *sub_lo, const float *sub_hi, uint32_t n,
                          uint32_t flags, int nthreads,
                          uint32_t *counts, uint64_t *digests, double *seconds)
{
    it_tree t;
    double t0 = now_s();
    if (it_create(&t, sub_lo, sub_hi, n) != 0) return UINT64_MAX;
    double t1 = now_s();
    uint64_t K = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : K) num_threads(nthreads)
#endif
    for (int64_t jj = 0; jj < (int64_t)m; ++jj) {
        it_query q;
        memset(&q, 0, sizeof q);
        q.d = d; q.open = (flags & ORACLE_OPEN) != 0;
        q.ulo = upd_lo; q.uhi = upd_hi; q.m = m; q.j = (uint32_t)jj;
        q.slo = sub_lo; q.shi = sub_hi; q.n = n;
        it_query_walk(&t, &q);
        if (counts) counts[jj] = q.count;
        if (digests) digests[jj] = q.digest;
        K += q.count;
    }
    if (seconds) {
        seconds[0] = t1 - t0;
        seconds[1] = now_s() - t1;
    }
    free(t.v);
    return K;
}

/* Sequential ITM producing the pair list, update by update; within an
 * update the pairs come in tree (in-order) order. */
uint64_t oracle_itm_pairs(int d,
                          const float *upd_lo, const float *upd_hi, uint32_t m,
                          const float *sub_lo, const float *sub_hi, uint32_t n,
                          uint32_t flags,
                          uint32_t *out_upd, uint32_t *out_sub, uint64_t cap)
{
    it_tree t;
    if (it_create(&t, sub_lo, sub_hi, n) != 0) return UINT64_MAX;
    uint64_t K = 0;
    for (uint32_t j = 0; j < m; ++j) {
        it_query q;
        memset(&q, 0, sizeof q);
        q.d = d; q.open = (flags & ORACLE_OPEN) != 0;
        q.ulo = upd_lo; q.uhi = upd_hi; q.m = m; q.j = j;
        q.slo = sub_lo; q.shi = sub_hi; q.n = n;
        q.out_sub = out_sub ? out_sub + (K < cap ? K : cap) : NULL;
        q.cap = K < cap ? cap - K : 0;
        it_query_walk(&t, &q);
        if (out_upd)
            for (uint64_t r = K; r < K + q.count && r < cap; ++r) out_upd[r] = j;
        K += q.count;
    }
    free(t.v);
    return K;
}

/* In-order sequence of the interval tree: subscription ids sorted by
 * (lower, upper, id) on dimension 0; also reports the tree height. */
static void inorder(const it_tree *t, int32_t x, uint32_t *out, uint32_t *pos)
{
    if (x < 0) return;
    inorder(t, t->v[x].left, out, pos);
    out[(*pos)++] = t->v[x].id;
    inorder(t, t->v[x].right, out, pos);
}

int oracle_tree_order(const float *lo0, const float *hi0, uint32_t n, uint32_t *order, int32_t *height)
{
    it_tree t;
    if (it_create(&t, lo0, hi0, n) != 0) return -1;
    uint32_t pos = 0;
    inorder(&t, t.root, order, &pos);
    if (height) *height = h_of(&t, t.root);
    free(t.v);
    return 0;
}

/* ------------------------------------------------------------------ */
/* BITS counting (Layer et al., Section II), d = 1, closed rule only:  */
/* |B| minus the intervals ending before q.low minus those starting    */
/* after q.high; for lo <= hi the two events are disjoint.             */
/* ------------------------------------------------------------------ */
static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* number of v[] strictly less than key (v sorted ascending) */
static uint32_t count_less(const float *v, uint32_t n, double key)
{
    uint32_t a = 0, b = n;
    while (a < b) {
        uint32_t mid = a + (b - a) / 2;
        if (v[mid] < key) a = mid + 1; else b = mid;
    }
    return a;
}

/* number of v[] less than or equal to key */
static uint32_t count_le(const float *v, uint32_t n, double key)
{
    uint32_t a = 0, b = n;
    while (a < b) {
        uint32_t mid = a + (b - a) / 2;
        if (v[mid] <= key) a = mid + 1; else b = mid;
    }
    return a;
}

uint64_t oracle_bits_count(const float *upd_lo, const float *upd_hi, uint32_t m,
                           const float *sub_lo, const float *sub_hi, uint32_t n,
                           uint32_t *counts)
{
    float *bs = (float *)malloc((size_t)(n ? n : 1) * sizeof(float));
    float *be = (float *)malloc((size_t)(n ? n : 1) * sizeof(float));
    if (!bs || !be) { free(bs); free(be); return UINT64_MAX; }
    memcpy(bs, sub_lo, (size_t)n * sizeof(float));
    memcpy(be, sub_hi, (size_t)n * sizeof(float));
    qsort(bs, n, sizeof(float), cmp_float);
    qsort(be, n, sizeof(float), cmp_float);
    uint64_t K = 0;
    for (uint32_t j = 0; j < m; ++j) {
        uint32_t end_before = count_less(be, n, upd_lo[j]);      /* S.hi < q.lo */
        uint32_t start_after = n - count_le(bs, n, upd_hi[j]);   /* S.lo > q.hi */
        uint32_t c = n - end_before - start_after;
        if (counts) counts[j] = c;
        K += c;
    }
    free(bs);
    free(be);
    return K;
}

int oracle_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
