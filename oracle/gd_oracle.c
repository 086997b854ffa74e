/*
 * CPU oracle for exact Euclidean DBSCAN (GriT-DBSCAN, arXiv 2210.07580).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * never calls it and shares no code with it.
 *
 * Two implementations of the same result:
 *
 *   oracle_bruteforce  -- the DBSCAN definitions (Section 3.1, Defs. 1-5)
 *                         written out as O(n^2) loops over all point pairs.
 *   oracle_grid        -- the paper's own method (Section 4): Eq. 1 grid,
 *                         Alg. 1 partitioning, the grid-tree neighbour query
 *                         of Alg. 3 (on the sorted cell array), core points
 *                         as in G13 (Section 3.2), merging of core grids by
 *                         union-find in ascending core-count order (the LDF
 *                         variant, Section 5.2) and border assignment.
 *                         Cross-checked against brute force by the tests.
 *
 * Readings where the paper is silent or loose (each one is listed in the
 * design notes):
 *   - |N_eps(p)| counts p itself and the boundary is inclusive:
 *     dist(p,q) <= eps  <=>  dist2(p,q) <= eps2 for integer coordinates,
 *     with eps2 = floor(eps^2) passed in by the caller.
 *   - Eq. 1 uses the real side eps/sqrt(d).  Here the side is the integer
 *     s = 1 + isqrt(eps2 / d), the largest s with d*(s-1)^2 <= eps2, so two
 *     integer points of one cell are within eps (the property Eq. 1 exists
 *     to give).  Labels do not depend on the side.
 *   - The neighbour test of Alg. 3 ("offset >= d", keys within +-ceil(sqrt d))
 *     is replaced by its exact integer form: cells a, b are neighbours iff
 *     sum_j gap_j^2 <= eps2 with gap_j = (|a_j-b_j|-1)*s+1 when a_j != b_j
 *     and 0 otherwise -- the smallest squared coordinate difference two
 *     integer points of the two cells can have.
 *   - Nei(g) contains g itself.
 *   - Canonical labels: a cluster's id is the smallest input index among its
 *     core points; a border point takes the smallest id among the clusters
 *     of the core points within eps; noise is -1.
 *   - FastMerging (Alg. 5) starts from the first point of s_i instead of a
 *     random one, and returns "no" as soon as a pruning empties a set.  The
 *     triangle-inequality pruning of Alg. 4 is evaluated exactly in integers;
 *     the angle-based pruning is left out (it only saves work, Thm. 2).
 *
 * All distances are exact int64 squared distances.  The caller must ensure
 * d * (max_j range_j)^2 < 2^62 (checked: returns ORACLE_ERANGE).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;
typedef uint64_t u64;

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ERANGE 2
#define ORACLE_ENOMEM 3

/* ------------------------------------------------------------------ */
/* Small helpers                                                        */
/* ------------------------------------------------------------------ */

/* Squared Euclidean distance of two integer points (Section 3.1). */
static i64 sqdist(const int32_t *a, const int32_t *b, int d)
{
    i64 s = 0;
    for (int j = 0; j < d; ++j) {
        i64 t = (i64)a[j] - (i64)b[j];
        s += t * t;
    }
    return s;
}

/* floor(sqrt(v)) by bisection on the answer: the largest r with r*r <= v. */
static u64 isqrt_u64(u64 v)
{
    u64 lo = 0, hi = 4294967296ull; /* (2^32)^2 > any u64 */
    while (hi - lo > 1) {
        u64 mid = lo + (hi - lo) / 2;
        if ((unsigned __int128)mid * mid <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* The integer cell side: largest s >= 1 with d*(s-1)^2 <= eps2 (Eq. 1). */
long long oracle_cell_side(long long eps2, int d)
{
    return 1 + (long long)isqrt_u64((u64)eps2 / (u64)d);
}

/* Sequential union-find over integers; the root of a set is its smallest
 * member (the larger root is always linked under the smaller one). */
static i64 uf_find(i64 *parent, i64 x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

static void uf_union(i64 *parent, i64 a, i64 b)
{
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b)
        return;
    if (a < b)
        parent[b] = a;
    else
        parent[a] = b;
}

/* Per-dimension min and max and the range check d * R^2 < 2^62. */
static int bounds(const int32_t *X, i64 n, int d, int32_t *mn, int32_t *mx)
{
    for (int j = 0; j < d; ++j) {
        mn[j] = X[j];
        mx[j] = X[j];
    }
    for (i64 i = 1; i < n; ++i)
        for (int j = 0; j < d; ++j) {
            int32_t v = X[i * d + j];
            if (v < mn[j]) mn[j] = v;
            if (v > mx[j]) mx[j] = v;
        }
    unsigned __int128 rmax = 0;
    for (int j = 0; j < d; ++j) {
        unsigned __int128 r = (unsigned __int128)((i64)mx[j] - (i64)mn[j]);
        if (r > rmax) rmax = r;
    }
    if ((unsigned __int128)d * rmax * rmax >= ((unsigned __int128)1 << 62))
        return ORACLE_ERANGE;
    return ORACLE_OK;
}

static int check_args(const int32_t *X, i64 n, int d, i64 eps2, int32_t minpts,
                      const int32_t *labels, const uint8_t *is_core)
{
    if (d < 1 || d > 8 || n < 0 || eps2 < 0 || minpts < 1)
        return ORACLE_EINVAL;
    if (n > 0 && (!X || !labels || !is_core))
        return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Brute force: the definitions written out (Section 3.1, Defs. 1-5)    */
/* ------------------------------------------------------------------ */

int oracle_bruteforce(const int32_t *X, long long n, int d, long long eps2, int minpts,
                      int32_t *labels, uint8_t *is_core)
{
    int rc = check_args(X, n, d, eps2, minpts, labels, is_core);
    if (rc != ORACLE_OK || n == 0)
        return rc;
    int32_t mn[8], mx[8];
    rc = bounds(X, n, d, mn, mx);
    if (rc != ORACLE_OK)
        return rc;

    /* Def. 1: p is core iff |N_eps(p)| >= MinPts, p itself counted. */
    for (i64 p = 0; p < n; ++p) {
        i64 cnt = 0;
        for (i64 q = 0; q < n; ++q)
            if (sqdist(X + p * d, X + q * d, d) <= eps2)
                cnt++;
        is_core[p] = (uint8_t)(cnt >= minpts);
    }

    /* Defs. 2-5: the core points of a cluster are a connected component of
     * the graph on core points with an edge iff dist <= eps.  The root of
     * each set is its smallest index, which is the canonical cluster id. */
    i64 *parent = (i64 *)malloc(sizeof(i64) * (size_t)n);
    if (!parent)
        return ORACLE_ENOMEM;
    for (i64 p = 0; p < n; ++p)
        parent[p] = p;
    for (i64 p = 0; p < n; ++p) {
        if (!is_core[p]) continue;
        for (i64 q = p + 1; q < n; ++q)
            if (is_core[q] && sqdist(X + p * d, X + q * d, d) <= eps2)
                uf_union(parent, p, q);
    }

    /* Core points take their component's id; a non-core point is a border
     * point of every cluster holding a core point within eps (it takes the
     * smallest such id) and noise (-1) when there is none. */
    for (i64 p = 0; p < n; ++p) {
        if (is_core[p]) {
            labels[p] = (int32_t)uf_find(parent, p);
            continue;
        }
        i64 best = -1;
        for (i64 q = 0; q < n; ++q) {
            if (!is_core[q] || sqdist(X + p * d, X + q * d, d) > eps2) continue;
            i64 c = uf_find(parent, q);
            if (best < 0 || c < best) best = c;
        }
        labels[p] = (int32_t)best;
    }
    free(parent);
    return ORACLE_OK;
}

/* Per-point core counts for a list of query points, by brute force over all n
 * points (Def. 1).  Used for sampled checks at sizes where the full O(n^2)
 * run is out of reach.  counts[k] = |N_eps(X[query[k]])|. */
int oracle_neighbor_counts(const int32_t *X, long long n, int d, long long eps2,
                           const long long *query, long long nq, long long *counts)
{
    if (d < 1 || d > 8 || n < 0 || eps2 < 0 || nq < 0)
        return ORACLE_EINVAL;
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 k = 0; k < nq; ++k) {
        const int32_t *p = X + query[k] * d;
        i64 cnt = 0;
        for (i64 q = 0; q < n; ++q)
            if (sqdist(p, X + q * d, d) <= eps2)
                cnt++;
        counts[k] = cnt;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Set minimum distance: Def. 7 and FastMerging (Alg. 4, Alg. 5)        */
/* ------------------------------------------------------------------ */

/* Def. 6/7 written out: is MinDist(A, B) <= eps?  Stops at the first pair. */
static int mindist_le_plain(const int32_t *A, i64 na, const int32_t *B, i64 nb, int d, i64 eps2)
{
    for (i64 a = 0; a < na; ++a)
        for (i64 b = 0; b < nb; ++b)
            if (sqdist(A + a * d, B + b * d, d) <= eps2)
                return 1;
    return 0;
}

/* Alg. 4, triangle-inequality part, in exact integers.  x is trivial when
 * dist(x,p) < dist(p,q) - eps.  With A = dist2(x,p), B = dist2(p,q) > eps2:
 *   sqrt(A) + sqrt(eps2) < sqrt(B)
 *   <=>  B - A - eps2 > 0  and  4*A*eps2 < (B - A - eps2)^2            */
static int triangle_trivial(i64 A, i64 B, i64 eps2)
{
    i64 t = B - A - eps2;
    if (t <= 0)
        return 0;
    unsigned __int128 lhs = (unsigned __int128)4 * (u64)A * (u64)eps2;
    unsigned __int128 rhs = (unsigned __int128)(u64)t * (u64)t;
    return lhs < rhs;
}

/* Alg. 4, angle part (Def. 8, Thm. 1): lambda is the largest
 *   lambda_y = arcsin(eps / dist(p,y)) + arccos(pq.py / (dist(p,q) dist(p,y)))
 * over the points y of the other set O (index list oidx, ocnt points); a
 * point x whose angle between pq and px exceeds lambda is trivial.  The
 * paper's reals are doubles here.  arcsin and arccos are 1/2-Hoelder
 * continuous (|acos a - acos b| <= pi * sqrt(|a - b| / 2)) and their
 * arguments are a few correctly rounded operations on exact integers
 * (relative error a few units of 2^-53), so the computed angles are within
 * 1e-7 of the exact ones: x is removed only when its angle exceeds lambda by
 * ANGLE_MARGIN, which keeps every removal one the exact test makes. */
#define ANGLE_MARGIN 1e-6

static i64 dot_from(const int32_t *o, const int32_t *u, const int32_t *v, int d)
{
    i64 s = 0;
    for (int j = 0; j < d; ++j)
        s += ((i64)u[j] - o[j]) * ((i64)v[j] - o[j]);
    return s;
}

static double clamp1(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

static double angle_lambda(const int32_t *O, const i64 *oidx, i64 ocnt, const int32_t *p, const int32_t *q,
                           int d, i64 eps2)
{
    const double a = sqrt((double)sqdist(p, q, d)), eps = sqrt((double)eps2);
    double lambda = 0.0;
    for (i64 k = 0; k < ocnt; ++k) {
        const int32_t *y = O + oidx[k] * d;
        const double b = sqrt((double)sqdist(p, y, d));
        const double ly = asin(clamp1(eps / b)) + acos(clamp1((double)dot_from(p, q, y, d) / (a * b)));
        if (ly > lambda) lambda = ly;
    }
    return lambda;
}

/* Alg. 4 on a set held as an index list: drop every x that the triangle test
 * (pivot p, nearest partner q at squared distance B) or the angle test
 * (bound lambda) shows to be trivial. */
static i64 prune_set(const int32_t *S, i64 *idx, i64 cnt, const int32_t *p, const int32_t *q, i64 B,
                     double lambda, int d, i64 eps2)
{
    i64 kept = 0;
    const double a = sqrt((double)B);
    for (i64 k = 0; k < cnt; ++k) {
        const int32_t *x = S + idx[k] * d;
        i64 A = sqdist(x, p, d);
        if (triangle_trivial(A, B, eps2))
            continue;
        if (A > 0) {
            const double theta = acos(clamp1((double)dot_from(p, q, x, d) / (a * sqrt((double)A))));
            if (lambda + ANGLE_MARGIN < theta)
                continue;
        }
        idx[kept++] = idx[k];
    }
    return kept;
}

/* Index (into idx) of the point of S nearest to p; ties go to the first. */
static i64 nearest(const int32_t *S, const i64 *idx, i64 cnt, const int32_t *p, int d, i64 *best2)
{
    i64 bk = 0, bd = -1;
    for (i64 k = 0; k < cnt; ++k) {
        i64 v = sqdist(S + idx[k] * d, p, d);
        if (bd < 0 || v < bd) {
            bd = v;
            bk = k;
        }
    }
    *best2 = bd;
    return bk;
}

/* Alg. 5 FastMerging: yes (1) iff MinDist(A, B) <= eps.  *iters receives the
 * number of repeat-loop rounds taken (kappa of Section 4.3.3). */
static int fastmerging(const int32_t *A, i64 na, const int32_t *B, i64 nb, int d, i64 eps2,
                       i64 *ia, i64 *ib, i64 *iters)
{
    for (i64 k = 0; k < na; ++k) ia[k] = k;
    for (i64 k = 0; k < nb; ++k) ib[k] = k;
    i64 ca = na, cb = nb, rounds = 0;
    const int32_t *p = A; /* first point of s_i */
    int ans = 0;
    while (ca > 0 && cb > 0) {
        rounds++;
        i64 dpq;
        i64 kq = nearest(B, ib, cb, p, d, &dpq);
        const int32_t *q = B + ib[kq] * d;
        if (dpq <= eps2) { ans = 1; break; }
        ca = prune_set(A, ia, ca, p, q, dpq, angle_lambda(B, ib, cb, p, q, d, eps2), d, eps2);
        if (ca == 0) break;
        i64 kp = nearest(A, ia, ca, q, d, &dpq);
        p = A + ia[kp] * d;
        if (dpq <= eps2) { ans = 1; break; }
        cb = prune_set(B, ib, cb, q, p, dpq, angle_lambda(A, ia, ca, q, p, d, eps2), d, eps2);
    }
    if (iters) *iters = rounds;
    return ans;
}

/* Exported for the tests: MinDist(A, B) <= eps by Def. 7 (mode 0) or by
 * FastMerging (mode 1).  A is [na][d], B is [nb][d]. */
int oracle_mindist_le(const int32_t *A, long long na, const int32_t *B, long long nb, int d,
                      long long eps2, int mode, long long *iters)
{
    if (d < 1 || d > 8 || na < 0 || nb < 0 || eps2 < 0)
        return -1;
    if (iters) *iters = 0;
    if (mode == 0)
        return mindist_le_plain(A, na, B, nb, d, eps2);
    i64 *ia = (i64 *)malloc(sizeof(i64) * (size_t)(na + 1));
    i64 *ib = (i64 *)malloc(sizeof(i64) * (size_t)(nb + 1));
    if (!ia || !ib) { free(ia); free(ib); return -1; }
    i64 rounds = 0;
    int r = fastmerging(A, na, B, nb, d, eps2, ia, ib, &rounds);
    if (iters) *iters = rounds;
    free(ia);
    free(ib);
    return r;
}

/* ------------------------------------------------------------------ */
/* Grid method (Section 4)                                              */
/* ------------------------------------------------------------------ */

/* Sort context for qsort (the oracle is not reentrant). */
static const i64 *g_cellc; /* [n][d] cell identifiers of the points */
static int g_d;

/* Lexicographic order of identifiers, dimension 1 first (Alg. 1), ties by
 * input index so the order inside a cell is the input order. */
static int cmp_points(const void *pa, const void *pb)
{
    i64 a = *(const i64 *)pa, b = *(const i64 *)pb;
    const i64 *ca = g_cellc + a * g_d, *cb = g_cellc + b * g_d;
    for (int j = 0; j < g_d; ++j) {
        if (ca[j] < cb[j]) return -1;
        if (ca[j] > cb[j]) return 1;
    }
    return (a < b) ? -1 : (a > b);
}

typedef struct {
    i64 n, C;
    int d;
    i64 s, r, eps2;
    i64 *order;      /* [n]   input index of the k-th point in grid order */
    int32_t *Xs;     /* [n][d] coordinates in grid order */
    i64 *start;      /* [C+1] first point of each non-empty grid */
    i64 *coord;      /* [C][d] identifiers of the non-empty grids */
    i64 *nei_start;  /* [C+1] CSR of Nei(g) */
    i64 *nei;        /* neighbour grid indices */
} grid_t;

static void grid_free(grid_t *g)
{
    free(g->order);
    free(g->Xs);
    free(g->start);
    free(g->coord);
    free(g->nei_start);
    free(g->nei);
    memset(g, 0, sizeof(*g));
}

/* Eq. 1 and Alg. 1: identifiers, lexicographic sort, non-empty grids. */
static int partition(grid_t *g, const int32_t *X, i64 n, int d, i64 eps2, const int32_t *mn)
{
    g->n = n;
    g->d = d;
    g->eps2 = eps2;
    g->s = oracle_cell_side(eps2, d);
    /* r: the largest |a_j - b_j| whose gap alone stays within eps
     * (the integer form of Alg. 3's key window +-ceil(sqrt d)). */
    i64 re = (i64)isqrt_u64((u64)eps2);
    g->r = (eps2 == 0) ? 0 : 1 + (re - 1) / g->s;

    i64 *cellc = (i64 *)malloc(sizeof(i64) * (size_t)(n * d));
    g->order = (i64 *)malloc(sizeof(i64) * (size_t)n);
    g->Xs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * d));
    if (!cellc || !g->order || !g->Xs) { free(cellc); return ORACLE_ENOMEM; }
    for (i64 i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j)
            cellc[i * d + j] = ((i64)X[i * d + j] - (i64)mn[j]) / g->s; /* Eq. 1 */
    for (i64 i = 0; i < n; ++i)
        g->order[i] = i;
    g_cellc = cellc;
    g_d = d;
    qsort(g->order, (size_t)n, sizeof(i64), cmp_points);

    /* Alg. 1: scan the sorted points and cut where the grid changes. */
    g->start = (i64 *)malloc(sizeof(i64) * (size_t)(n + 1));
    g->coord = (i64 *)malloc(sizeof(i64) * (size_t)(n * d));
    if (!g->start || !g->coord) { free(cellc); return ORACLE_ENOMEM; }
    i64 C = 0;
    for (i64 k = 0; k < n; ++k) {
        const i64 *ck = cellc + g->order[k] * d;
        int is_new = (k == 0);
        if (!is_new) {
            const i64 *cp = cellc + g->order[k - 1] * d;
            for (int j = 0; j < d; ++j)
                if (ck[j] != cp[j]) { is_new = 1; break; }
        }
        if (is_new) {
            g->start[C] = k;
            memcpy(g->coord + C * d, ck, sizeof(i64) * (size_t)d);
            C++;
        }
        memcpy(g->Xs + k * d, X + g->order[k] * d, sizeof(int32_t) * (size_t)d);
    }
    g->start[C] = n;
    g->C = C;
    free(cellc);
    return ORACLE_OK;
}

/* First grid index in [lo, hi) whose identifier in dimension j is >= v.
 * Grids in [lo, hi) share the first j identifiers, so dimension j is sorted
 * there: this range is the child list of one grid-tree node (Section 4.2.1). */
static i64 lower_dim(const grid_t *g, i64 lo, i64 hi, int j, i64 v)
{
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (g->coord[mid * g->d + j] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Alg. 3 NeighboringGridsQuery for grid `cell`, descending one dimension per
 * level.  [lo, hi) is the current node's subtree, `partial` the sum of the
 * gap terms so far (Eq. 2 in integer form).  Calls emit() per neighbour. */
typedef void (*emit_fn)(void *ctx, i64 nb);

static void query_rec(const grid_t *g, const i64 *gc, int j, i64 lo, i64 hi, i64 partial,
                      emit_fn emit, void *ctx)
{
    if (j == g->d) { /* leaf: exactly one grid */
        emit(ctx, lo);
        return;
    }
    i64 a = lower_dim(g, lo, hi, j, gc[j] - g->r);
    while (a < hi) {
        i64 key = g->coord[a * g->d + j];
        if (key > gc[j] + g->r) break;
        i64 b = lower_dim(g, a, hi, j, key + 1); /* children with this key */
        i64 delta = key > gc[j] ? key - gc[j] : gc[j] - key;
        i64 gap = delta == 0 ? 0 : (delta - 1) * g->s + 1;
        i64 off = partial + gap * gap;
        if (off <= g->eps2)
            query_rec(g, gc, j + 1, a, b, off, emit, ctx);
        a = b;
    }
}

typedef struct { i64 *buf; i64 cnt; } nbr_sink;

static void sink_count(void *ctx, i64 nb) { (void)nb; ((nbr_sink *)ctx)->cnt++; }
static void sink_store(void *ctx, i64 nb)
{
    nbr_sink *s = (nbr_sink *)ctx;
    s->buf[s->cnt++] = nb;
}

/* Nei(g) for every grid, stored as CSR (the paper keeps them in a vector). */
static int all_neighbors(grid_t *g)
{
    i64 C = g->C;
    g->nei_start = (i64 *)malloc(sizeof(i64) * (size_t)(C + 1));
    if (!g->nei_start) return ORACLE_ENOMEM;
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 c = 0; c < C; ++c) {
        nbr_sink s = {NULL, 0};
        query_rec(g, g->coord + c * g->d, 0, 0, C, 0, sink_count, &s);
        g->nei_start[c + 1] = s.cnt;
    }
    g->nei_start[0] = 0;
    for (i64 c = 0; c < C; ++c)
        g->nei_start[c + 1] += g->nei_start[c];
    g->nei = (i64 *)malloc(sizeof(i64) * (size_t)(g->nei_start[C] + 1));
    if (!g->nei) return ORACLE_ENOMEM;
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 c = 0; c < C; ++c) {
        nbr_sink s = {g->nei + g->nei_start[c], 0};
        query_rec(g, g->coord + c * g->d, 0, 0, C, 0, sink_store, &s);
    }
    return ORACLE_OK;
}

/* Exported for the tests: the non-empty grids and their neighbour lists.
 * Returns the number of grids C, or a negative oracle error.  Buffers may be
 * NULL to only query sizes: order[n], cell_start[C+1], cell_coord[C][d]
 * (identifiers), nei_start[C+1], nei[nei_start[C]].  *n_nei gets the total. */
long long oracle_grid_structure(const int32_t *X, long long n, int d, long long eps2,
                                long long *order, long long *cell_start, long long *cell_coord,
                                long long *nei_start, long long *nei, long long *n_nei)
{
    if (d < 1 || d > 8 || n <= 0 || eps2 < 0 || !X)
        return -ORACLE_EINVAL;
    int32_t mn[8], mx[8];
    int rc = bounds(X, n, d, mn, mx);
    if (rc != ORACLE_OK) return -rc;
    grid_t g;
    memset(&g, 0, sizeof(g));
    rc = partition(&g, X, n, d, eps2, mn);
    if (rc == ORACLE_OK) rc = all_neighbors(&g);
    if (rc != ORACLE_OK) { grid_free(&g); return -rc; }
    if (order) memcpy(order, g.order, sizeof(i64) * (size_t)n);
    if (cell_start) memcpy(cell_start, g.start, sizeof(i64) * (size_t)(g.C + 1));
    if (cell_coord) memcpy(cell_coord, g.coord, sizeof(i64) * (size_t)(g.C * d));
    if (nei_start) memcpy(nei_start, g.nei_start, sizeof(i64) * (size_t)(g.C + 1));
    if (nei) memcpy(nei, g.nei, sizeof(i64) * (size_t)g.nei_start[g.C]);
    if (n_nei) *n_nei = g.nei_start[g.C];
    i64 C = g.C;
    grid_free(&g);
    return C;
}

/* Order of core grids for the LDF merging: ascending core-point count, ties
 * by grid index. */
static const i64 *g_mcount;
static int cmp_by_m(const void *pa, const void *pb)
{
    i64 a = *(const i64 *)pa, b = *(const i64 *)pb;
    if (g_mcount[a] != g_mcount[b]) return g_mcount[a] < g_mcount[b] ? -1 : 1;
    return (a < b) ? -1 : (a > b);
}

/* GriT-DBSCAN(-LDF) on the CPU.  merge_mode 0 decides each merge by Def. 7
 * directly, merge_mode 1 by FastMerging (Alg. 5).  stats (may be NULL, else
 * 20 entries) receives {C, merge tests run, max FastMerging rounds, core
 * grids}, then FastMerging calls by rounds 1..15 and >= 16. */
int oracle_grid(const int32_t *X, long long n, int d, long long eps2, int minpts,
                int32_t *labels, uint8_t *is_core, int merge_mode, long long *stats)
{
    int rc = check_args(X, n, d, eps2, minpts, labels, is_core);
    if (rc != ORACLE_OK || n == 0) return rc;
    int32_t mn[8], mx[8];
    rc = bounds(X, n, d, mn, mx);
    if (rc != ORACLE_OK) return rc;

    /* Step 1: partitioning (Alg. 1), grid tree and Nei(g) (Alg. 2-3). */
    grid_t g;
    memset(&g, 0, sizeof(g));
    rc = partition(&g, X, n, d, eps2, mn);
    if (rc == ORACLE_OK) rc = all_neighbors(&g);
    if (rc != ORACLE_OK) { grid_free(&g); return rc; }
    const i64 C = g.C;

    /* Step 2: core points as in G13 (Section 3.2).  A grid holding at least
     * MinPts points has only core points (its diameter is <= eps); in the
     * others each point counts its neighbours in Nei(g) up to MinPts. */
    uint8_t *core_s = (uint8_t *)calloc((size_t)n, 1); /* grid order */
    i64 *m = (i64 *)calloc((size_t)C, sizeof(i64));    /* core points per grid */
    if (!core_s || !m) { free(core_s); free(m); grid_free(&g); return ORACLE_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 c = 0; c < C; ++c) {
        i64 b = g.start[c], e = g.start[c + 1];
        if (e - b >= minpts) {
            for (i64 k = b; k < e; ++k) core_s[k] = 1;
            m[c] = e - b;
            continue;
        }
        i64 mc = 0;
        for (i64 k = b; k < e; ++k) {
            i64 cnt = 0;
            for (i64 t = g.nei_start[c]; t < g.nei_start[c + 1] && cnt < minpts; ++t) {
                i64 c2 = g.nei[t];
                for (i64 k2 = g.start[c2]; k2 < g.start[c2 + 1] && cnt < minpts; ++k2)
                    if (sqdist(g.Xs + k * d, g.Xs + k2 * d, d) <= eps2)
                        cnt++;
            }
            core_s[k] = (uint8_t)(cnt >= minpts);
            mc += core_s[k];
        }
        m[c] = mc;
    }

    /* Core point sets s_i, packed per grid (Section 4.3.1). */
    i64 *cstart = (i64 *)malloc(sizeof(i64) * (size_t)(C + 1));
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * d) + 4);
    i64 *sidx = (i64 *)malloc(sizeof(i64) * (size_t)(n + 1)); /* grid-order index */
    i64 *parent = (i64 *)malloc(sizeof(i64) * (size_t)(C + 1));
    i64 *ord = (i64 *)malloc(sizeof(i64) * (size_t)(C + 1));
    i64 *ia = (i64 *)malloc(sizeof(i64) * (size_t)(n + 1));
    i64 *ib = (i64 *)malloc(sizeof(i64) * (size_t)(n + 1));
    if (!cstart || !S || !sidx || !parent || !ord || !ia || !ib) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    cstart[0] = 0;
    for (i64 c = 0; c < C; ++c) {
        i64 w = cstart[c];
        for (i64 k = g.start[c]; k < g.start[c + 1]; ++k)
            if (core_s[k]) {
                memcpy(S + w * d, g.Xs + k * d, sizeof(int32_t) * (size_t)d);
                sidx[w] = k;
                w++;
            }
        cstart[c + 1] = w;
    }

    /* Step 3: merging (GriT-DBSCAN-LDF, Section 5.2).  Core grids are visited
     * in ascending order of core-point count; for each core grid in Nei(g_i)
     * the pair is skipped when union-find already joins them, else merged
     * when MinDist(s_i, s_j) <= eps (Def. 6). */
    i64 ncore = 0, tests = 0, max_rounds = 0;
    if (stats)
        for (int t = 4; t < 20; ++t) stats[t] = 0;
    for (i64 c = 0; c < C; ++c) {
        parent[c] = c;
        if (m[c] > 0) ord[ncore++] = c;
    }
    g_mcount = m;
    qsort(ord, (size_t)ncore, sizeof(i64), cmp_by_m);
    for (i64 t = 0; t < ncore; ++t) {
        i64 ci = ord[t];
        for (i64 u = g.nei_start[ci]; u < g.nei_start[ci + 1]; ++u) {
            i64 cj = g.nei[u];
            if (cj == ci || m[cj] == 0) continue;
            if (uf_find(parent, ci) == uf_find(parent, cj)) continue;
            const int32_t *A = S + cstart[ci] * d, *B = S + cstart[cj] * d;
            i64 na = m[ci], nb = m[cj], rounds = 0;
            int yes = merge_mode == 0 ? mindist_le_plain(A, na, B, nb, d, eps2)
                                      : fastmerging(A, na, B, nb, d, eps2, ia, ib, &rounds);
            tests++;
            if (rounds > max_rounds) max_rounds = rounds;
            if (stats && merge_mode == 1) stats[4 + (rounds < 16 ? rounds : 16) - 1]++;
            if (yes) uf_union(parent, ci, cj);
        }
    }

    /* Cluster ids: smallest input index over the core points of each set. */
    {
        i64 *cid = ia; /* reuse: cid per root grid, -1 when unset */
        for (i64 c = 0; c < C; ++c) cid[c] = -1;
        for (i64 c = 0; c < C; ++c) {
            if (m[c] == 0) continue;
            i64 root = uf_find(parent, c);
            for (i64 w = cstart[c]; w < cstart[c + 1]; ++w) {
                i64 orig = g.order[sidx[w]];
                if (cid[root] < 0 || orig < cid[root]) cid[root] = orig;
            }
        }
        for (i64 c = 0; c < C; ++c) ib[c] = (m[c] > 0) ? cid[uf_find(parent, c)] : -1;

        /* Step 4: non-core points (Section 4.4): border if a core point lies
         * within eps, taking the smallest adjacent cluster id; else noise. */
#pragma omp parallel for schedule(dynamic, 16)
        for (i64 c = 0; c < C; ++c) {
            for (i64 k = g.start[c]; k < g.start[c + 1]; ++k) {
                i64 orig = g.order[k];
                is_core[orig] = core_s[k];
                if (core_s[k]) {
                    labels[orig] = (int32_t)ib[c];
                    continue;
                }
                i64 best = -1;
                for (i64 u = g.nei_start[c]; u < g.nei_start[c + 1]; ++u) {
                    i64 c2 = g.nei[u];
                    if (m[c2] == 0) continue;
                    if (best >= 0 && ib[c2] >= best) continue;
                    for (i64 w = cstart[c2]; w < cstart[c2 + 1]; ++w)
                        if (sqdist(g.Xs + k * d, S + w * d, d) <= eps2) {
                            best = ib[c2];
                            break;
                        }
                }
                labels[orig] = (int32_t)best;
            }
        }
    }
    if (stats) {
        stats[0] = C;
        stats[1] = tests;
        stats[2] = max_rounds;
        stats[3] = ncore;
    }
    rc = ORACLE_OK;
done:
    free(core_s);
    free(m);
    free(cstart);
    free(S);
    free(sidx);
    free(parent);
    free(ord);
    free(ia);
    free(ib);
    grid_free(&g);
    return rc;
}

/* Number of OpenMP threads the oracle runs with. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
