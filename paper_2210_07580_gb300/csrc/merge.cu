// Merging core grids (Section 4.3, Def. 6-7): two neighbouring core grids
// belong to one cluster iff some core point of one is within eps of some core
// point of the other.  The grids are joined with a lock-free union-find, as
// in the LDF variant (Section 5.2): a pair whose grids are already in one set
// is skipped before any distance is computed.
#include "gd_internal.cuh"

namespace gd {

// ------------------------------------------------- core points per grid

// m_c (core points per grid) and reset of the grid's core bounding box.
__global__ void core_count_kernel(int minpts, int d, const unsigned char* __restrict__ core_s,
                                  const int* __restrict__ cell_start, int C, int* __restrict__ core_cnt,
                                  int* __restrict__ bbox) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int b = cell_start[c], e = cell_start[c + 1];
    int m = e - b;
    if (m < minpts) {
        m = 0;
        for (int k = b; k < e; ++k) m += core_s[k];
    }
    core_cnt[c] = m;
    for (int j = 0; j < d; ++j) {
        bbox[(long long)c * 2 * d + j] = 0x7fffffff;
        bbox[(long long)c * 2 * d + d + j] = (int)0x80000000;
    }
}

cudaError_t launch_core_count(const Params& p, const unsigned char* core_s, const int* cell_start, int C,
                              int* core_cnt, int* bbox, cudaStream_t st) {
    core_count_kernel<<<(C + 255) / 256, 256, 0, st>>>(p.minpts, p.d, core_s, cell_start, C, core_cnt, bbox);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Core points of each grid packed contiguously (s_i of Section 4.3.1), one
// thread per point in grid order, and the bounding box of each grid's core
// points: a warp's lanes hold consecutive points, so the lanes of one grid
// form a run; the run is min/max-reduced with shuffles and its first lane
// applies one atomic per dimension.
__global__ void __launch_bounds__(256) core_pack_kernel(Params p, const int* __restrict__ Xs,
                                                        const unsigned char* __restrict__ core_s,
                                                        const int* __restrict__ pt_cell,
                                                        const int* __restrict__ cell_start,
                                                        const int* __restrict__ core_start, int* __restrict__ Xc,
                                                        int* __restrict__ bbox) {
    const int lane = lane_id(), d = p.d, dp = p.dp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = ((long long)p.n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < p.n;
        const int c = valid ? pt_cell[i] : -1 - lane;
        const bool core = valid && core_s[i];
        int x[kMaxD];
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) x[j] = (core && j < dp) ? Xs[i * dp + j] : 0;
        if (core) {
            const int b = cell_start[c];
            long long pos;
            if (cell_start[c + 1] - b >= p.minpts) {
                pos = core_start[c] + (i - b);
            } else {
                int r = 0;
                for (long long k = b; k < i; ++k) r += core_s[k];
                pos = core_start[c] + r;
            }
#pragma unroll
            for (int j = 0; j < kMaxD; ++j)
                if (j < dp) Xc[pos * dp + j] = x[j];
        }
        const unsigned peers = __match_any_sync(kFull, c);
        const bool leader = lane == __ffs(peers) - 1;
        const bool any_core = (__ballot_sync(kFull, core) & peers) != 0;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            if (j >= d) break;
            int lo = core ? x[j] : 0x7fffffff, hi = core ? x[j] : (int)0x80000000;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int olo = __shfl_down_sync(kFull, lo, o);
                const int ohi = __shfl_down_sync(kFull, hi, o);
                const int oc = __shfl_down_sync(kFull, c, o);
                if (lane + o < 32 && oc == c) {
                    lo = min(lo, olo);
                    hi = max(hi, ohi);
                }
            }
            if (leader && any_core) {
                atomicMin(bbox + (long long)c * 2 * d + j, lo);
                atomicMax(bbox + (long long)c * 2 * d + d + j, hi);
            }
        }
    }
}

cudaError_t launch_core_pack(const Params& p, const int* Xs, const unsigned char* core_s, const int* pt_cell,
                             const int* cell_start, const int* core_start, int* Xc, int* bbox, cudaStream_t st) {
    long long blocks = ((long long)p.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    core_pack_kernel<<<(int)blocks, 256, 0, st>>>(p, Xs, core_s, pt_cell, cell_start, core_start, Xc, bbox);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Largest grid (bounds the per-block pruning bitmaps of the merge).
__global__ void cell_max_kernel(const int* __restrict__ cell_start, int C, int* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    int m = c < C ? cell_start[c + 1] - cell_start[c] : 0;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if (lane_id() == 0 && m > 0) atomicMax(out, m);
}

cudaError_t launch_cell_max(const int* cell_start, int C, int* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    cell_max_kernel<<<(C + 255) / 256, 256, 0, st>>>(cell_start, C, out);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// -------------------------------------------------------- candidate pairs
// Pairs (i, j) of core grids with j in Nei(i) and j > i, in two waves:
// touching grids (identifiers differ by at most 1 in every dimension) first,
// all others after them.  Touching core grids are nearly always merged, so
// once the first wave has joined them the union-find precheck skips most of
// the second wave (the LDF idea of Section 5.2: establish clusters early so
// that later checks can be skipped).

template <bool FILL>
__global__ void pair_kernel(int d, const int* __restrict__ nbr_start, const int* __restrict__ nbr,
                            const int* __restrict__ core_start, const int* __restrict__ coord, int C,
                            int* __restrict__ t_cnt_or_start, int* __restrict__ f_cnt_or_start,
                            int2* __restrict__ pairs) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int kt = 0, kf = 0;
    if (core_start[c + 1] > core_start[c]) {
        int2* out_t = nullptr;
        int2* out_f = nullptr;
        if (FILL) {
            out_t = pairs + t_cnt_or_start[c];
            out_f = pairs + t_cnt_or_start[C] + f_cnt_or_start[c];
        }
        int g[kMaxD];
        for (int j = 0; j < d; ++j) g[j] = coord[(long long)c * d + j];
        for (int t = nbr_start[c]; t < nbr_start[c + 1]; ++t) {
            const int j2 = nbr[t];
            if (j2 <= c || core_start[j2 + 1] == core_start[j2]) continue;
            bool touching = true;
            for (int j = 0; j < d; ++j) {
                const int dl = coord[(long long)j2 * d + j] - g[j];
                if (dl > 1 || dl < -1) touching = false;
            }
            if (touching) {
                if (FILL) out_t[kt] = make_int2(c, j2);
                kt++;
            } else {
                if (FILL) out_f[kf] = make_int2(c, j2);
                kf++;
            }
        }
    }
    if (!FILL) {
        t_cnt_or_start[c] = kt;
        f_cnt_or_start[c] = kf;
    }
}

cudaError_t launch_pair_count(const Params& p, const int* nbr_start, const int* nbr, const int* core_start,
                              const int* cell_coord, int C, int* t_count, int* f_count, cudaStream_t st) {
    pair_kernel<false><<<(C + 255) / 256, 256, 0, st>>>(p.d, nbr_start, nbr, core_start, cell_coord, C, t_count,
                                                        f_count, nullptr);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_pair_fill(const Params& p, const int* nbr_start, const int* nbr, const int* core_start,
                             const int* cell_coord, int C, const int* t_start, const int* f_start, int2* pairs,
                             cudaStream_t st) {
    pair_kernel<true><<<(C + 255) / 256, 256, 0, st>>>(p.d, nbr_start, nbr, core_start, cell_coord, C,
                                                       const_cast<int*>(t_start), const_cast<int*>(f_start), pairs);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// range[0..1] = touching pairs, range[2..3] = the others; hard counters reset.
__global__ void merge_ranges_kernel(const int* __restrict__ t_start, const int* __restrict__ f_start, int C,
                                   int* range, int* hard_cnt) {
    if (threadIdx.x == 0) {
        const int nt = t_start[C], nf = f_start[C];
        range[0] = 0;
        range[1] = nt;
        range[2] = nt;
        range[3] = nt + nf;
        hard_cnt[0] = 0;
        hard_cnt[1] = 0;
    }
}

cudaError_t launch_merge_ranges(const int* t_start, const int* f_start, int C, int* range, int* hard_cnt,
                                cudaStream_t st) {
    merge_ranges_kernel<<<1, 32, 0, st>>>(t_start, f_start, C, range, hard_cnt);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------ union-find
// Of two roots, the one with the lower priority is linked under the other
// (atomicCAS on the root), and finds halve paths with plain stores: every
// stored parent is an ancestor, so concurrent halving never breaks a path.
// The priority is a fixed bijective hash of the index, not the index itself:
// grids are in lexicographic order, so index-ordered linking builds long
// chains along clusters, while a random-looking order keeps trees shallow.
// (Cluster ids do not depend on which grid ends up the root.)

__global__ void uf_init_kernel(int* parent, int C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) parent[c] = c;
}

cudaError_t launch_uf_init(int* parent, int C, cudaStream_t st) {
    uf_init_kernel<<<(C + 255) / 256, 256, 0, st>>>(parent, C);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Returns false if the retry cap was hit.
__device__ __forceinline__ bool uf_union(int* parent, int a, int b) {
    for (int it = 0; it < kMaxUfRetries; ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        if (uf_priority(a) < uf_priority(b)) {
            const int t = a;
            a = b;
            b = t;
        }
        // link root b (lower priority) under root a
        if (atomicCAS(parent + b, b, a) == b) return true;
    }
    return false;
}


// Both box tests of a candidate pair.  Returns 0 (no: boxes farther than
// eps), 1 (yes: the boxes are within eps even at their farthest corners) or
// -1 (undecided).
template <int D>
__device__ __forceinline__ int box_decision(const int* bi, const int* bj, long long eps2) {
    long long mind = 0, maxd = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int ilo = bi[j], ihi = bi[D + j], jlo = bj[j], jhi = bj[D + j];
        long long gap = 0;
        if (jlo > ihi) gap = (long long)jlo - ihi;
        else if (ilo > jhi) gap = (long long)ilo - jhi;
        mind += gap * gap;
        const long long a = (long long)jhi - ilo, b = (long long)ihi - jlo;
        const long long far = a > b ? a : b;
        maxd += far * far;
    }
    if (mind > eps2) return 0;
    if (maxd <= eps2) return 1;
    return -1;
}

// ----------------------------------------------------- the warp-level test
// One warp per candidate pair of a wave:
//   1. skip if the grids are already in one set;
//   2. the two box tests;
//   3. the exact test over core points in 32 x 32 tiles (lane l holds a point
//      of s_j, points of s_i are broadcast), stopping at the first pair within
//      eps.  Pairs of two small sets (both at most kSmallSet points) are
//      decided here in full (at most 16 tiles); any other pair gets `budget`
//      diagonal tiles (distinct chunks of both sets), which finds a witness
//      for nearly every pair that has many, and is otherwise handed to the
//      block-level FastMerging kernel -- in particular a few points against
//      thousands, where one scan of the large set usually decides.
constexpr int kSmallSet = 128;

template <int D, int DP>
__global__ void __launch_bounds__(256) merge_warp_kernel(Params p, const int2* __restrict__ pairs,
                                                         const int* __restrict__ range,
                                                         const int* __restrict__ Xc,
                                                         const int* __restrict__ core_start,
                                                         const int* __restrict__ bbox, int* parent,
                                                         unsigned* status, int2* __restrict__ hard,
                                                         int* __restrict__ hard_cnt, int budget) {
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long eps2 = p.eps2;
    const int lo = range[0], hi = range[1];
    for (long long w = lo + (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < hi; w += warps) {
        const int2 pr = pairs[w];
        int same = 0;
        if (lane == 0) {
            const int ra = uf_find(parent, pr.x), rb = uf_find(parent, pr.y);
            if (ra < 0 || rb < 0) atomicOr(status, kDevTimeout);
            same = ra == rb;
        }
        if (__shfl_sync(kFull, same, 0)) continue;

        const int dec = box_decision<D>(bbox + (long long)pr.x * 2 * D, bbox + (long long)pr.y * 2 * D, eps2);
        bool yes = dec == 1;
        bool handed = false;
        if (dec < 0) {
            const int ai = core_start[pr.x], mi = core_start[pr.x + 1] - ai;
            const int aj = core_start[pr.y], mj = core_start[pr.y + 1] - aj;
            const int na = (mi + 31) >> 5, nb = (mj + 31) >> 5;
            const long long tiles = (long long)na * nb;
            const bool exhaustive = mi <= kSmallSet && mj <= kSmallSet;
            const long long limit = exhaustive ? tiles : (tiles < budget ? tiles : budget);
            for (long long t = 0; t < limit; ++t) {
                const int ta = exhaustive ? (int)(t / nb) : (int)(t % na);
                const int tb = exhaustive ? (int)(t % nb) : (int)(t % nb);
                const int a0 = ta << 5, b0 = tb << 5;
                const int ca = min(32, mi - a0);
                int P[D], Q[D];
                const bool vq = b0 + lane < mj;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    P[j] = lane < ca ? Xc[(long long)(ai + a0 + lane) * DP + j] : 0;
                    Q[j] = vq ? Xc[(long long)(aj + b0 + lane) * DP + j] : 0;
                }
                bool hit = false;
                for (int u = 0; u < ca; ++u) {
                    int pt[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) pt[j] = __shfl_sync(kFull, P[j], u);
                    hit |= vq && sqdist<D>(pt, Q) <= eps2;
                }
                if (__any_sync(kFull, hit)) {
                    yes = true;
                    break;
                }
            }
            handed = !yes && limit < tiles;
        }
        if (lane == 0) {
            if (yes) {
                if (!uf_union(parent, pr.x, pr.y)) atomicOr(status, kDevTimeout);
            } else if (handed) {
                hard[lo + atomicAdd(hard_cnt, 1)] = pr;
            }
        }
    }
}

// ------------------------------------------------- FastMerging, per block
// Alg. 5 for one pair per block, exact:
//   p starts at the point of s_i nearest to the centre of s_j's box;
//   q = argmin over s_j of dist(p, .); yes if dist(p, q) <= eps;
//   otherwise prune s_i around p (Alg. 4, triangle part: x goes when
//   dist(x, p) < dist(p, q) - eps, decided in integers), take p = argmin over
//   the rest of s_i of dist(., q), test, prune s_j around q, and repeat;
//   no as soon as a pruning empties a set (Thm. 2: only points with no
//   partner within eps are ever removed).
// Each pruning is fused with the next argmin, so a round is two passes over
// the live points.  Every round removes p from s_i and q from s_j, so the
// loop ends after at most min(m_i, m_j) rounds.  The live sets are bitmaps
// (one word per 32 points) in the block's slice of global scratch.
// The angle-based part of Alg. 4 is not used: it needs arcsin/arccos, and
// only saves work.

__device__ __forceinline__ bool triangle_trivial(long long A, long long B, long long eps2) {
    // x is trivial iff sqrt(A) + sqrt(eps2) < sqrt(B)
    //   <=> B - A - eps2 > 0 and 4*A*eps2 < (B - A - eps2)^2   (B > eps2)
    const long long t = B - A - eps2;
    if (t <= 0) return false;
    const unsigned __int128 lhs = (unsigned __int128)4 * (unsigned long long)A * (unsigned long long)eps2;
    const unsigned __int128 rhs = (unsigned __int128)(unsigned long long)t * (unsigned long long)t;
    return lhs < rhs;
}

struct BestPt {
    long long d;
    int i;
};

__device__ __forceinline__ BestPt better(BestPt a, BestPt b) {
    if (b.d < a.d || (b.d == a.d && b.i < a.i)) return b;
    return a;
}

constexpr int kFmBlock = 256;
constexpr int kFmWarps = kFmBlock / 32;

// Block-wide argmin and live count; every thread gets the result.
__device__ __forceinline__ BestPt block_best(BestPt v, int cnt, BestPt* sb, int* sc, int* total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        BestPt u;
        u.d = __shfl_down_sync(kFull, v.d, o);
        u.i = __shfl_down_sync(kFull, v.i, o);
        v = better(v, u);
        cnt += __shfl_down_sync(kFull, cnt, o);
    }
    if (lane == 0) {
        sb[warp] = v;
        sc[warp] = cnt;
    }
    __syncthreads();
    BestPt r = sb[0];
    int c = sc[0];
#pragma unroll
    for (int w = 1; w < kFmWarps; ++w) {
        r = better(r, sb[w]);
        c += sc[w];
    }
    *total = c;
    __syncthreads();
    return r;
}

template <int D, int DP>
__device__ __forceinline__ void load_pt(const int* __restrict__ S, int k, int* x) {
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = S[(long long)k * DP + j];
}

template <int D>
__device__ __forceinline__ long long sqdist_ll(const int* a, const long long* b) {
    long long s = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const long long t = (long long)a[j] - b[j];
        s += t * t;
    }
    return s;
}

// One pass over a live set S (bitmap `live`, m points): optionally prune
// around pivot `piv` with nearest-distance B, and return the argmin of the
// distance to `tgt` over the points kept, plus their count.
template <int D, int DP, bool PRUNE>
__device__ BestPt fm_pass(const int* __restrict__ S, int m, unsigned* live, const long long* piv, long long B,
                          const long long* tgt, long long eps2, BestPt* sb, int* sc, int* count) {
    const int lane = lane_id();
    BestPt best{0x7fffffffffffffffll, 0x7fffffff};
    int cnt = 0;
    for (int base = 0; base < m; base += kFmBlock) {
        const int k = base + threadIdx.x;
        // the 32 lanes of a warp hold one bitmap word's 32 points; lane 0 has
        // the lowest, so the word exists whenever lane 0 is inside the set
        const unsigned word = k < m ? live[k >> 5] : 0u;
        bool alive = (word >> lane) & 1u;
        int x[D];
        if (alive) {
            load_pt<D, DP>(S, k, x);
            if (PRUNE && triangle_trivial(sqdist_ll<D>(x, piv), B, eps2)) alive = false;
        }
        if (PRUNE) {
            const unsigned nw = __ballot_sync(kFull, alive);
            if (lane == 0 && k < m && nw != word) live[k >> 5] = nw;
        }
        if (alive) {
            cnt++;
            best = better(best, BestPt{sqdist_ll<D>(x, tgt), k});
        }
    }
    return block_best(best, cnt, sb, sc, count);
}

template <int D, int DP>
__global__ void __launch_bounds__(kFmBlock) merge_block_kernel(Params p, const int2* __restrict__ hard,
                                                               const int* __restrict__ range,
                                                               const int* __restrict__ hard_cnt,
                                                               const int* __restrict__ Xc,
                                                               const int* __restrict__ core_start,
                                                               const int* __restrict__ bbox, int* parent,
                                                               unsigned* status, unsigned* scratch, int wpb) {
    __shared__ BestPt sb[kFmWarps];
    __shared__ int sc[kFmWarps];
    __shared__ int s_same;
    const long long eps2 = p.eps2;
    const int lo = range[0], nh = *hard_cnt;
    unsigned* live_a = scratch + (long long)blockIdx.x * 2 * wpb;
    unsigned* live_b = live_a + wpb;
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int2 pr = hard[lo + h];
        if (threadIdx.x == 0) {
            const int ra = uf_find(parent, pr.x), rb = uf_find(parent, pr.y);
            if (ra < 0 || rb < 0) atomicOr(status, kDevTimeout);
            s_same = ra == rb;
        }
        __syncthreads();
        const bool same = s_same;
        __syncthreads();
        if (same) continue;

        // s_i is the smaller set: each round removes at least its pivot, and
        // a small set is usually emptied by the first pruning
        int gi = pr.x, gj = pr.y;
        if (core_start[gi + 1] - core_start[gi] > core_start[gj + 1] - core_start[gj]) {
            gi = pr.y;
            gj = pr.x;
        }
        const int* A = Xc + (long long)core_start[gi] * DP;
        const int* B = Xc + (long long)core_start[gj] * DP;
        const int ma = core_start[gi + 1] - core_start[gi];
        const int mb = core_start[gj + 1] - core_start[gj];
        const int wa = (ma + 31) >> 5, wb = (mb + 31) >> 5;
        for (int w = threadIdx.x; w < wa; w += kFmBlock)
            live_a[w] = (w < wa - 1 || (ma & 31) == 0) ? 0xffffffffu : ((1u << (ma & 31)) - 1u);
        for (int w = threadIdx.x; w < wb; w += kFmBlock)
            live_b[w] = (w < wb - 1 || (mb & 31) == 0) ? 0xffffffffu : ((1u << (mb & 31)) - 1u);
        __syncthreads();

        long long piv[D], tgt[D];
        const int* bj = bbox + (long long)gj * 2 * D;
#pragma unroll
        for (int j = 0; j < D; ++j) tgt[j] = ((long long)bj[j] + bj[D + j]) / 2;
        int cnt;
        BestPt bp = fm_pass<D, DP, false>(A, ma, live_a, nullptr, 0, tgt, eps2, sb, sc, &cnt);
        int px[D];
        load_pt<D, DP>(A, bp.i, px);
#pragma unroll
        for (int j = 0; j < D; ++j) piv[j] = px[j];
        BestPt bq = fm_pass<D, DP, false>(B, mb, live_b, nullptr, 0, piv, eps2, sb, sc, &cnt);
        bool yes = false;
        for (int round = 0; round <= ma + mb; ++round) {
            if (bq.d <= eps2) {
                yes = true;
                break;
            }
            // prune s_i around p (nearest in s_j at distance^2 bq.d), then p' = argmin over s_i of dist(., q)
            int qx[D];
            load_pt<D, DP>(B, bq.i, qx);
            long long qv[D];
#pragma unroll
            for (int j = 0; j < D; ++j) qv[j] = qx[j];
            bp = fm_pass<D, DP, true>(A, ma, live_a, piv, bq.d, qv, eps2, sb, sc, &cnt);
            if (cnt == 0) break;
            if (bp.d <= eps2) {
                yes = true;
                break;
            }
            load_pt<D, DP>(A, bp.i, px);
#pragma unroll
            for (int j = 0; j < D; ++j) piv[j] = px[j];
            // prune s_j around q (nearest in s_i at distance^2 bp.d), then q' = argmin over s_j of dist(p', .)
            bq = fm_pass<D, DP, true>(B, mb, live_b, qv, bp.d, piv, eps2, sb, sc, &cnt);
            if (cnt == 0) break;
        }
        if (yes && threadIdx.x == 0) {
            if (!uf_union(parent, pr.x, pr.y)) atomicOr(status, kDevTimeout);
        }
        __syncthreads();
    }
}

// Between the waves: point every grid at its root, so that the second wave's
// precheck costs two loads per pair.
__global__ void uf_flatten_kernel(int* parent, int C, unsigned* status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int r = uf_find(parent, c);
    if (r < 0)
        atomicOr(status, kDevTimeout);
    else if (r != c)
        parent[c] = r;
}

cudaError_t launch_uf_flatten(int* parent, int C, unsigned* status, cudaStream_t st) {
    uf_flatten_kernel<<<(C + 255) / 256, 256, 0, st>>>(parent, C, status);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

template <int D>
static void merge_waves_launch(const Params& p, int wave, const int2* pairs, const int* range, int max_pairs,
                               const int* Xc, const int* core_start, const int* bbox, int* parent, unsigned* status,
                               int2* hard, int* hard_cnt, unsigned* scratch, int wpb, int fm_blocks,
                               cudaStream_t st) {
    constexpr int DP = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
    long long blocks = ((long long)max_pairs * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    const int* r = range + 2 * wave;
    merge_warp_kernel<D, DP><<<(int)blocks, 256, 0, st>>>(p, pairs, r, Xc, core_start, bbox, parent, status, hard,
                                                          hard_cnt + wave, 2);
    GD_COUNT_LAUNCH();
    merge_block_kernel<D, DP><<<fm_blocks, kFmBlock, 0, st>>>(p, hard, r, hard_cnt + wave, Xc, core_start, bbox,
                                                              parent, status, scratch, wpb);
    GD_COUNT_LAUNCH();
}

int merge_fm_blocks() { return 152 * 8; }

cudaError_t launch_merge_wave(const Params& p, int wave, const int2* pairs, const int* range, int max_pairs,
                              const int* Xc, const int* core_start, const int* bbox, int* parent, unsigned* status,
                              int2* hard, int* hard_cnt, unsigned* scratch, int wpb, int fm_blocks, cudaStream_t st) {
    if (max_pairs <= 0) return cudaSuccess;
    const int fb = fm_blocks;
    switch (p.d) {
#define GD_WAVE(DD) \
    case DD: merge_waves_launch<DD>(p, wave, pairs, range, max_pairs, Xc, core_start, bbox, parent, status, hard, hard_cnt, scratch, wpb, fb, st); break;
        GD_WAVE(1) GD_WAVE(2) GD_WAVE(3) GD_WAVE(4) GD_WAVE(5) GD_WAVE(6) GD_WAVE(7)
        default: merge_waves_launch<8>(p, wave, pairs, range, max_pairs, Xc, core_start, bbox, parent, status, hard,
                                       hard_cnt, scratch, wpb, fb, st); break;
#undef GD_WAVE
    }
    return cudaGetLastError();
}

}  // namespace gd
