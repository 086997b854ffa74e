// Merging core grids (Section 4.3, Def. 6-7): two neighbouring core grids
// belong to one cluster iff some core point of one is within eps of some core
// point of the other.  The grids are joined with a lock-free union-find, as
// in the LDF variant (Section 5.2): a pair whose grids are already in one set
// is skipped before any distance is computed.
#include "gd_internal.cuh"

namespace gd {

// ------------------------------------------------- core points per grid

__global__ void core_count_kernel(int minpts, const unsigned char* __restrict__ core_s,
                                  const int* __restrict__ cell_start, int C, int* __restrict__ core_cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int b = cell_start[c], e = cell_start[c + 1];
    int m = e - b;
    if (m < minpts) {
        m = 0;
        for (int k = b; k < e; ++k) m += core_s[k];
    }
    core_cnt[c] = m;
}

cudaError_t launch_core_count(const Params& p, const unsigned char* core_s, const int* cell_start, int C,
                              int* core_cnt, cudaStream_t st) {
    core_count_kernel<<<(C + 255) / 256, 256, 0, st>>>(p.minpts, core_s, cell_start, C, core_cnt);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Core points of each grid packed contiguously (s_i of Section 4.3.1) and the
// bounding box of each grid's core points.  One warp per grid.
__global__ void __launch_bounds__(256) core_compact_kernel(Params p, const int* __restrict__ Xs,
                                                           const unsigned char* __restrict__ core_s,
                                                           const int* __restrict__ cell_start,
                                                           const int* __restrict__ core_start, int C,
                                                           int* __restrict__ Xc, int* __restrict__ bbox) {
    const int lane = lane_id(), dp = p.dp, d = p.d;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const int cs = core_start[c], m = core_start[c + 1] - cs;
        if (m == 0) continue;
        const int b = cell_start[c], e = cell_start[c + 1];
        int lo[kMaxD], hi[kMaxD];
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            lo[j] = 0x7fffffff;
            hi[j] = (int)0x80000000;
        }
        int w = cs;
        for (int k0 = b; k0 < e; k0 += 32) {
            const int k = k0 + lane;
            const bool is = k < e && core_s[k];
            const unsigned bal = __ballot_sync(kFull, is);
            if (is) {
                const int dst = w + __popc(bal & lanemask_lt());
#pragma unroll
                for (int j = 0; j < kMaxD; ++j)
                    if (j < dp) {
                        const int v = Xs[(long long)k * dp + j];
                        Xc[(long long)dst * dp + j] = v;
                        if (j < d) {
                            lo[j] = min(lo[j], v);
                            hi[j] = max(hi[j], v);
                        }
                    }
            }
            w += __popc(bal);
        }
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            for (int o = 16; o > 0; o >>= 1) {
                lo[j] = min(lo[j], __shfl_xor_sync(kFull, lo[j], o));
                hi[j] = max(hi[j], __shfl_xor_sync(kFull, hi[j], o));
            }
        }
        if (lane < d) {
            int l = lo[0], h = hi[0];
#pragma unroll
            for (int j = 1; j < kMaxD; ++j)
                if (lane == j) {
                    l = lo[j];
                    h = hi[j];
                }
            bbox[(long long)c * 2 * d + lane] = l;
            bbox[(long long)c * 2 * d + d + lane] = h;
        }
    }
}

cudaError_t launch_core_compact(const Params& p, const int* Xs, const unsigned char* core_s, const int* cell_start,
                                const int* core_start, int C, int* Xc, int* bbox, cudaStream_t st) {
    long long blocks = ((long long)C * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    core_compact_kernel<<<(int)blocks, 256, 0, st>>>(p, Xs, core_s, cell_start, core_start, C, Xc, bbox);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// -------------------------------------------------------- candidate pairs
// Pairs (i, j) of core grids with j in Nei(i) and j > i.

template <bool FILL>
__global__ void pair_kernel(const int* __restrict__ nbr_start, const int* __restrict__ nbr,
                            const int* __restrict__ core_start, int C, int* __restrict__ cnt_or_start,
                            int2* __restrict__ pairs) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int k = 0;
    if (core_start[c + 1] > core_start[c]) {
        int2* out = FILL ? pairs + cnt_or_start[c] : nullptr;
        for (int t = nbr_start[c]; t < nbr_start[c + 1]; ++t) {
            const int j = nbr[t];
            if (j > c && core_start[j + 1] > core_start[j]) {
                if (FILL) out[k] = make_int2(c, j);
                k++;
            }
        }
    }
    if (!FILL) cnt_or_start[c] = k;
}

cudaError_t launch_pair_count(const int* nbr_start, const int* nbr, const int* core_start, int C, int* pair_count,
                              cudaStream_t st) {
    pair_kernel<false><<<(C + 255) / 256, 256, 0, st>>>(nbr_start, nbr, core_start, C, pair_count, nullptr);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_pair_fill(const int* nbr_start, const int* nbr, const int* core_start, int C,
                             const int* pair_start, int2* pairs, cudaStream_t st) {
    pair_kernel<true><<<(C + 255) / 256, 256, 0, st>>>(nbr_start, nbr, core_start, C, const_cast<int*>(pair_start),
                                                       pairs);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------ union-find
// Roots are always linked under the smaller index (atomicCAS on the root),
// and finds halve paths with plain stores: every stored parent is an
// ancestor, so concurrent halving never breaks a path.

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
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        // link root b under root a
        if (atomicCAS(parent + b, b, a) == b) return true;
    }
    return false;
}

// ------------------------------------------------------------- the test
// One warp per candidate pair:
//   1. skip if the grids are already in one set;
//   2. no if the bounding boxes of the two core sets are farther than eps;
//   3. yes if the boxes are within eps at their farthest corners;
//   4. otherwise the exact MinDist test over the core points, 32 x 32 tiles
//      (lane l holds a point of s_j, points of s_i are broadcast), stopping at
//      the first pair within eps.
template <int D, int DP>
__global__ void __launch_bounds__(256) merge_kernel(Params p, const int2* __restrict__ pairs,
                                                    const int* __restrict__ npairs_dev,
                                                    const int* __restrict__ Xc, const int* __restrict__ core_start,
                                                    const int* __restrict__ bbox, int* parent,
                                                    unsigned* status) {
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long eps2 = p.eps2;
    const int npairs = *npairs_dev;
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < npairs; w += warps) {
        const int2 pr = pairs[w];
        int same = 0;
        if (lane == 0) {
            const int ra = uf_find(parent, pr.x), rb = uf_find(parent, pr.y);
            if (ra < 0 || rb < 0) atomicOr(status, kDevTimeout);
            same = ra == rb;
        }
        if (__shfl_sync(kFull, same, 0)) continue;

        const int* bi = bbox + (long long)pr.x * 2 * D;
        const int* bj = bbox + (long long)pr.y * 2 * D;
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
        bool yes;
        if (mind > eps2) {
            yes = false;
        } else if (maxd <= eps2) {
            yes = true;
        } else {
            yes = false;
            const int ai = core_start[pr.x], mi = core_start[pr.x + 1] - ai;
            const int aj = core_start[pr.y], mj = core_start[pr.y + 1] - aj;
            for (int a0 = 0; a0 < mi && !yes; a0 += 32) {
                const int na = min(32, mi - a0);
                int P[D];
#pragma unroll
                for (int j = 0; j < D; ++j) P[j] = lane < na ? Xc[(long long)(ai + a0 + lane) * DP + j] : 0;
                for (int b0 = 0; b0 < mj; b0 += 32) {
                    const bool vq = b0 + lane < mj;
                    int Q[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) Q[j] = vq ? Xc[(long long)(aj + b0 + lane) * DP + j] : 0;
                    bool hit = false;
                    for (int t = 0; t < na; ++t) {
                        int pt[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) pt[j] = __shfl_sync(kFull, P[j], t);
                        hit |= vq && sqdist<D>(pt, Q) <= eps2;
                    }
                    if (__any_sync(kFull, hit)) {
                        yes = true;
                        break;
                    }
                }
            }
        }
        if (yes && lane == 0) {
            if (!uf_union(parent, pr.x, pr.y)) atomicOr(status, kDevTimeout);
        }
    }
}

template <int D>
static void merge_launch(const Params& p, const int2* pairs, const int* npairs, int max_pairs, const int* Xc,
                         const int* core_start, const int* bbox, int* parent, unsigned* status, cudaStream_t st) {
    constexpr int DP = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
    long long blocks = ((long long)max_pairs * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    merge_kernel<D, DP><<<(int)blocks, 256, 0, st>>>(p, pairs, npairs, Xc, core_start, bbox, parent, status);
    GD_COUNT_LAUNCH();
}

cudaError_t launch_merge(const Params& p, const int2* pairs, const int* npairs, int max_pairs, const int* Xc,
                         const int* core_start, const int* bbox, int* parent, unsigned* status, cudaStream_t st) {
    if (max_pairs <= 0) return cudaSuccess;
    switch (p.d) {
        case 1: merge_launch<1>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 2: merge_launch<2>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 3: merge_launch<3>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 4: merge_launch<4>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 5: merge_launch<5>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 6: merge_launch<6>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        case 7: merge_launch<7>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
        default: merge_launch<8>(p, pairs, npairs, max_pairs, Xc, core_start, bbox, parent, status, st); break;
    }
    return cudaGetLastError();
}

}  // namespace gd
