// Core points (Def. 1) by the G13 rule of Section 3.2: a grid holding at least
// MinPts points has only core points, since its diameter is <= eps.  In every
// other grid each point counts the points within eps over Nei(g) and stops as
// soon as it reaches MinPts (as in the paper, counting can stop early).
#include "gd_internal.cuh"

namespace gd {

__global__ void core_full_kernel(int n, int minpts, const int* __restrict__ cell_start,
                                 const int* __restrict__ pt_cell, unsigned char* __restrict__ core_s) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = pt_cell[i];
        core_s[i] = (cell_start[c + 1] - cell_start[c]) >= minpts ? 1 : 0;
    }
}

// Points of grids with fewer than MinPts points, as a flat list: nf_start is
// the exclusive scan of (grid size if the grid is not full, else 0).
__global__ void nonfull_count_kernel(int minpts, const int* __restrict__ cell_start, int C, int* __restrict__ nf) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int m = cell_start[c + 1] - cell_start[c];
    nf[c] = m < minpts ? m : 0;
}

// One warp per point p of a non-full grid g.  The lanes take the grids of
// Nei(g) 32 at a time and compare each grid's box (its identifier range,
// which holds every point of the grid) with p:
//   - box entirely within eps of p: all its points count, no distances;
//   - box entirely beyond eps: skipped;
//   - otherwise its points are tested one by one (the straddling grids'
//     points are streamed as one flat sequence, lane k taking the k-th).
// g itself is always entirely within eps (its diameter is <= eps).  Whole
// grids are counted first; straddling grids are then scanned -- for short
// neighbour lists in three bands of increasing box distance (up to eps/4,
// eps/2, eps), so that a core point usually reaches MinPts among the nearest
// points.  The warp stops as soon as the count reaches MinPts.
struct BoxDist {
    long long mind, maxd;
};

template <int D>
__device__ __forceinline__ BoxDist box_dist(const long long* x, const int* __restrict__ coord, int cc,
                                            const Params& p) {
    BoxDist r{0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const long long blo = (long long)p.mn[j] + (long long)coord[(long long)cc * D + j] * p.s;
        const long long bhi = blo + p.s - 1;
        long long g = 0;
        if (blo > x[j]) g = blo - x[j];
        else if (x[j] > bhi) g = x[j] - bhi;
        r.mind += g * g;
        const long long a = x[j] - blo, b = bhi - x[j];
        const long long f = a > b ? a : b;
        r.maxd += f * f;
    }
    return r;
}

template <int D, int DP>
__global__ void __launch_bounds__(256) core_point_kernel(Params p, const int* __restrict__ Xs,
                                                         const int* __restrict__ cell_start,
                                                         const int* __restrict__ coord, int C,
                                                         const int* __restrict__ nf_start,
                                                         const int* __restrict__ nbr_start,
                                                         const int* __restrict__ nbr,
                                                         unsigned char* __restrict__ core_s) {
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long eps2 = p.eps2;
    const int minpts = p.minpts;
    const int total = nf_start[C];
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        // grid of flat position w: last c with nf_start[c] <= w
        int lo = 0, hi = C - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (nf_start[mid] <= w)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int c = lo;
        const long long i = (long long)cell_start[c] + (w - nf_start[c]);
        long long x[D];
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = Xs[i * DP + j];
        int cnt = 0;
        const int t_begin = nbr_start[c], t_end = nbr_start[c + 1];
        // whole grids
        for (int t0 = t_begin; t0 < t_end && cnt < minpts; t0 += 32) {
            int whole = 0;
            if (t0 + lane < t_end) {
                const int cc = nbr[t0 + lane];
                const BoxDist bd = box_dist<D>(x, coord, cc, p);
                if (bd.maxd <= eps2) whole = cell_start[cc + 1] - cell_start[cc];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) whole += __shfl_xor_sync(kFull, whole, o);
            cnt += whole;
        }
        // straddling grids, nearest band first when the list is short (dense
        // neighbourhoods: few grids, many points each); one pass otherwise
        const int nbands = (t_end - t_begin) <= 128 ? 3 : 1;
        for (int band = 0; band < nbands && cnt < minpts; ++band) {
            const long long blo = band == 0 ? -1 : (band == 1 ? eps2 / 16 : eps2 / 4);
            const long long bhi = nbands == 1 ? eps2 : (band == 0 ? eps2 / 16 : (band == 1 ? eps2 / 4 : eps2));
            for (int t0 = t_begin; t0 < t_end && cnt < minpts; t0 += 32) {
                int st = 0, sz = 0;
                if (t0 + lane < t_end) {
                    const int cc = nbr[t0 + lane];
                    const BoxDist bd = box_dist<D>(x, coord, cc, p);
                    if (bd.maxd > eps2 && bd.mind > blo && bd.mind <= bhi) {
                        st = cell_start[cc];
                        sz = cell_start[cc + 1] - st;
                    }
                }
                const int incl = warp_inclusive_scan(sz);
                const int flat = __shfl_sync(kFull, incl, 31);
                for (int k0 = 0; k0 < flat; k0 += 32) {
                    const int k = k0 + lane;
                    int lo2 = 0, hi2 = 31;
#pragma unroll
                    for (int step = 0; step < 5; ++step) {
                        const int mid = (lo2 + hi2) >> 1;
                        if (__shfl_sync(kFull, incl, mid) > k)
                            hi2 = mid;
                        else
                            lo2 = mid + 1;
                    }
                    const int gst = __shfl_sync(kFull, st, lo2);
                    const int gex = __shfl_sync(kFull, incl, lo2) - __shfl_sync(kFull, sz, lo2);
                    bool hit = false;
                    if (k < flat) {
                        const long long qi = (long long)gst + (k - gex);
                        long long dd = 0;
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            const long long t = (long long)Xs[qi * DP + j] - x[j];
                            dd += t * t;
                        }
                        hit = dd <= eps2;
                    }
                    cnt += __popc(__ballot_sync(kFull, hit));
                    if (cnt >= minpts) break;
                }
            }
        }
        if (lane == 0) core_s[i] = cnt >= minpts ? 1 : 0;
    }
}

template <int D>
static void core_point_launch(const Params& p, const int* Xs, const int* cell_start, const int* coord, int C,
                              const int* nf_start, const int* nbr_start, const int* nbr, unsigned char* core_s,
                              cudaStream_t st) {
    constexpr int DP = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
    core_point_kernel<D, DP><<<152 * 16, 256, 0, st>>>(p, Xs, cell_start, coord, C, nf_start, nbr_start, nbr, core_s);
    GD_COUNT_LAUNCH();
}

cudaError_t launch_core(const Params& p, const int* Xs, const int* cell_start, const int* pt_cell,
                        const int* cell_coord, int C, const int* nbr_start, const int* nbr, int* nf_start, int* tmp,
                        unsigned char* core_s, cudaStream_t st) {
    int blocks = (p.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    core_full_kernel<<<blocks, 256, 0, st>>>(p.n, p.minpts, cell_start, pt_cell, core_s);
    GD_COUNT_LAUNCH();
    nonfull_count_kernel<<<(C + 255) / 256, 256, 0, st>>>(p.minpts, cell_start, C, nf_start);
    GD_COUNT_LAUNCH();
    cudaError_t e = scan_exclusive(nf_start, nf_start, C, tmp, st);
    if (e != cudaSuccess) return e;
    switch (p.d) {
#define GD_CORE(DD) \
    case DD: core_point_launch<DD>(p, Xs, cell_start, cell_coord, C, nf_start, nbr_start, nbr, core_s, st); break;
        GD_CORE(1) GD_CORE(2) GD_CORE(3) GD_CORE(4) GD_CORE(5) GD_CORE(6) GD_CORE(7)
        default: core_point_launch<8>(p, Xs, cell_start, cell_coord, C, nf_start, nbr_start, nbr, core_s, st); break;
#undef GD_CORE
    }
    return cudaGetLastError();
}

}  // namespace gd
