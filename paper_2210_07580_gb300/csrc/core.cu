// Core points (Def. 1) by the G13 rule of Section 3.2: a grid holding at least
// MinPts points has only core points, since its diameter is <= eps.  In every
// other grid each point counts the points within eps over Nei(g) and stops as
// soon as it reaches MinPts.
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

// One warp per grid with fewer than MinPts points.  Lane t holds own point t
// (groups of 32).  Neighbour grids whose box lies farther than eps from the
// box of the group's points cannot contribute and are dropped.  The remaining
// grids' points are streamed as one flat sequence, 32 at a time (lane k takes
// the k-th), so that small grids still fill the warp; each own point is
// broadcast in turn and its count grows by the popcount of the ballot of
// hits.  The warp stops once every own point has reached MinPts.
template <int D, int DP>
__global__ void __launch_bounds__(256) core_sparse_kernel(Params p, const int* __restrict__ Xs,
                                                          const int* __restrict__ cell_start,
                                                          const int* __restrict__ coord, int C,
                                                          const int* __restrict__ nbr_start,
                                                          const int* __restrict__ nbr,
                                                          unsigned char* __restrict__ core_s) {
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long eps2 = p.eps2;
    const int minpts = p.minpts;
    for (long long c = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const int b = cell_start[c], e = cell_start[c + 1];
        if (e - b >= minpts) continue;
        const int t_begin = nbr_start[c], t_end = nbr_start[c + 1];
        for (int g0 = b; g0 < e; g0 += 32) {
            const int mg = min(32, e - g0);
            int own[D];
#pragma unroll
            for (int j = 0; j < D; ++j) own[j] = lane < mg ? Xs[(long long)(g0 + lane) * DP + j] : 0;
            long long olo[D], ohi[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                int lo = lane < mg ? own[j] : 0x7fffffff, hi = lane < mg ? own[j] : (int)0x80000000;
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(kFull, lo, o));
                    hi = max(hi, __shfl_xor_sync(kFull, hi, o));
                }
                olo[j] = lo;
                ohi[j] = hi;
            }
            int cnt = 0;
            bool all_done = false;
            for (int t0 = t_begin; t0 < t_end && !all_done; t0 += 32) {
                const int nb = min(32, t_end - t0);
                int st = 0, sz = 0;
                if (lane < nb) {
                    const int cc = nbr[t0 + lane];
                    long long g2 = 0;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const long long clo = (long long)p.mn[j] + (long long)coord[(long long)cc * D + j] * p.s;
                        const long long chi = clo + p.s - 1;
                        long long g = 0;
                        if (clo > ohi[j]) g = clo - ohi[j];
                        else if (olo[j] > chi) g = olo[j] - chi;
                        g2 += g * g;
                    }
                    if (g2 <= eps2) {
                        st = cell_start[cc];
                        sz = cell_start[cc + 1] - st;
                    }
                }
                const int incl = warp_inclusive_scan(sz);
                const int total = __shfl_sync(kFull, incl, 31);
                for (int k0 = 0; k0 < total; k0 += 32) {
                    const int k = k0 + lane;
                    // which of the 32 grids holds flat position k: first lane with incl > k
                    int lo = 0, hi = 31;
#pragma unroll
                    for (int step = 0; step < 5; ++step) {
                        const int mid = (lo + hi) >> 1;
                        const int v = __shfl_sync(kFull, incl, mid);
                        if (v > k)
                            hi = mid;
                        else
                            lo = mid + 1;
                    }
                    const int gi = lo;
                    const int gst = __shfl_sync(kFull, st, gi);
                    const int gex = __shfl_sync(kFull, incl, gi) - __shfl_sync(kFull, sz, gi);
                    const bool valid = k < total;
                    int q[D];
                    const long long qi = (long long)gst + (k - gex);
#pragma unroll
                    for (int j = 0; j < D; ++j) q[j] = valid ? Xs[qi * DP + j] : 0;
                    for (int t = 0; t < mg; ++t) {
                        int pt[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) pt[j] = __shfl_sync(kFull, own[j], t);
                        const bool hit = valid && sqdist<D>(pt, q) <= eps2;
                        const int add = __popc(__ballot_sync(kFull, hit));
                        if (lane == t) cnt += add;
                    }
                    if (__all_sync(kFull, lane >= mg || cnt >= minpts)) {
                        all_done = true;
                        break;
                    }
                }
            }
            if (lane < mg) core_s[g0 + lane] = cnt >= minpts ? 1 : 0;
        }
    }
}

template <int D>
static void core_sparse_launch(const Params& p, const int* Xs, const int* cell_start, const int* coord, int C,
                               const int* nbr_start, const int* nbr, unsigned char* core_s, cudaStream_t st) {
    constexpr int DP = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
    long long blocks = ((long long)C * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    core_sparse_kernel<D, DP><<<(int)blocks, 256, 0, st>>>(p, Xs, cell_start, coord, C, nbr_start, nbr, core_s);
    GD_COUNT_LAUNCH();
}

cudaError_t launch_core(const Params& p, const int* Xs, const int* cell_start, const int* pt_cell,
                        const int* cell_coord, int C, const int* nbr_start, const int* nbr, unsigned char* core_s,
                        cudaStream_t st) {
    int blocks = (p.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    core_full_kernel<<<blocks, 256, 0, st>>>(p.n, p.minpts, cell_start, pt_cell, core_s);
    GD_COUNT_LAUNCH();
    switch (p.d) {
        case 1: core_sparse_launch<1>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 2: core_sparse_launch<2>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 3: core_sparse_launch<3>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 4: core_sparse_launch<4>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 5: core_sparse_launch<5>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 6: core_sparse_launch<6>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        case 7: core_sparse_launch<7>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
        default: core_sparse_launch<8>(p, Xs, cell_start, cell_coord, C, nbr_start, nbr, core_s, st); break;
    }
    return cudaGetLastError();
}

}  // namespace gd
