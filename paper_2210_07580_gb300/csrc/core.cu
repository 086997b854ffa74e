// Core points (Def. 1) by the G13 rule of Section 3.2, over a batch: a grid
// holding at least MinPts points has only core points, since its diameter is
// <= eps.  In every other grid each point counts the points within eps over
// Nei(g) and stops as soon as it reaches MinPts (as in the paper, counting can
// stop early).
#include "gd_internal.cuh"

namespace gd {

static int blocks_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    return b < 1 ? 1 : (int)b;
}

// Core flags of the points of full grids (1) and of the others (0, set by
// core_point_kernel later).  A grid's points are contiguous in sorted order:
// a lane takes a grid and fills the range of a small one itself, while the
// warp fills the ranges of its lanes' large grids together, one after the
// other, with 16-byte stores between the unaligned ends.
constexpr int kFillLane = 64;  // largest grid a lane fills alone

__global__ void __launch_bounds__(256) core_full_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    const int lane = lane_id();
    const long long stride = (long long)gridDim.x * blockDim.x;
    FlatCursor cur;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const long long w = base + lane;
        long long b = 0, e = 0;
        unsigned char v = 0;
        const Inst* I = nullptr;
        if (w < total) {
            cur.seek(f, w);
            I = ins + f.idx[cur.k];
            const long long c = w - cur.lo;
            b = I->cell_start[c];
            e = I->cell_start[c + 1];
            v = e - b >= I->p.minpts ? 1 : 0;
            if (e - b <= kFillLane)
                for (long long q = b; q < e; ++q) I->core_s[q] = v;
        }
        unsigned big = __ballot_sync(kFull, e - b > kFillLane);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const long long bb = __shfl_sync(kFull, b, src), ee = __shfl_sync(kFull, e, src);
            const unsigned char vv = (unsigned char)__shfl_sync(kFull, (int)v, src);
            unsigned char* p = reinterpret_cast<unsigned char*>(__shfl_sync(kFull, (unsigned long long)(size_t)(I ? I->core_s : nullptr), src));
            const unsigned long long A = (unsigned long long)(size_t)p;
            const long long a0 = min(ee, bb + (long long)((16 - (A + bb) % 16) % 16));
            const long long a1 = max(a0, ee - (long long)((A + ee) % 16));
            for (long long q = bb + lane; q < a0; q += 32) p[q] = vv;
            const unsigned wv = vv ? 0x01010101u : 0u;
            const uint4 word = make_uint4(wv, wv, wv, wv);
            for (long long q = a0 + 16ll * lane; q < a1; q += 16 * 32) *reinterpret_cast<uint4*>(p + q) = word;
            for (long long q = a1 + lane; q < ee; q += 32) p[q] = vv;
        }
    }
}

// nf_start[c] = size of grid c if it is not full, else 0 (scanned next).
__global__ void nonfull_count_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int m = I.cell_start[c + 1] - I.cell_start[c];
        I.nf_start[c] = m < I.p.minpts ? m : 0;
    }
}

// Statistics (not timed): for each non-full grid, its points and the rows of
// its neighbour grids -- the points a count that stages every neighbour grid
// once per non-full grid reads.
__global__ void core_stats_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = i - cur.lo;
        const int m = I.cell_start[c + 1] - I.cell_start[c];
        if (m >= I.p.minpts) continue;
        unsigned long long rows = 0;
        for (int t = I.nbr_start[c]; t < I.nbr_start[c + 1]; ++t) {
            const int cc = I.nbr[t];
            rows += (unsigned long long)(I.cell_start[cc + 1] - I.cell_start[cc]);
        }
        stat_add(I.stats, kStNonfull, (unsigned long long)m);
        stat_add(I.stats, kStCountRows, rows);
    }
}

cudaError_t launch_core_stats(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    core_stats_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_core_full(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    core_full_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// After the scan of nf_start: the points counted one by one, listed by their
// index in grid order (a thread per grid), so that a warp of
// core_point_kernel finds its point and grid with two loads.
__global__ void nf_index_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = i - cur.lo;
        const int C = I.small[kSmCells];
        const int lo = I.nf_start[c], hi = c + 1 < C ? I.nf_start[c + 1] : I.small[kSmNonfull];
        const int b = I.cell_start[c];
        for (int k = 0; k < hi - lo; ++k) I.nf_pts[lo + k] = b + k;
    }
}

cudaError_t launch_nf_index(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    nf_index_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_nonfull_count(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    nonfull_count_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

struct BoxDist {
    long long mind, maxd;
};

// Squared distances from x to the nearest and farthest corner of grid cc's
// point box (which holds every point of the grid).
// Coordinates span less than 2^31 per dimension and a box's lower end lies
// within the data, so the gap and x - lo fit in 32 bits; a large grid's box
// is its identifier range, whose upper end may lie beyond the data, so
// hi - x takes 64.
template <int D>
__device__ __forceinline__ BoxDist box_dist(const int* x, const int* __restrict__ pbox, int cc) {
    BoxDist r{0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int blo = __ldg(pbox + (long long)cc * 2 * D + j);
        const int bhi = __ldg(pbox + (long long)cc * 2 * D + D + j);
        int g = 0;
        if (blo > x[j]) g = blo - x[j];
        else if (x[j] > bhi) g = x[j] - bhi;
        r.mind += (long long)g * g;
        const long long a = x[j] - blo, b = (long long)bhi - x[j];
        const long long f = a > b ? a : b;
        r.maxd += f * f;
    }
    return r;
}

// Points of the straddling grids of one 32-entry chunk of a neighbour list,
// streamed as one flat sequence (lane k taking the k-th point): lane t holds
// the chunk's t-th grid as (first row st, rows sz; sz = 0 for a grid that is
// not straddling).  Adds the hits to cnt and stops once it reaches MinPts.
template <int D, int DP>
__device__ __forceinline__ void count_straddling(const int* __restrict__ Xs, const int* x, int st, int sz,
                                                 long long eps2, int minpts, int& cnt, unsigned& ndist) {
    const int lane = lane_id();
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
                const int t = Xs[qi * DP + j] - x[j];  // both points in the data: fits 32 bits
                dd += (long long)t * t;
            }
            hit = dd <= eps2;
        }
        cnt += __popc(__ballot_sync(kFull, hit));
        ndist += (unsigned)min(32, flat - k0);
        if (cnt >= minpts) break;
    }
}

// One warp per point p of a non-full grid g.  The lanes take the grids of
// Nei(g) 32 at a time and compare each grid's point box with p:
//   - box entirely within eps of p: all its points count, no distances;
//   - box entirely beyond eps: skipped;
//   - otherwise (straddling) its points are tested one by one
//     (count_straddling).
// g itself is always entirely within eps (its diameter is <= eps).  Whole
// grids are counted first, over the whole list, which also gives the points
// of the straddling grids; the straddling grids are then scanned -- for
// short neighbour lists in three bands of increasing box distance (up to
// eps/4, eps/2, eps), so that a core point usually reaches MinPts among the
// nearest points.  The warp stops as soon as the count reaches MinPts, or
// as soon as the straddling points not yet tested could no longer bring it
// there (p is then not core; in sparse data most non-core points stop
// before testing any distance).
template <int D>
__global__ void __launch_bounds__(256) core_point_kernel(const Inst* __restrict__ ins, Flat f, int band_limit) {
    constexpr int DP = Padded<D>::value;
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = flat_total(f);
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        const int kk = flat_find(f, w);
        const Inst& I = ins[f.idx[kk]];
        const long long lw = w - f.off[kk];
        const Params& p = I.p;
        const long long eps2 = p.eps2;
        const int minpts = p.minpts;
        const int* cell_start = I.cell_start;
        const int* pbox = I.pbox;
        const int* Xs = I.Xs;
        const long long i = I.nf_pts[lw];
        const int c = I.pt_cell[i];
        int x[D];
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = Xs[i * DP + j];
        int cnt = 0;
        long long rest = 0;  // points of the straddling grids not yet tested
        unsigned ndist = 0;  // statistics: distances this warp evaluated
        const int t_begin = I.nbr_start[c], t_end = I.nbr_start[c + 1];
        const int* nbr = I.nbr;
        // whole grids, and the size of the straddling ones (each chunk's grid
        // ids loaded one chunk ahead)
        int cc_next = t_begin + lane < t_end ? __ldg(nbr + t_begin + lane) : -1;
        for (int t0 = t_begin; t0 < t_end && cnt < minpts; t0 += 32) {
            int whole = 0, part = 0;
            const int cc = cc_next;
            cc_next = t0 + 32 + lane < t_end ? __ldg(nbr + t0 + 32 + lane) : -1;
            if (cc >= 0) {
                const int a = __ldg(cell_start + cc), b = __ldg(cell_start + cc + 1);
                const BoxDist bd = box_dist<D>(x, pbox, cc);
                if (bd.maxd <= eps2) whole = b - a;
                else if (bd.mind <= eps2) part = b - a;
            }
            cnt += __reduce_add_sync(kFull, whole);
            rest += __reduce_add_sync(kFull, part);
        }
        // straddling grids, nearest band first when the list is short
        // (dense neighbourhoods: few grids, many points each); one pass
        // otherwise
        const int nbands = (t_end - t_begin) <= band_limit ? 3 : 1;
        for (int band = 0; band < nbands && cnt < minpts && cnt + rest >= minpts; ++band) {
            const long long blo = band == 0 ? -1 : (band == 1 ? eps2 / 16 : eps2 / 4);
            const long long bhi = nbands == 1 ? eps2 : (band == 0 ? eps2 / 16 : (band == 1 ? eps2 / 4 : eps2));
            for (int t0 = t_begin; t0 < t_end && cnt < minpts && cnt + rest >= minpts; t0 += 32) {
                int st = 0, sz = 0;
                if (t0 + lane < t_end) {
                    const int cc = nbr[t0 + lane];
                    const BoxDist bd = box_dist<D>(x, pbox, cc);
                    if (bd.maxd > eps2 && bd.mind > blo && bd.mind <= bhi) {
                        st = cell_start[cc];
                        sz = cell_start[cc + 1] - st;
                    }
                }
                count_straddling<D, DP>(Xs, x, st, sz, eps2, minpts, cnt, ndist);
                rest -= __reduce_add_sync(kFull, sz);
            }
        }
        if (lane == 0) {
            I.core_s[i] = cnt >= minpts ? 1 : 0;
            stat_add(I.stats, kStDistCore, ndist);
        }
    }
}

// One warp per grid g that is not full (per-grid form of core_point_kernel).
// The grid's points -- 32 at a time -- are staged in shared memory; the warp
// reads g's neighbour list and the neighbours' point boxes once per 32 list
// entries (lane t loading entry t into shared memory) and applies them to
// every point of g in turn, so a grid of m points reads its list once
// instead of m times.  For each point p:
//   pass 1, over the whole list: grids entirely within eps of p count whole;
//   pass 2, while p is short of MinPts: the straddling grids' points are
//     streamed as one flat sequence (lane k taking the k-th) -- for short
//     lists nearest band first, as in core_point_kernel.
// A point stops as soon as its count reaches MinPts.  (Bounding the count by
// the straddling points left, as core_point_kernel does, costs a second
// reduction per point and entry here and did not pay on 3-d data.)
constexpr int kCoreWarps = 8;

template <int D>
__global__ void __launch_bounds__(32 * kCoreWarps)
    core_grid_kernel(const Inst* __restrict__ ins, Flat f, long long total, int band_limit) {
    total = flat_total(f);
    constexpr int DP = Padded<D>::value;
    __shared__ int sx[kCoreWarps][32][D];      // the grid's points (32 at a time)
    __shared__ int sbox[kCoreWarps][2 * D][32];  // the entries' boxes: lo then hi, lane-major
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    FlatCursor cur;
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + wib; w < total; w += warps) {
        cur.seek(f, w);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = w - cur.lo;
        const int* cell_start = I.cell_start;
        const int b = cell_start[c], m = cell_start[c + 1] - b;
        const int minpts = I.p.minpts;
        if (m >= minpts) continue;  // full: core_full_kernel set its flags
        const long long eps2 = I.p.eps2;
        const int* Xs = I.Xs;
        const int* pbox = I.pbox;
        const int* nbr = I.nbr;
        const int t_begin = I.nbr_start[c], t_end = I.nbr_start[c + 1];
        const int nbands = (t_end - t_begin) <= band_limit ? 3 : 1;
        unsigned ndist = 0;  // statistics: distances this warp evaluated
        // the entries t0 .. t0+31 into shared memory; returns the lane's
        // entry's first point and size (0 past the list)
        auto load_entries = [&](int t0, int* st_out) {
            int sz = 0, st = 0;
            if (t0 + lane < t_end) {
                const int cc = nbr[t0 + lane];
#pragma unroll
                for (int j = 0; j < 2 * D; ++j) sbox[wib][j][lane] = pbox[(long long)cc * 2 * D + j];
                st = cell_start[cc];
                sz = cell_start[cc + 1] - st;
            }
            *st_out = st;
            __syncwarp();
            return sz;
        };
        for (int own0 = 0; own0 < m; own0 += 32) {
            const int mo = min(32, m - own0);
            if (lane < mo) {
#pragma unroll
                for (int j = 0; j < D; ++j) sx[wib][lane][j] = Xs[(long long)(b + own0 + lane) * DP + j];
            }
            __syncwarp();
            int cnt = 0;  // lane p < mo: the count of own point p
            const unsigned own = mo == 32 ? kFull : ((1u << mo) - 1u);
            // pass 1: whole grids
            for (int t0 = t_begin; t0 < t_end; t0 += 32) {
                int st0;
                const int sz0 = load_entries(t0, &st0);
                for (int p = 0; p < mo; ++p) {
                    int whole = 0;
                    if (sz0 > 0) {
                        long long maxd = 0;
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            // x - lo fits 32 bits; hi - x takes 64 (box_dist)
                            const int x = sx[wib][p][j];
                            const long long a = x - sbox[wib][j][lane], bb = (long long)sbox[wib][D + j][lane] - x;
                            const long long fm = a > bb ? a : bb;
                            maxd += fm * fm;
                        }
                        if (maxd <= eps2) whole = sz0;
                    }
                    whole = __reduce_add_sync(kFull, whole);
                    if (lane == p) cnt += whole;
                }
                __syncwarp();
                if (__ballot_sync(kFull, cnt >= minpts) == own) break;
            }
            // pass 2: straddling grids, per point still short of MinPts
            for (int band = 0; band < nbands; ++band) {
                unsigned pend = own & ~__ballot_sync(kFull, cnt >= minpts);
                if (!pend) break;
                const long long blo = band == 0 ? -1 : (band == 1 ? eps2 / 16 : eps2 / 4);
                const long long bhi = nbands == 1 ? eps2 : (band == 0 ? eps2 / 16 : (band == 1 ? eps2 / 4 : eps2));
                for (int t0 = t_begin; t0 < t_end && pend; t0 += 32) {
                    int st0;
                    const int sz0 = load_entries(t0, &st0);
                    for (unsigned pp = pend; pp; pp &= pp - 1) {
                        const int p = __ffs(pp) - 1;
                        int x[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) x[j] = sx[wib][p][j];
                        int cp = __shfl_sync(kFull, cnt, p);
                        int sz = 0;
                        if (sz0 > 0) {
                            long long mind = 0, maxd = 0;
#pragma unroll
                            for (int j = 0; j < D; ++j) {
                                const int l = sbox[wib][j][lane], h = sbox[wib][D + j][lane];
                                int g = 0;
                                if (l > x[j]) g = l - x[j];
                                else if (x[j] > h) g = x[j] - h;
                                mind += (long long)g * g;
                                const long long a = x[j] - l, bb = (long long)h - x[j];
                                const long long fm = a > bb ? a : bb;
                                maxd += fm * fm;
                            }
                            if (maxd > eps2 && mind > blo && mind <= bhi) sz = sz0;
                        }
                        const int incl = warp_inclusive_scan(sz);
                        const int flat = __shfl_sync(kFull, incl, 31);
                        for (int k0 = 0; k0 < flat && cp < minpts; k0 += 32) {
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
                            const int gst = __shfl_sync(kFull, st0, lo2);
                            const int gex = __shfl_sync(kFull, incl, lo2) - __shfl_sync(kFull, sz, lo2);
                            bool hit = false;
                            if (k < flat) {
                                const long long qi = (long long)gst + (k - gex);
                                long long dd = 0;
#pragma unroll
                                for (int j = 0; j < D; ++j) {
                                    const int t = Xs[qi * DP + j] - x[j];
                                    dd += (long long)t * t;
                                }
                                hit = dd <= eps2;
                            }
                            cp += __popc(__ballot_sync(kFull, hit));
                            ndist += (unsigned)min(32, flat - k0);
                        }
                        if (lane == p) cnt = cp;
                        if (cp >= minpts) pend &= ~(1u << p);
                    }
                    __syncwarp();
                }
            }
            if (lane < mo) I.core_s[b + own0 + lane] = cnt >= minpts ? 1 : 0;
            __syncwarp();
        }
        if (lane == 0) stat_add(I.stats, kStDistCore, ndist);
    }
}

cudaError_t launch_core_grid(const Inst* ins, Flat cells, long long total, int d, int band_limit, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long nb = (total + kCoreWarps - 1) / kCoreWarps;
    if (nb > kPersistBlocks) nb = kPersistBlocks;
    switch (d) {
#define GD_CG(DD) \
    case DD: core_grid_kernel<DD><<<(int)nb, 32 * kCoreWarps, 0, st>>>(ins, cells, total, band_limit); break;
        GD_CG(1) GD_CG(2) GD_CG(3) GD_CG(4) GD_CG(5) GD_CG(6) GD_CG(7) GD_CG(8)
#undef GD_CG
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_core_point(const Inst* ins, Flat nf_pts, int d, int band_limit, cudaStream_t st) {
    switch (d) {
#define GD_CORE(DD) \
    case DD: core_point_kernel<DD><<<kPersistBlocks, 256, 0, st>>>(ins, nf_pts, band_limit); break;
        GD_CORE(1) GD_CORE(2) GD_CORE(3) GD_CORE(4) GD_CORE(5) GD_CORE(6) GD_CORE(7) GD_CORE(8)
#undef GD_CORE
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
