// Grid tree and non-empty neighbouring grids (Section 4.2), over a batch.
//
// The tree of Alg. 2 is held as d sorted levels.  Because the grids are in
// lexicographic order (Alg. 1), the nodes of level j are the distinct prefixes
// (g_1..g_{j+1}) of consecutive grids; each node stores its key g_{j+1} and the
// index of its first child on level j+1, so every child list is a contiguous,
// key-sorted range.  Level d-1 is the grid list itself.  The hash table h of
// Alg. 2 is not needed: a child range is searched by bisection.
//
// The query of Alg. 3 descends the levels, keeping at each level the children
// whose key lies within +-r of the query's identifier and whose partial offset
// (Eq. 2) stays within eps.  Offsets are exact integers, computed from the
// query grid's point box (the range its points actually span) rather than its
// whole identifier range: in dimension j a child with key k spans
// [mn_j + k*s, mn_j + k*s + s - 1], and its gap to the point box is the
// smallest coordinate difference any point pair can have there.  At a leaf
// the candidate's own point box replaces its key range, so a grid is a
// neighbour iff the two point boxes are within eps -- a subset of the paper's
// Nei(g) that still holds every grid with a point within eps of a point of g
// (in sparse, high-dimensional data, where grids hold about one point, it is
// an order of magnitude smaller).  Grids of more than kBoxPoints points use
// their identifier range as their box, and their own lists skip the leaf
// test: dense grids fill their range, so it would only cost loads.
#include "gd_internal.cuh"

namespace gd {

#define GD_FOR_FLAT(i, total)                                                                         \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (total);                 \
         i += (long long)gridDim.x * blockDim.x)

static int blocks_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    return b < 1 ? 1 : (int)b;
}

// Grids of more than kBoxPoints points keep their identifier range as their
// box (it holds all their points; refining dense grids gains nothing).
constexpr int kBoxPoints = 32;

// Box of every grid: one warp per grid; the lanes reduce the points of grids
// of at most kBoxPoints points, larger grids take their identifier range.
__global__ void __launch_bounds__(256) point_box_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    FlatCursor cur;
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        cur.seek(f, w);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = w - cur.lo;
        const int d = I.p.d, dp = I.p.dp;
        const int b = I.cell_start[c], e = I.cell_start[c + 1];
        if (e - b > kBoxPoints) {
            if (lane < d) {
                const long long blo = (long long)I.p.mn[lane] + (long long)I.cell_coord[c * d + lane] * I.p.s;
                I.pbox[c * 2 * d + lane] = (int)blo;
                I.pbox[c * 2 * d + d + lane] = (int)(blo + I.p.s - 1 < 0x7fffffffll ? blo + I.p.s - 1 : 0x7fffffffll);
            }
            continue;
        }
        int lo[kMaxD], hi[kMaxD];
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            lo[j] = 0x7fffffff;
            hi[j] = (int)0x80000000;
        }
        for (int q = b + lane; q < e; q += 32) {
#pragma unroll
            for (int j = 0; j < kMaxD; ++j)
                if (j < d) {
                    const int v = I.Xs[(long long)q * dp + j];
                    lo[j] = min(lo[j], v);
                    hi[j] = max(hi[j], v);
                }
        }
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            if (j >= d) break;
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
            I.pbox[c * 2 * d + lane] = l;
            I.pbox[c * 2 * d + d + lane] = h;
        }
    }
}

cudaError_t launch_point_boxes(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long b = (total * 32 + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    point_box_kernel<<<(int)b, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// L[c] = first dimension in which grid c differs from grid c-1 (0 for c = 0).
__global__ void level_diff_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int d = I.p.d;
        int l = 0;
        if (c > 0) {
            l = d;
            for (int j = 0; j < d; ++j)
                if (I.cell_coord[c * d + j] != I.cell_coord[(c - 1) * d + j]) {
                    l = j;
                    break;
                }
        }
        I.lv_L[c] = l;
    }
}

// A grid c starts a node on level j iff L[c] <= j.  Flat space: the grids of
// instances with d - 1 > j.
__global__ void level_flag_kernel(const Inst* __restrict__ ins, Flat f, long long total, int j) {
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int C = I.small[kSmCells];
        I.lv_E[(long long)j * (C + 1) + c] = I.lv_L[c] <= j ? 1 : 0;
    }
}

// After the scans, E_j[c] (exclusive) is the node index on level j of the node
// starting at grid c, and E_j[C] the node count of level j.
__global__ void level_write_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int d = I.p.d, C = I.small[kSmCells];
        const int* E = I.lv_E;
        const int l = I.lv_L[c];
        for (int j = l; j < d; ++j) {
            const long long u = (j < d - 1) ? E[(long long)j * (C + 1) + c] : c;
            I.lv_key[j][u] = I.cell_coord[c * d + j];
            if (j < d - 1) I.lv_cb[j][u] = (j + 1 < d - 1) ? E[(long long)(j + 1) * (C + 1) + c] : (int)c;
        }
        if (c == 0) {
            for (int j = 0; j < d; ++j) {
                const int nj = (j < d - 1) ? E[(long long)j * (C + 1) + C] : C;
                I.small[kSmLevelCount + j] = nj;
                if (j < d - 1) I.lv_cb[j][nj] = (j + 1 < d - 1) ? E[(long long)(j + 1) * (C + 1) + C] : C;
            }
        }
    }
}

cudaError_t launch_level_diff(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    level_diff_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_level_flag(const Inst* ins, Flat cells, long long total, int level, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    level_flag_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total, level);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_level_write(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    level_write_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// First index u in [lo, hi) with key[u] >= v (hi if none).
__device__ __forceinline__ int lower_key(const int* __restrict__ key, int lo, int hi, long long v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)__ldg(key + mid) < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Depth-first walk of the levels for one grid (Alg. 3).  FILL == false
// counts the neighbours into nbr_start[c]; FILL == true writes them at
// nbr + nbr_start[c] in lexicographic order (the query grid itself included).
template <bool FILL>
__global__ void __launch_bounds__(128) walk_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    FlatCursor cur;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int d = I.p.d;
        const long long r = I.p.r, s = I.p.s, eps2 = I.p.eps2;
        int g[kMaxD];
        long long olo[kMaxD], ohi[kMaxD], base[kMaxD];
        for (int j = 0; j < d; ++j) {
            g[j] = I.cell_coord[c * d + j];
            olo[j] = I.pbox[c * 2 * d + j];
            ohi[j] = I.pbox[c * 2 * d + d + j];
            base[j] = I.p.mn[j];
        }
        const int* pbox = I.pbox;
        // refine leaves by point boxes only around small grids
        const bool refine = I.cell_start[c + 1] - I.cell_start[c] <= kBoxPoints;
        const int* const* lkey = I.lv_key;
        const int* const* lcb = I.lv_cb;

        int cur[kMaxD], end[kMaxD];
        long long part[kMaxD];
        int* out = FILL ? I.nbr + I.nbr_start[c] : nullptr;
        int found = 0;

        int j = 0;
        part[0] = 0;
        end[0] = I.small[kSmLevelCount];
        cur[0] = lower_key(lkey[0], 0, end[0], (long long)g[0] - r);
        while (j >= 0) {
            if (cur[j] >= end[j]) {
                if (--j >= 0) cur[j]++;
                continue;
            }
            const int u = cur[j];
            const long long key = __ldg(lkey[j] + u);
            if (key > (long long)g[j] + r) {
                if (--j >= 0) cur[j]++;
                continue;
            }
            // gap between the query's point box and the child's key range
            const long long klo = base[j] + key * s, khi = klo + s - 1;
            long long gap = 0;
            if (klo > ohi[j]) gap = klo - ohi[j];
            else if (olo[j] > khi) gap = olo[j] - khi;
            const long long off = part[j] + gap * gap;
            if (off > eps2) {
                cur[j]++;
                continue;
            }
            if (j == d - 1) {
                // leaf: the two grids' boxes
                long long g2 = 0;
                if (refine) {
                    const int* ub = pbox + (long long)u * 2 * d;
                    for (int t = 0; t < d; ++t) {
                        long long gg = 0;
                        if (ub[t] > ohi[t]) gg = ub[t] - ohi[t];
                        else if (olo[t] > ub[d + t]) gg = olo[t] - ub[d + t];
                        g2 += gg * gg;
                    }
                }
                if (g2 <= eps2) {
                    if (FILL) out[found] = u;
                    found++;
                }
                cur[j]++;
                continue;
            }
            const int lo = __ldg(lcb[j] + u), hi = __ldg(lcb[j] + u + 1);
            j++;
            part[j] = off;
            end[j] = hi;
            cur[j] = lower_key(lkey[j], lo, hi, (long long)g[j] - r);
        }
        if (!FILL) I.nbr_start[c] = found;
    }
}

cudaError_t launch_walk(const Inst* ins, Flat cells, long long total, bool fill, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long b = (total + 127) / 128;
    if (b > kPersistBlocks * 2) b = kPersistBlocks * 2;
    if (fill)
        walk_kernel<true><<<(int)b, 128, 0, st>>>(ins, cells, total);
    else
        walk_kernel<false><<<(int)b, 128, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
