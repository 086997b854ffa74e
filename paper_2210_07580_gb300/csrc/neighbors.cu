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

// Walk of the levels for one grid (Alg. 3), one warp per query grid.
//
// The warp keeps a stack of key ranges in shared memory: (level j, nodes
// [lo, hi) of level j, partial offset of the path above them).  Each step
// takes the entries of the top level -- up to 32 nodes across several
// ranges, the last range possibly split -- and the lanes test one node each:
// key within +-r, offset within eps (and, at a leaf, the point-box test);
// surviving inner nodes push their child range (narrowed to keys within +-r
// by bisection when it is long), surviving leaves are counted (FILL == false,
// into nbr_start[c]) or written at nbr + nbr_start[c] (FILL == true; both
// passes visit the nodes in the same order).
//
// Stack bound: levels never decrease from the bottom of the stack to its top
// (a step pops the top level j and pushes level j + 1), so a level receives
// pushes only when nothing deeper is left, and one step pushes at most 32
// entries.  Hence at most 32 entries per level below the root: 1 + 32 (d - 1).
constexpr int kWalkWarps = 4;
constexpr int kWalkStack = 1 + 32 * (kMaxD - 1);
// child ranges longer than this are narrowed by bisection before the push
constexpr int kNarrowAbove = 16;

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

struct WalkShared {
    int lo[kWalkWarps][kWalkStack];
    int hi[kWalkWarps][kWalkStack];
    long long part[kWalkWarps][kWalkStack];
    signed char lvl[kWalkWarps][kWalkStack];
    long long qlo[kWalkWarps][kMaxD], qhi[kWalkWarps][kMaxD];    // query point box
    long long klo[kWalkWarps][kMaxD], khi[kWalkWarps][kMaxD];    // key window g_j -+ r
    long long base[kWalkWarps][kMaxD];                           // mn_j
};

template <bool FILL>
__global__ void __launch_bounds__(32 * kWalkWarps) walk_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    __shared__ WalkShared sh;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    int* const slo = sh.lo[w];
    int* const shi = sh.hi[w];
    long long* const spart = sh.part[w];
    signed char* const slvl = sh.lvl[w];
    const long long warps = (long long)gridDim.x * kWalkWarps;
    const unsigned lt = lanemask_lt();
    FlatCursor cur;
    for (long long q = (long long)blockIdx.x * kWalkWarps + w; q < total; q += warps) {
        cur.seek(f, q);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = q - cur.lo;
        const int d = I.p.d;
        const long long r = I.p.r, s = I.p.s, eps2 = I.p.eps2;
        if (lane < d) {
            const long long g = I.cell_coord[c * d + lane];
            sh.qlo[w][lane] = I.pbox[c * 2 * d + lane];
            sh.qhi[w][lane] = I.pbox[c * 2 * d + d + lane];
            sh.klo[w][lane] = g - r;
            sh.khi[w][lane] = g + r;
            sh.base[w][lane] = I.p.mn[lane];
        }
        __syncwarp();
        const bool refine = I.cell_start[c + 1] - I.cell_start[c] <= kBoxPoints;
        const int* pbox = I.pbox;
        int* out = FILL ? I.nbr + I.nbr_start[c] : nullptr;
        int found = 0;
        int top = 0;
        {
            const int n0 = I.small[kSmLevelCount];
            const int a0 = lower_key(I.lv_key[0], 0, n0, sh.klo[w][0]);
            const int b0 = lower_key(I.lv_key[0], a0, n0, sh.khi[w][0] + 1);
            if (b0 > a0) {
                if (lane == 0) {
                    slo[0] = a0;
                    shi[0] = b0;
                    spart[0] = 0;
                    slvl[0] = 0;
                }
                top = 1;
            }
        }
        __syncwarp();
        while (top > 0) {
            // the group: the entries of the top level, lane i holding entry top-1-i
            const int J = slvl[top - 1];
            const int e = top - 1 - lane;
            const bool in_group = e >= 0 && slvl[e] == J;
            int elo = 0, sz = 0;
            long long epart = 0;
            if (in_group) {
                elo = slo[e];
                sz = min(shi[e] - elo, 64);
                epart = spart[e];
            }
            const int P = warp_inclusive_scan(sz);
            const int start = P - sz;
            const int taken = min(32, __shfl_sync(kFull, P, 31));
            const unsigned starts = __reduce_or_sync(kFull, (in_group && start < 32) ? (1u << start) : 0u);
            const int consumed = __popc(__ballot_sync(kFull, in_group && P <= 32));
            // the entry split at 32 nodes keeps its remainder on the stack
            if (in_group && P > 32 && start < 32) slo[e] = elo + (32 - start);
            // each lane's node: entry index = number of segment starts at or
            // below the lane, minus one
            const int ei = __popc(starts & ((2u << lane) - 1u)) - 1;
            const int my_lo = __shfl_sync(kFull, elo, ei < 0 ? 0 : ei);
            const int my_start = __shfl_sync(kFull, start, ei < 0 ? 0 : ei);
            const long long my_part = __shfl_sync(kFull, epart, ei < 0 ? 0 : ei);
            top -= consumed;
            __syncwarp();

            const bool act = lane < taken;
            const int u = my_lo + (lane - my_start);
            bool ok = false;
            long long off = 0;
            if (act) {
                const long long key = __ldg(I.lv_key[J] + u);
                if (key >= sh.klo[w][J] && key <= sh.khi[w][J]) {
                    const long long clo = sh.base[w][J] + key * s, chi = clo + s - 1;
                    const long long ql = sh.qlo[w][J], qh = sh.qhi[w][J];
                    long long gap = 0;
                    if (clo > qh) gap = clo - qh;
                    else if (ql > chi) gap = ql - chi;
                    off = my_part + gap * gap;
                    ok = off <= eps2;
                }
            }
            if (J == d - 1) {
                // leaf: the two grids' point boxes
                if (ok && refine) {
                    const int* ub = pbox + (long long)u * 2 * d;
                    long long g2 = 0;
                    for (int t = 0; t < d; ++t) {
                        const long long bl = __ldg(ub + t), bh = __ldg(ub + d + t);
                        const long long ql = sh.qlo[w][t], qh = sh.qhi[w][t];
                        long long gg = 0;
                        if (bl > qh) gg = bl - qh;
                        else if (ql > bh) gg = ql - bh;
                        g2 += gg * gg;
                    }
                    ok = g2 <= eps2;
                }
                const unsigned m = __ballot_sync(kFull, ok);
                if (FILL && ok) out[found + __popc(m & lt)] = u;
                found += __popc(m);
            } else {
                int clo = 0, chi = 0;
                if (ok) {
                    clo = __ldg(I.lv_cb[J] + u);
                    chi = __ldg(I.lv_cb[J] + u + 1);
                    if (chi - clo > kNarrowAbove) {
                        const int* nk = I.lv_key[J + 1];
                        clo = lower_key(nk, clo, chi, sh.klo[w][J + 1]);
                        chi = lower_key(nk, clo, chi, sh.khi[w][J + 1] + 1);
                    }
                    ok = chi > clo;
                }
                const unsigned m = __ballot_sync(kFull, ok);
                if (ok) {
                    const int at = top + __popc(m & lt);
                    slo[at] = clo;
                    shi[at] = chi;
                    spart[at] = off;
                    slvl[at] = (signed char)(J + 1);
                }
                top += __popc(m);
            }
            __syncwarp();
        }
        if (!FILL && lane == 0) I.nbr_start[c] = found;
        __syncwarp();
    }
}

cudaError_t launch_walk(const Inst* ins, Flat cells, long long total, bool fill, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long b = (total + kWalkWarps - 1) / kWalkWarps;
    if (b > kPersistBlocks * 2) b = kPersistBlocks * 2;
    if (fill)
        walk_kernel<true><<<(int)b, 32 * kWalkWarps, 0, st>>>(ins, cells, total);
    else
        walk_kernel<false><<<(int)b, 32 * kWalkWarps, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
