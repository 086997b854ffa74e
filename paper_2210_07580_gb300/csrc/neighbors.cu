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
// their identifier range as their box (such dense grids fill their range).
//
// The relation "boxes within eps" is symmetric, so each pair is found once:
// the walk from grid c enumerates only the grids g' >= c (lexicographic
// order, the order of the grid list): while the path it descends equals c's
// own identifier prefix, a level's key window is [g_j, g_j + r] instead of
// [g_j - r, g_j + r].  Each pair (c, g'), g' > c, then also enters g''s list
// (its backward part), placed by an atomic cursor per grid.  The walk does
// about half the work of a full one, and the lists are the same sets.
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
// box (it holds all their points).  Below that the exact box pays: the core
// boxes of full grids are these boxes, and the border search and the merge
// prune by them (a grid at a cluster's edge fills only part of its range).
constexpr int kBoxPoints = 1024;

// Box of every grid: one warp per grid; the lanes reduce the points of grids
// of at most kBoxPoints points (d <= 4: eight 16-byte rows per lane in
// flight), larger grids take their identifier range.
__global__ void __launch_bounds__(256) point_box_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
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
        int q = b + lane;
        if (dp == 4)  // eight rows per lane in flight (the dense, low-dimensional grids)
            for (; q + 224 < e; q += 256) {
                int4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = *reinterpret_cast<const int4*>(I.Xs + (long long)(q + 32 * u) * 4);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    lo[0] = min(lo[0], v[u].x);
                    hi[0] = max(hi[0], v[u].x);
                    lo[1] = min(lo[1], v[u].y);
                    hi[1] = max(hi[1], v[u].y);
                    lo[2] = min(lo[2], v[u].z);
                    hi[2] = max(hi[2], v[u].z);
                    lo[3] = min(lo[3], v[u].w);
                    hi[3] = max(hi[3], v[u].w);
                }
            }
        for (; q < e; q += 32) {
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
    total = flat_total(f);
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
        I.nbr_bwd[c] = 0;  // backward-entry counts of the walk that follows
    }
}

// A grid c starts a node on level j iff L[c] <= j.  Flat space: the grids of
// instances with d - 1 > j.
__global__ void level_flag_kernel(const Inst* __restrict__ ins, Flat f, long long total, int j) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        I.lv_E[(long long)j * (I.p.n + 1) + c] = I.lv_L[c] <= j ? 1 : 0;
    }
}

// After the scans, E_j[c] (exclusive) is the node index on level j of the node
// starting at grid c, and E_j[C] the node count of level j.  Row j of lv_E
// starts at j * (n + 1): n bounds the grid count C.
__global__ void level_write_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int d = I.p.d, C = I.small[kSmCells];
        const long long R = (long long)I.p.n + 1;  // row stride of lv_E
        const int* E = I.lv_E;
        const int l = I.lv_L[c];
        for (int j = l; j < d; ++j) {
            const long long u = (j < d - 1) ? E[j * R + c] : c;
            I.lv_key[j][u] = I.cell_coord[c * d + j];
            if (j < d - 1) I.lv_cb[j][u] = (j + 1 < d - 1) ? E[(j + 1) * R + c] : (int)c;
        }
        if (c == 0) {
            for (int j = 0; j < d; ++j) {
                const int nj = (j < d - 1) ? E[j * R + C] : C;
                I.small[kSmLevelCount + j] = nj;
                if (j < d - 1) I.lv_cb[j][nj] = (j + 1 < d - 1) ? E[(j + 1) * R + C] : C;
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
// [lo, hi) of level j, partial offset of the path above them, whether the
// path equals the query's own prefix).  Each step takes the entries of the
// top level -- up to 32 nodes across several ranges, the last range possibly
// split -- and the lanes test one node each: key within the window, offset
// within eps (and, at a leaf, the point-box test); surviving inner nodes push
// their child range narrowed to the child window (so no pushed node fails
// its key test), surviving leaves are the forward neighbours g' >= c: counted
// into nbr_fwd[c] and written -- at nbr + nbr_start[c] once the counts are
// scanned (kWalkFill), or to the pool in runs of up to kPoolRun (kWalkPool, see
// WalkPool) -- while each g' > c also counts (count and pool modes) or
// receives (fill mode) the backward entry c.  Every mode visits the nodes in
// the same order.
//
// Stack bound: levels never decrease from the bottom of the stack to its top
// (a step pops the top level j and pushes level j + 1), so a level receives
// pushes only when nothing deeper is left, and one step pushes at most 32
// entries.  Hence at most 32 entries per level below the root: 1 + 32 (d - 1).
constexpr int kWalkWarps = 4;
constexpr int kWalkStack = 1 + 32 * (kMaxD - 1);
// stack entry level byte: the level in the low bits, kTight when the path to
// the range equals the query's identifier prefix
constexpr int kTight = 0x10;

// Narrow the key-sorted range [*lo, *hi) to keys in [vlo, vhi]: the two
// bisections run side by side, so their loads overlap.
__device__ __forceinline__ void narrow_range(const int* __restrict__ key, int* lo, int* hi, int vlo, int vhi) {
    const int a = *lo, b = *hi;
    if (a >= b) return;
    // The keys are distinct increasing integers, so key[a + t] >= key[a] + t
    // and key[b - 1 - t] <= key[b - 1] - t: the two end keys bound where each
    // answer can lie, to within the key gaps (dense child ranges leave a few
    // candidates, sparse ones the whole range).
    const int ka = __ldg(key + a), kb = __ldg(key + b - 1);
    int l1, h1, l2, h2;  // first key >= vlo in [l1, h1]; first key > vhi in [l2, h2]
    if (vlo <= ka) {
        l1 = h1 = a;
    } else if (vlo > kb) {
        l1 = h1 = b;
    } else {
        l1 = max(a + 1, b - 1 - (kb - vlo));
        h1 = min(b - 1, a + (vlo - ka));
    }
    if (vhi < ka) {
        l2 = h2 = a;
    } else if (vhi >= kb) {
        l2 = h2 = b;
    } else {
        l2 = max(a + 1, b - (kb - vhi));
        h2 = min(b - 1, a + (vhi - ka) + 1);
    }
    while (l1 < h1 || l2 < h2) {
        const int m1 = (l1 + h1) >> 1, m2 = (l2 + h2) >> 1;
        const int k1 = l1 < h1 ? __ldg(key + m1) : 0;
        const int k2 = l2 < h2 ? __ldg(key + m2) : 0;
        if (l1 < h1) {
            if (k1 < vlo) l1 = m1 + 1;
            else h1 = m1;
        }
        if (l2 < h2) {
            if (k2 <= vhi) l2 = m2 + 1;
            else h2 = m2;
        }
    }
    *lo = l1;
    *hi = l2;
}

// The key offsets delta in [lo, hi] of one level whose squared gap (table
// gap2, index delta + kMaxR, non-decreasing in |delta| on each side, 0 at
// delta = 0) is within `rem`; lo >= 0 when `fwd` (a range on the query's own
// path).  rem >= 0, so delta = 0 always qualifies.
template <typename T>
__device__ __forceinline__ void budget_window(const T* gap2, T rem, int r, bool fwd, int* lo, int* hi) {
    int h = 0, l = 0;
#pragma unroll
    for (int t = 1; t <= kMaxR; ++t)
        if (t <= r && gap2[kMaxR + t] <= rem) h = t;
    if (!fwd) {
#pragma unroll
        for (int t = 1; t <= kMaxR; ++t)
            if (t <= r && gap2[kMaxR - t] <= rem) l = -t;
    }
    *lo = l;
    *hi = h;
}

// Offsets (partial sums of squared gaps) are 64-bit in general, 32-bit when
// the batch's eps2 < 2^31: the table entries are then saturated at eps2 + 1
// and a pushed path's offset is at most eps2, so no sum exceeds 2^32 - 1.
template <typename T>
struct WalkShared {
    int lo[kWalkWarps][kWalkStack];
    int hi[kWalkWarps][kWalkStack];
    T part[kWalkWarps][kWalkStack];
    signed char lvl[kWalkWarps][kWalkStack];
    int qlo[kWalkWarps][kMaxD], qhi[kWalkWarps][kMaxD];  // query point box
    int g[kWalkWarps][kMaxD];                                    // query identifier
    // squared gap in dimension j between the query's point box and the cell
    // at key offset delta = key - g_j, index delta + kMaxR (saturated above
    // eps2: at 2^62, or at eps2 + 1 for 32-bit offsets)
    T gap2[kWalkWarps][kMaxD][2 * kMaxR + 1];
    int buf[kWalkWarps][kPoolRun + 32];  // kWalkPool: neighbours not yet flushed
};

// kWalkPool: hand `len` buffered neighbours of query c (instance k), the run
// at offset `off` of its list, to the pool.
__device__ __forceinline__ void pool_flush(const WalkPool& pool, const int* buf, int len, int k, int c, int off,
                                           int lane) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(pool.ctr, (1ull << kPoolBits) | (unsigned long long)len);
    t = __shfl_sync(kFull, t, 0);
    const long long pos = (long long)(t & ((1ull << kPoolBits) - 1)), si = (long long)(t >> kPoolBits);
    if (pos + len <= pool.cap && si < pool.seg_cap) {
        for (int i = lane; i < len; i += 32) pool.data[pos + i] = buf[i];
        if (lane == 0) pool.seg[si] = PoolSeg{pos, k, c, off, len};
    }
}

// The backward entry c in the list of grid u > c (fill mode and the pool
// scatter): after the forward part, at the next free slot (nbr_bwd[u] holds
// that slot's absolute position from the list check on: one atomic, no
// other lookup).  Writes stay inside the list buffer whatever the counts say.
__device__ __forceinline__ void put_backward(const Inst& I, int u, int c) {
    const long long at = atomicAdd(I.nbr_bwd + u, 1);
    if (at >= 0 && at < I.nbr_cap) I.nbr[at] = c;
}

// Whether the neighbour lists of an instance were given up (see nbr_check).
__device__ __forceinline__ bool lists_dropped(const Inst& I) {
    return (*reinterpret_cast<const volatile unsigned*>(I.small + kSmStatus) & kDevOverflow) != 0;
}

// Whether the pool held the whole walk (else the lists are filled by a
// second walk).
__device__ __forceinline__ bool pool_fits(const WalkPool& pool) {
    if (!pool.data) return false;
    const unsigned long long t = *pool.ctr;
    return (long long)(t & ((1ull << kPoolBits) - 1)) <= pool.cap && (long long)(t >> kPoolBits) <= pool.seg_cap;
}

template <int MODE, typename T, int D>
__global__ void __launch_bounds__(32 * kWalkWarps)
    walk_kernel(const Inst* __restrict__ ins, Flat f, long long total, WalkPool pool) {
    total = flat_total(f);
    constexpr bool FILL = MODE == kWalkFill, POOL = MODE == kWalkPool;
    __shared__ WalkShared<T> sh;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    int* const slo = sh.lo[w];
    int* const shi = sh.hi[w];
    T* const spart = sh.part[w];
    signed char* const slvl = sh.lvl[w];
    const long long warps = (long long)gridDim.x * kWalkWarps;
    const unsigned lt = lanemask_lt();
    // the filling walk runs only when the pool could not hold the walk
    if (FILL && pool_fits(pool)) return;
    FlatCursor cur;
    for (long long q = (long long)blockIdx.x * kWalkWarps + w; q < total; q += warps) {
        cur.seek(f, q);
        const int kin = f.idx[cur.k];
        const Inst& I = ins[kin];
        if (FILL && lists_dropped(I)) continue;
        const long long c = q - cur.lo;
        constexpr int d = D;
        const long long r = I.p.r, s = I.p.s;
        const int ri = (int)r;  // <= kMaxR
        const T eps2 = (T)I.p.eps2;  // < 2^31 when T is 32-bit
        const long long sat = sizeof(T) == 8 ? (1ll << 62) : I.p.eps2 + 1;
        if (lane < d) {
            const int gi = I.cell_coord[c * d + lane];
            const long long g = gi, ql = I.pbox[c * 2 * d + lane], qh = I.pbox[c * 2 * d + d + lane];
            sh.qlo[w][lane] = ql;
            sh.qhi[w][lane] = qh;
            sh.g[w][lane] = gi;
            // the cell at offset delta spans [cl + delta s, cl + delta s + s - 1]
            const long long cl = (long long)I.p.mn[lane] + g * s;
#pragma unroll
            for (int t = 0; t <= 2 * kMaxR; ++t) {
                const long long dl = t - kMaxR;
                long long gap = 0;
                if (dl > 0) gap = cl + dl * s - qh;
                else if (dl < 0) gap = ql - (cl + dl * s + s - 1);
                sh.gap2[w][lane][t] = (T)(gap >= (1ll << 31) ? sat : min(gap * gap, sat));
            }
        }
        __syncwarp();
        const int* pbox = I.pbox;
        int* out = FILL ? I.nbr + I.nbr_start[c] : nullptr;
        int found = 0;
        int nbuf = 0;     // kWalkPool: buffered neighbours
        int flushed = 0;  // kWalkPool: neighbours already in the pool
        int* const buf = sh.buf[w];
        int top = 0;
        {
            // the root range: level-0 keys in [g_0, g_0 + r] (on the query's
            // path), narrowed to the offsets whose gap alone is within eps
            int a0 = 0, b0 = I.small[kSmLevelCount];
            int dlo, dhi;
            budget_window<T>(sh.gap2[w][0], eps2, ri, true, &dlo, &dhi);
            narrow_range(I.lv_key[0], &a0, &b0, sh.g[w][0] + dlo, sh.g[w][0] + dhi);
            if (b0 > a0) {
                if (lane == 0) {
                    slo[0] = a0;
                    shi[0] = b0;
                    spart[0] = 0;
                    slvl[0] = (signed char)kTight;
                }
                top = 1;
            }
        }
        __syncwarp();
        long long nodes = 0, steps = 0;  // statistics
        while (top > 0) {
            // the group: the entries of the top level, lane i holding entry top-1-i
            const int J = slvl[top - 1] & (kTight - 1);
            const int e = top - 1 - lane;
            const int ev = e >= 0 ? slvl[e] : -1;
            const bool in_group = e >= 0 && (ev & (kTight - 1)) == J;
            int elo = 0, sz = 0, etight = 0;
            T epart = 0;
            if (in_group) {
                elo = slo[e];
                sz = min(shi[e] - elo, 64);
                epart = spart[e];
                etight = ev & kTight;
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
            const int src = ei < 0 ? 0 : ei;
            const int my_lo = __shfl_sync(kFull, elo, src);
            const int my_start = __shfl_sync(kFull, start, src);
            const T my_part = __shfl_sync(kFull, epart, src);
            const int my_tight = __shfl_sync(kFull, etight, src);
            top -= consumed;
            nodes += taken;
            ++steps;
            __syncwarp();

            const bool act = lane < taken;
            const int u = my_lo + (lane - my_start);
            bool ok = false, tight = false;
            T off = 0;
            // Every range on the stack was narrowed to the keys whose gap fits
            // the budget its path left (the budget windows), so on consistent
            // data each node passes its key test: a leaf needs only its box
            // test.  An inner node needs its offset (for its children's
            // window), loaded with its child range (one round trip); its key
            // is still checked against the window, which keeps the table
            // index in bounds when the levels are inconsistent (a run whose
            // key layout did not fit its plan, discarded and run again).
            int clo = 0, chi = 0;
            if (act) {
                if (J < d - 1) {
                    const int key = __ldg(I.lv_key[J] + u);
                    clo = __ldg(I.lv_cb[J] + u);
                    chi = __ldg(I.lv_cb[J] + u + 1);
                    const int dl = key - sh.g[w][J];
                    if (dl >= -ri && dl <= ri) {
                        off = my_part + sh.gap2[w][J][dl + kMaxR];
                        ok = off <= eps2;
                        tight = my_tight && dl == 0;
                    }
                } else {
                    ok = true;
                }
            }
            if (J == d - 1) {
                // leaf: the two grids' boxes (a forward neighbour u >= c)
                if (ok) {
                    const int* ub = pbox + (long long)u * 2 * d;
                    // the box row (2d ints at 8d-byte steps from a 256-byte
                    // aligned base) by 16-byte loads for even d, 8-byte ones
                    // for odd d
                    int row[2 * D];
                    if constexpr (D % 2 == 0) {
#pragma unroll
                        for (int v = 0; v < D / 2; ++v) {
                            const int4 q = __ldg(reinterpret_cast<const int4*>(ub) + v);
                            row[4 * v] = q.x;
                            row[4 * v + 1] = q.y;
                            row[4 * v + 2] = q.z;
                            row[4 * v + 3] = q.w;
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < D; ++v) {
                            const int2 q = __ldg(reinterpret_cast<const int2*>(ub) + v);
                            row[2 * v] = q.x;
                            row[2 * v + 1] = q.y;
                        }
                    }
                    // coordinates span less than 2^31 per dimension (the
                    // range check), so each gap fits in 32 bits; its square
                    // and the sum take 64
                    long long g2 = 0;
#pragma unroll
                    for (int t = 0; t < d; ++t) {
                        const int bl = row[t], bh = row[d + t];
                        const int ql = sh.qlo[w][t], qh = sh.qhi[w][t];
                        int gg = 0;
                        if (bl > qh) gg = bl - qh;
                        else if (ql > bh) gg = ql - bh;
                        g2 += (long long)gg * gg;
                    }
                    ok = g2 <= eps2;
                }
                const unsigned m = __ballot_sync(kFull, ok);
                if (ok && u != (int)c) {
                    if (FILL)
                        put_backward(I, u, (int)c);
                    else
                        atomicAdd(I.nbr_bwd + u, 1);
                }
                if (FILL && ok) {
                    const int at = found + __popc(m & lt);
                    if (I.nbr_start[c] + (long long)at < I.nbr_cap) out[at] = u;
                }
                found += __popc(m);
                if (POOL) {
                    if (ok) buf[nbuf + __popc(m & lt)] = u;
                    nbuf += __popc(m);
                    __syncwarp();
                    if (nbuf >= kPoolRun) {
                        pool_flush(pool, buf, kPoolRun, kin, (int)c, flushed, lane);
                        flushed += kPoolRun;
                        nbuf -= kPoolRun;  // < 32 left
                        const int rest = lane < nbuf ? buf[kPoolRun + lane] : 0;
                        __syncwarp();
                        if (lane < nbuf) buf[lane] = rest;
                    }
                }
            } else {
                if (ok) {
                    // a child window: [g - r, g + r], or [g, g + r] below a node
                    // on the query's own path, narrowed to the key offsets whose
                    // gap still fits in what the path leaves of eps^2
                    int dlo, dhi;
                    budget_window<T>(sh.gap2[w][J + 1], eps2 - off, ri, tight, &dlo, &dhi);
                    const int g1 = sh.g[w][J + 1];
                    narrow_range(I.lv_key[J + 1], &clo, &chi, g1 + dlo, g1 + dhi);
                    ok = chi > clo;
                }
                const unsigned m = __ballot_sync(kFull, ok);
                if (ok) {
                    const int at = top + __popc(m & lt);
                    slo[at] = clo;
                    shi[at] = chi;
                    spart[at] = off;
                    slvl[at] = (signed char)((J + 1) | (tight ? kTight : 0));
                }
                top += __popc(m);
            }
            __syncwarp();
        }
        if (POOL && nbuf > 0) pool_flush(pool, buf, nbuf, kin, (int)c, flushed, lane);
        if (!FILL && lane == 0) {
            I.nbr_fwd[c] = found;
            stat_add(I.stats, kStWalkNodes, (unsigned long long)nodes);
            stat_add(I.stats, kStWalkSteps, (unsigned long long)steps);
        }
        __syncwarp();
    }
}

template <int D>
static void walk_d(const Inst* ins, Flat cells, long long total, int mode, WalkPool pool, int b, bool small_eps,
                   cudaStream_t st) {
#define GD_WALK(M, T) walk_kernel<M, T, D><<<b, 32 * kWalkWarps, 0, st>>>(ins, cells, total, pool)
    if (small_eps) {
        if (mode == kWalkFill) GD_WALK(kWalkFill, unsigned);
        else if (mode == kWalkPool) GD_WALK(kWalkPool, unsigned);
        else GD_WALK(kWalkCount, unsigned);
    } else {
        if (mode == kWalkFill) GD_WALK(kWalkFill, long long);
        else if (mode == kWalkPool) GD_WALK(kWalkPool, long long);
        else GD_WALK(kWalkCount, long long);
    }
#undef GD_WALK
}

cudaError_t launch_walk(const Inst* ins, Flat cells, long long total, int mode, WalkPool pool, int blocks,
                        bool small_eps, int d, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long b = (total + kWalkWarps - 1) / kWalkWarps;
    if (b > blocks) b = blocks;
    switch (d) {
#define GD_WD(DD) \
    case DD: walk_d<DD>(ins, cells, total, mode, pool, (int)b, small_eps, st); break;
        GD_WD(1) GD_WD(2) GD_WD(3) GD_WD(4) GD_WD(5) GD_WD(6) GD_WD(7) GD_WD(8)
#undef GD_WD
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// The pool's segments into the scanned lists, one warp per segment: each
// run of forward neighbours of query c goes to its place in c's list, and
// every neighbour u > c receives the backward entry c.
// The segment count is the pool counter's (read on the device); nothing is
// done when the pool overflowed (the filling walk runs instead).
__global__ void __launch_bounds__(256) pool_scatter_kernel(const Inst* __restrict__ ins, WalkPool pool) {
    if (!pool_fits(pool)) return;
    const long long nseg = (long long)(*pool.ctr >> kPoolBits);
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long sgi = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); sgi < nseg;
         sgi += warps) {
        const PoolSeg sg = pool.seg[sgi];
        const Inst& I = ins[sg.inst];
        if (lists_dropped(I)) continue;
        const long long base = (long long)I.nbr_start[sg.c] + sg.off;
        for (int i = lane; i < sg.len; i += 32) {
            const int u = pool.data[sg.pos + i];
            if (base + i < I.nbr_cap) I.nbr[base + i] = u;
            if (u != sg.c) put_backward(I, u, sg.c);
        }
    }
}

// After the list scan: an instance whose lists need more entries than its
// buffer holds (a capacity taken from an earlier call) gives them up -- every
// list empty, forward parts included, so that no later kernel reads an
// entry that was not written -- and records kDevOverflow: the call is then
// run again with exact sizes.
__global__ void nbr_check_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = i - cur.lo;
        if ((long long)(unsigned)I.small[kSmNnbr] > I.nbr_cap) {
            I.nbr_start[c] = 0;
            I.nbr_fwd[c] = 0;
            if (c == 0) {
                I.nbr_start[I.small[kSmCells]] = 0;
                set_status(I, kDevOverflow);
            }
        }
        // the cursor that places the backward entries: their first position
        I.nbr_bwd[c] = I.nbr_start[c] + I.nbr_fwd[c];
    }
}

cudaError_t launch_nbr_check(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    nbr_check_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// List lengths before the scan: forward + backward entries of each grid; the
// backward counts restart at zero as the cursors that place the entries.
__global__ void nbr_total_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = i - cur.lo;
        I.nbr_start[c] = I.nbr_fwd[c] + I.nbr_bwd[c];
    }
}

cudaError_t launch_nbr_total(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    nbr_total_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_pool_scatter(const Inst* ins, WalkPool pool, cudaStream_t st) {
    if (!pool.data || pool.seg_cap <= 0) return cudaSuccess;
    long long b = (pool.seg_cap * 32 + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    pool_scatter_kernel<<<(int)b, 256, 0, st>>>(ins, pool);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
