// Grid tree and non-empty neighbouring grids (Section 4.2).
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
// (Eq. 2) stays within eps.  Offsets are exact integers: two grids whose
// identifiers differ by delta != 0 in one dimension hold integer points at
// least (|delta|-1)*s+1 apart there, and a neighbour needs the sum of the
// squares of those gaps to be <= eps2.
#include "gd_internal.cuh"

namespace gd {

size_t levels_tmp_ints(int C, int d) { return (size_t)(C + 1) * (size_t)d + (size_t)C + scan_tmp_ints(C); }

// L[c] = first dimension in which grid c differs from grid c-1 (0 for c = 0).
__global__ void level_diff_kernel(const int* __restrict__ coord, int C, int d, int* __restrict__ L) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int l = 0;
    if (c > 0) {
        l = d;
        for (int j = 0; j < d; ++j)
            if (coord[(long long)c * d + j] != coord[(long long)(c - 1) * d + j]) {
                l = j;
                break;
            }
    }
    L[c] = l;
}

// A grid c starts a node on level j iff L[c] <= j.
__global__ void level_flag_kernel(const int* __restrict__ L, int C, int j, int* __restrict__ f) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) f[c] = L[c] <= j ? 1 : 0;
}

// After the scans, E_j[c] (exclusive) is the node index on level j of the node
// starting at grid c, and E_j[C] the node count of level j.
__global__ void level_write_kernel(const int* __restrict__ coord, int C, int d, const int* __restrict__ L,
                                   const int* __restrict__ E, Levels lv) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) {
        const int l = L[c];
        for (int j = l; j < d; ++j) {
            const int u = (j < d - 1) ? E[(long long)j * (C + 1) + c] : c;
            lv.key[j][u] = coord[(long long)c * d + j];
            if (j < d - 1) lv.child_begin[j][u] = (j + 1 < d - 1) ? E[(long long)(j + 1) * (C + 1) + c] : c;
        }
    }
    if (c == 0) {
        for (int j = 0; j < d; ++j) {
            const int nj = (j < d - 1) ? E[(long long)j * (C + 1) + C] : C;
            lv.count[j] = nj;
            if (j < d - 1) lv.child_begin[j][nj] = (j + 1 < d - 1) ? E[(long long)(j + 1) * (C + 1) + C] : C;
        }
    }
}

cudaError_t build_levels(const Params& p, const int* cell_coord, int C, Levels lv, int* tmp, cudaStream_t st) {
    const int d = p.d;
    int* E = tmp;                                   // d x (C+1)
    int* L = tmp + (size_t)(C + 1) * d;             // C
    int* scan_tmp = L + C;
    const int tb = 256, nb = (C + tb - 1) / tb;
    level_diff_kernel<<<nb, tb, 0, st>>>(cell_coord, C, d, L);
    GD_COUNT_LAUNCH();
    for (int j = 0; j < d - 1; ++j) {
        int* Ej = E + (size_t)j * (C + 1);
        level_flag_kernel<<<nb, tb, 0, st>>>(L, C, j, Ej);
        GD_COUNT_LAUNCH();
        cudaError_t e = scan_exclusive(Ej, Ej, C, scan_tmp, st);
        if (e != cudaSuccess) return e;
    }
    level_write_kernel<<<nb, tb, 0, st>>>(cell_coord, C, d, L, E, lv);
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

// Depth-first walk of the levels for grid c (Alg. 3).  FILL == false counts
// the neighbours; FILL == true writes them at nbr + nbr_start[c] in
// lexicographic order (the query grid itself included).
template <bool FILL>
__global__ void __launch_bounds__(128) walk_kernel(Params p, const int* __restrict__ coord, int C, Levels lv,
                                                   int* __restrict__ cnt_or_start, int* __restrict__ nbr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int d = p.d;
    const long long r = p.r;
    const long long s = p.s, eps2 = p.eps2;
    int g[kMaxD];
    for (int j = 0; j < d; ++j) g[j] = coord[(long long)c * d + j];

    int cur[kMaxD], end[kMaxD];
    long long part[kMaxD];
    int* out = FILL ? nbr + cnt_or_start[c] : nullptr;
    int found = 0;

    int j = 0;
    part[0] = 0;
    end[0] = __ldg(lv.count);
    cur[0] = lower_key(lv.key[0], 0, end[0], (long long)g[0] - r);
    while (j >= 0) {
        if (cur[j] >= end[j]) {
            if (--j >= 0) cur[j]++;
            continue;
        }
        const int u = cur[j];
        const long long key = __ldg(lv.key[j] + u);
        if (key > (long long)g[j] + r) {
            if (--j >= 0) cur[j]++;
            continue;
        }
        const long long delta = key > g[j] ? key - g[j] : g[j] - key;
        const long long gap = delta == 0 ? 0 : (delta - 1) * s + 1;
        const long long off = part[j] + gap * gap;
        if (off > eps2) {
            cur[j]++;
            continue;
        }
        if (j == d - 1) {
            if (FILL) out[found] = u;
            found++;
            cur[j]++;
            continue;
        }
        const int* cb = lv.child_begin[j];
        const int lo = __ldg(cb + u), hi = __ldg(cb + u + 1);
        j++;
        part[j] = off;
        end[j] = hi;
        cur[j] = lower_key(lv.key[j], lo, hi, (long long)g[j] - r);
    }
    if (!FILL) cnt_or_start[c] = found;
}

cudaError_t launch_walk_count(const Params& p, const int* cell_coord, int C, Levels lv, int* nbr_count,
                              cudaStream_t st) {
    walk_kernel<false><<<(C + 127) / 128, 128, 0, st>>>(p, cell_coord, C, lv, nbr_count, nullptr);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_walk_fill(const Params& p, const int* cell_coord, int C, Levels lv, const int* nbr_start, int* nbr,
                             cudaStream_t st) {
    walk_kernel<true><<<(C + 127) / 128, 128, 0, st>>>(p, cell_coord, C, lv, const_cast<int*>(nbr_start), nbr);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
