// Cluster ids and labels (Section 4.4, Alg. 6 step 4), over a batch.
//   - each union-find set of core grids is one cluster; its id is the smallest
//     input index among its core points;
//   - a non-core point is a border point if a core point lies within eps and
//     takes the smallest id among such points' clusters, else it is noise (-1).
#include <climits>

#include "gd_internal.cuh"

namespace gd {

static int blocks_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    return b < 1 ? 1 : (int)b;
}

#define GD_FOR_FLAT(i, total)                                                                         \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (total);                 \
         i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ const int* perm_of(const Inst& I) { return (I.passes & 1) ? I.valB : I.valA; }

// Point every core grid at its root and reset the per-root minimum.
template <bool CAP>
__global__ void uf_compress_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const int c = (int)(i - cur.lo);
        I.cid_root[c] = INT_MAX;
        if (I.core_start[c + 1] > I.core_start[c]) {
            // read-only: concurrent halving could undo this grid's pointer
            const int r = uf_find_ro<CAP>(I.parent, c, I.p.uf_cap);
            if (r < 0)
                set_status(I, kDevTimeout);
            else
                I.parent[c] = r;
        }
    }
}

// Grid order keeps input order inside a grid (the sort is stable), so the
// first core point of a grid has the grid's smallest core input index.
__global__ void cid_min_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const int c = (int)(i - cur.lo);
        if (I.core_start[c + 1] == I.core_start[c]) continue;
        int q = I.cell_start[c];
        while (!I.core_s[q]) ++q;
        atomicMin(I.cid_root + I.parent[c], perm_of(I)[q]);
    }
}

__global__ void cell_cid_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const int c = (int)(i - cur.lo);
        I.cell_cid[c] = I.core_start[c + 1] > I.core_start[c] ? I.cid_root[I.parent[c]] : -1;
    }
}

cudaError_t launch_cluster_ids(const Inst* ins, Flat cells, long long total, bool cap, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int nb = blocks_for(total);
    if (cap)
        uf_compress_kernel<true><<<nb, 256, 0, st>>>(ins, cells, total);
    else
        uf_compress_kernel<false><<<nb, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    cid_min_kernel<<<nb, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    cell_cid_kernel<<<nb, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// The label of non-core point q (grid c): the smallest cluster id among the
// core points within eps, scanning the neighbour grids' core points and
// skipping grids whose cluster id cannot improve the best found so far or
// whose core box is farther than eps; -1 (noise) if there is none.
template <int D>
__device__ __forceinline__ int border_label(const Inst& I, long long q, int c, unsigned& ndist) {
    constexpr int DP = Padded<D>::value;
    int x[D];
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = I.Xs[q * DP + j];
    const long long eps2 = I.p.eps2;
    int best = INT_MAX;
    for (int t = I.nbr_start[c]; t < I.nbr_start[c + 1]; ++t) {
        const int c2 = I.nbr[t];
        const int id = I.cell_cid[c2];
        if (id < 0 || id >= best) continue;
        const int* bb = I.bbox + (long long)c2 * 2 * D;
        long long g2 = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            long long g = 0;
            if (bb[j] > x[j]) g = (long long)bb[j] - x[j];
            else if (x[j] > bb[D + j]) g = (long long)x[j] - bb[D + j];
            g2 += g * g;
        }
        if (g2 > eps2) continue;
        const int* Y = core_rows(I, c2, DP);
        const int m2 = I.core_start[c2 + 1] - I.core_start[c2];
        for (int u = 0; u < m2; ++u) {
            int y[D];
#pragma unroll
            for (int j = 0; j < D; ++j) y[j] = Y[(long long)u * DP + j];
            ++ndist;
            if (sqdist<D>(x, y) <= eps2) {
                best = id;
                break;
            }
        }
    }
    return best == INT_MAX ? -1 : best;
}

// Labels and core flags in input order (Alg. 6 step 4).  Warps take chunks
// of kLabelChunk consecutive points of the flat space (grid order) in turn,
// lanes on consecutive points, four points per lane in flight: a core point
// takes its grid's cluster id, a non-core point searches its neighbour grids
// (border_label).  Small chunks spread regions of costly (non-core) points
// over many warps.
constexpr int kLabelChunk = 128;

template <int D>
__global__ void __launch_bounds__(256, D >= 5 ? 4 : 1) labels_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    constexpr int U = 4;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5);
    FlatCursor cur;
    for (long long beg = wid * kLabelChunk; beg < total; beg += nwarps * kLabelChunk) {
        const long long end = min(total, beg + kLabelChunk);
        long long i = beg + lane_id();
        while (i < end) {
            cur.seek(f, i);
            const Inst& I = ins[f.idx[cur.k]];
            const int* perm = perm_of(I);
            const long long stop = min(end, cur.hi);
            for (; i < stop; i += 32 * U) {
                int c[U], o[U];
                unsigned char core[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long q = i - cur.lo + 32 * u;
                    const bool v = i + 32 * u < stop;
                    c[u] = v ? I.pt_cell[q] : 0;
                    core[u] = v ? I.core_s[q] : 0;
                    o[u] = v ? perm[q] : -1;
                }
                int lab[U];
#pragma unroll
                for (int u = 0; u < U; ++u) lab[u] = (o[u] >= 0 && core[u]) ? I.cell_cid[c[u]] : -1;
                unsigned ndist = 0;  // statistics: distances evaluated
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (o[u] >= 0 && !core[u]) lab[u] = border_label<D>(I, i - cur.lo + 32 * u, c[u], ndist);
                stat_add(I.stats, kStDistLabels, ndist);
                // with core flags wanted: one packed word per point, split by
                // label_split_kernel (half the scattered writes)
                const bool packed = I.is_core != nullptr;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (o[u] >= 0)
                        I.labels[o[u]] = packed ? (int)((unsigned)(lab[u] + 1) | ((unsigned)(core[u] != 0) << 31))
                                                : lab[u];
            }
            if (i >= stop && stop < end) i = stop + ((i - stop) & 31);
        }
    }
}

// Input order, instances that want core flags: the packed word (label + 1,
// core flag in bit 31) in labels[] split into the label and the flag.
// Coalesced reads and writes.
__global__ void __launch_bounds__(256) label_split_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        if (!I.is_core) continue;
        const long long q = i - cur.lo;
        const unsigned v = (unsigned)I.labels[q];
        I.labels[q] = (int)(v & 0x7fffffffu) - 1;
        I.is_core[q] = (unsigned char)(v >> 31);
    }
}

cudaError_t launch_labels(const Inst* ins, Flat pts, long long total, int d, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int nb = blocks_for(total);
    switch (d) {
#define GD_LB(DD) \
    case DD: labels_kernel<DD><<<nb, 256, 0, st>>>(ins, pts, total); break;
        GD_LB(1) GD_LB(2) GD_LB(3) GD_LB(4) GD_LB(5) GD_LB(6) GD_LB(7) GD_LB(8)
#undef GD_LB
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    label_split_kernel<<<nb, 256, 0, st>>>(ins, pts, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
