// Cluster ids and labels (Section 4.4, Alg. 6 step 4).
//   - each union-find set of core grids is one cluster; its id is the smallest
//     input index among its core points;
//   - a non-core point is a border point if a core point lies within eps and
//     takes the smallest id among such points' clusters, else it is noise (-1).
#include <climits>

#include "gd_internal.cuh"

namespace gd {

// Point every core grid at its root and reset the per-root minimum.
__global__ void uf_compress_kernel(int* parent, const int* __restrict__ core_start, int C, int* __restrict__ cid_root,
                                   unsigned* status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    cid_root[c] = INT_MAX;
    if (core_start[c + 1] > core_start[c]) {
        const int r = uf_find(parent, c);
        if (r < 0)
            atomicOr(status, kDevTimeout);
        else
            parent[c] = r;
    }
}

// Grid order keeps input order inside a grid (the sort is stable), so the
// first core point of a grid has the grid's smallest core input index.
__global__ void cid_min_kernel(int minpts, const int* __restrict__ parent, const int* __restrict__ core_start,
                               const int* __restrict__ cell_start, const unsigned char* __restrict__ core_s,
                               const int* __restrict__ perm, int C, int* __restrict__ cid_root) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C || core_start[c + 1] == core_start[c]) return;
    int k = cell_start[c];
    while (!core_s[k]) ++k;
    atomicMin(cid_root + parent[c], perm[k]);
}

__global__ void cell_cid_kernel(const int* __restrict__ parent, const int* __restrict__ core_start, int C,
                                const int* __restrict__ cid_root, int* __restrict__ cell_cid) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    cell_cid[c] = core_start[c + 1] > core_start[c] ? cid_root[parent[c]] : -1;
}

cudaError_t launch_cluster_ids(const Params& p, int* parent, const int* core_start, const int* cell_start,
                               const unsigned char* core_s, const int* perm, int C, int* cid_root, int* cell_cid,
                               cudaStream_t st, unsigned* status) {
    const int nb = (C + 255) / 256;
    uf_compress_kernel<<<nb, 256, 0, st>>>(parent, core_start, C, cid_root, status);
    GD_COUNT_LAUNCH();
    cid_min_kernel<<<nb, 256, 0, st>>>(p.minpts, parent, core_start, cell_start, core_s, perm, C, cid_root);
    GD_COUNT_LAUNCH();
    cell_cid_kernel<<<nb, 256, 0, st>>>(parent, core_start, C, cid_root, cell_cid);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// One thread per point in grid order; writes labels and core flags in input
// order.  Non-core points scan their neighbour grids' core points, skipping
// grids whose cluster id cannot improve the best found so far.
template <int D, int DP>
__global__ void __launch_bounds__(256) labels_kernel(Params p, const int* __restrict__ Xs,
                                                     const int* __restrict__ pt_cell,
                                                     const unsigned char* __restrict__ core_s,
                                                     const int* __restrict__ nbr_start, const int* __restrict__ nbr,
                                                     const int* __restrict__ core_start, const int* __restrict__ Xc,
                                                     const int* __restrict__ bbox,
                                                     const int* __restrict__ cell_cid, const int* __restrict__ perm,
                                                     int* __restrict__ labels, unsigned char* __restrict__ is_core) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const int c = pt_cell[i];
        const unsigned char core = core_s[i];
        int lab;
        if (core) {
            lab = cell_cid[c];
        } else {
            int x[D];
#pragma unroll
            for (int j = 0; j < D; ++j) x[j] = Xs[i * DP + j];
            int best = INT_MAX;
            for (int t = nbr_start[c]; t < nbr_start[c + 1]; ++t) {
                const int c2 = nbr[t];
                const int id = cell_cid[c2];
                if (id < 0 || id >= best) continue;
                // skip a grid whose core points' box is farther than eps from x
                const int* bb = bbox + (long long)c2 * 2 * D;
                long long g2 = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    long long g = 0;
                    if (bb[j] > x[j]) g = (long long)bb[j] - x[j];
                    else if (x[j] > bb[D + j]) g = (long long)x[j] - bb[D + j];
                    g2 += g * g;
                }
                if (g2 > p.eps2) continue;
                for (int k = core_start[c2]; k < core_start[c2 + 1]; ++k) {
                    int y[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) y[j] = Xc[(long long)k * DP + j];
                    if (sqdist<D>(x, y) <= p.eps2) {
                        best = id;
                        break;
                    }
                }
            }
            lab = best == INT_MAX ? -1 : best;
        }
        const int o = perm[i];
        labels[o] = lab;
        if (is_core) is_core[o] = core;
    }
}

template <int D>
static void labels_launch(const Params& p, const int* Xs, const int* pt_cell, const unsigned char* core_s,
                          const int* nbr_start, const int* nbr, const int* core_start, const int* Xc,
                          const int* bbox, const int* cell_cid, const int* perm, int* labels, unsigned char* is_core,
                          cudaStream_t st) {
    constexpr int DP = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
    int blocks = (p.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    labels_kernel<D, DP><<<blocks, 256, 0, st>>>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox,
                                                 cell_cid, perm, labels, is_core);
    GD_COUNT_LAUNCH();
}

cudaError_t launch_labels(const Params& p, const int* Xs, const int* cell_start, const int* pt_cell,
                          const unsigned char* core_s, const int* nbr_start, const int* nbr, const int* core_start,
                          const int* Xc, const int* bbox, const int* cell_cid, const int* perm, int* labels,
                          unsigned char* is_core, cudaStream_t st) {
    (void)cell_start;
    switch (p.d) {
        case 1: labels_launch<1>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 2: labels_launch<2>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 3: labels_launch<3>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 4: labels_launch<4>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 5: labels_launch<5>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 6: labels_launch<6>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        case 7: labels_launch<7>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
        default: labels_launch<8>(p, Xs, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm, labels, is_core, st); break;
    }
    return cudaGetLastError();
}

}  // namespace gd
