// Merging core grids (Section 4.3, Def. 6-7), over a batch: two neighbouring
// core grids belong to one cluster iff some core point of one is within eps
// of some core point of the other.  The grids are joined with a lock-free
// union-find, as in the LDF variant (Section 5.2): a pair whose grids are
// already in one set is skipped before any distance is computed.
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

// ------------------------------------------------- core points per grid

// m_c (core points per grid, into core_start before its scan).
__global__ void core_count_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const long long c = i - cur.lo;
        const int b = I.cell_start[c], e = I.cell_start[c + 1];
        int m = e - b;
        if (m < I.p.minpts) {
            m = 0;
            for (int q = b; q < e; ++q) m += I.core_s[q];
        }
        I.core_start[c] = m;
        if (c == 0)
            for (int b = 0; b < kLdfBuckets; ++b) I.ldf_ctr[b] = 0;
    }
}

cudaError_t launch_core_count(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    core_count_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Core points of the grids that are not full packed contiguously (s_i of
// Section 4.3.1; a full grid's core points are its rows in Xs, see
// core_rows), and the box of each grid's core points, a thread per grid.  A
// full grid (all core, G13) takes its point box from the grid tree's build:
// the exact box for grids of at most 1024 points, the identifier range for
// larger ones.  Either holds all the grid's points, which is what the
// merge's box tests and the border search need (a larger box decides fewer
// pairs by box alone, never a pair wrongly), and dense grids fill their
// range.  So only the points of grids that are not full are read.  A grid
// without core points keeps an empty box (minima above maxima).
template <int D>
__global__ void __launch_bounds__(256) core_pack_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    constexpr int DP = Padded<D>::value;
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const Inst& I = ins[f.idx[cur.k]];
        const long long c = i - cur.lo;
        const int b = I.cell_start[c], e = I.cell_start[c + 1];
        int* box = I.bbox + c * 2 * D;
        if (e - b >= I.p.minpts) {
            const int* pb = I.pbox + c * 2 * D;
#pragma unroll
            for (int j = 0; j < 2 * D; ++j) box[j] = pb[j];
            continue;
        }
        int lo[D], hi[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            lo[j] = 0x7fffffff;
            hi[j] = (int)0x80000000;
        }
        int* out = I.Xc + (long long)I.core_start[c] * DP;
        for (int q = b; q < e; ++q) {
            if (!I.core_s[q]) continue;
            int x[DP];
            if constexpr (DP == 4) {
                const int4 v = *reinterpret_cast<const int4*>(I.Xs + (long long)q * 4);
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < DP; ++j) x[j] = I.Xs[(long long)q * DP + j];
            }
#pragma unroll
            for (int j = 0; j < DP; ++j) out[j] = x[j];
            out += DP;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                lo[j] = min(lo[j], x[j]);
                hi[j] = max(hi[j], x[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            box[j] = lo[j];
            box[D + j] = hi[j];
        }
    }
}

cudaError_t launch_core_pack(const Inst* ins, Flat cells, long long total, int d, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int nb = blocks_for(total);
    switch (d) {
#define GD_CP(DD) \
    case DD: core_pack_kernel<DD><<<nb, 256, 0, st>>>(ins, cells, total); break;
        GD_CP(1) GD_CP(2) GD_CP(3) GD_CP(4) GD_CP(5) GD_CP(6) GD_CP(7) GD_CP(8)
#undef GD_CP
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}



// ------------------------------------------------ candidate pair orders
// The merge takes every unordered pair of neighbouring core grids once,
// straight from the neighbour lists (no pair array), in one of two orders
// (Params::ldf):
//   - touching first: grid i takes the pairs (i, j), j > i, of its forward
//     list, in two waves -- touching grids (identifiers differ by at most 1
//     in every dimension) first, all others after them.  Touching core grids
//     are nearly always merged, so once the first wave has joined them the
//     union-find precheck skips most of the second.
//   - low density first (GriT-DBSCAN-LDF, Section 5.2): one wave in which the
//     core grids are visited in ascending order of core-point count
//     (launch_ldf_order), each taking the pairs of its forward list (every
//     pair once, at the slot of its grid that comes first in grid order).
//     Clusters form among the sparse grids' pairs first and the precheck
//     skips most of the rest.  (Taking each pair at the slot of its grid with
//     fewer core points instead, from whole lists, skipped as many pairs but
//     read twice the entries: 40-45% slower on sparse data.)

__device__ __forceinline__ int ldf_bucket(int m) {
    if (m <= 0) return kLdfBuckets - 1;  // not a core grid: last
    if (m < 64) return m - 1;
    return 63 + (31 - __clz(m)) - 5;  // 64..127 -> 64, 128..255 -> 65, ...
}

__device__ __forceinline__ int core_m(const Inst& I, int c) { return I.core_start[c + 1] - I.core_start[c]; }

// Pass 1: bucket counts (ldf_ctr zeroed by core_count_kernel).
// Pass 2 (RANK): each grid's slot in the order, after the counts became
// starts: ldf_grid[slot] = grid.
template <bool RANK>
__global__ void __launch_bounds__(256) ldf_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + lane_id();
        const bool valid = i < total;
        const Inst* I = nullptr;
        long long c = 0;
        int b = 0;
        if (valid) {
            cur.seek(f, i);
            I = ins + f.idx[cur.k];
            c = i - cur.lo;
            if (!I->p.ldf) I = nullptr;
            else b = ldf_bucket(core_m(*I, (int)c));
        }
        // lanes of different instances never share a counter: aggregate per instance
        const unsigned long long key = I ? ((unsigned long long)(size_t)I << 8) | (unsigned)b : 0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        int at = 0;
        if (I && (int)lane_id() == leader) at = atomicAdd(I->ldf_ctr + b, __popc(peers));
        at = __shfl_sync(kFull, at, leader) + __popc(peers & lanemask_lt());
        if (RANK && I) I->ldf_grid[at] = (int)c;
    }
}

// Exclusive scan of each LDF instance's bucket counts (one block each).
__global__ void __launch_bounds__(kLdfBuckets) ldf_scan_kernel(const Inst* __restrict__ ins, const int* __restrict__ idx) {
    __shared__ int sm[33];
    const Inst& I = ins[idx[blockIdx.x]];
    if (!I.p.ldf) return;
    const int v = I.ldf_ctr[threadIdx.x];
    int total;
    const int ex = block_exclusive_scan(v, sm, &total);
    I.ldf_ctr[threadIdx.x] = ex;
}

cudaError_t launch_ldf_order(const Inst* ins, const int* idx, int K, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0 || K <= 0) return cudaSuccess;
    const int nb = blocks_for(total);
    ldf_kernel<false><<<nb, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    ldf_scan_kernel<<<K, kLdfBuckets, 0, st>>>(ins, idx);
    GD_COUNT_LAUNCH();
    ldf_kernel<true><<<nb, 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------ union-find
// Of two roots, the one with the lower priority is linked under the other
// (atomicCAS on the root), and finds halve paths with plain stores: every
// stored parent is an ancestor, so concurrent halving never breaks a path.
// The priority is a fixed bijective hash of the index, not the index itself:
// grids are in lexicographic order, so index-ordered linking builds long
// chains along clusters, while a random-looking order keeps trees shallow.
// (Cluster ids do not depend on which grid ends up the root.)

__global__ void uf_init_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const long long c = i - cur.lo;
        ins[f.idx[k]].parent[c] = (int)c;
    }
}

cudaError_t launch_uf_init(const Inst* ins, Flat cells, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    uf_init_kernel<<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Between the waves: point every grid at its root, so that the second wave's
// precheck costs two loads per pair.
template <bool CAP>
__global__ void uf_flatten_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    FlatCursor cur;
    GD_FOR_FLAT(i, total) {
        cur.seek(f, i);
        const int k = cur.k;
        const Inst& I = ins[f.idx[k]];
        const int c = (int)(i - cur.lo);
        const int r = uf_find<CAP>(I.parent, c, I.p.uf_cap);
        if (r < 0)
            set_status(I, kDevTimeout);
        else if (r != c)
            I.parent[c] = r;
    }
}

cudaError_t launch_uf_flatten(const Inst* ins, Flat cells, long long total, bool cap, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (cap)
        uf_flatten_kernel<true><<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    else
        uf_flatten_kernel<false><<<blocks_for(total), 256, 0, st>>>(ins, cells, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Returns false if the retry cap was hit.
template <bool CAP>
__device__ __forceinline__ bool uf_union(int* parent, int a, int b, int cap) {
    for (int it = 0; it < (CAP ? cap : kMaxUfRetries); ++it) {
        a = uf_find<CAP>(parent, a, cap);
        b = uf_find<CAP>(parent, b, cap);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        if (uf_priority(a) < uf_priority(b)) {
            const int t = a;
            a = b;
            b = t;
        }
        // link root b (lower priority) under root a
        if (atomicCAS(parent + b, b, a) == b) return true;
    }
    return false;
}

// Both box tests of a candidate pair.  Returns 0 (no: boxes farther than
// eps), 1 (yes: the boxes are within eps even at their farthest corners) or
// -1 (undecided).
template <int D>
__device__ __forceinline__ int box_decision(const int* bi, const int* bj, long long eps2) {
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
    if (mind > eps2) return 0;
    if (maxd <= eps2) return 1;
    return -1;
}

// ----------------------------------------------------- the warp-level test
// One warp per core grid i (slot order: grid order, or the LDF order), over
// the pairs (i, j) it takes from its list (see above), 32 at a time, one per
// lane:
//   1. skip if the grids are already in one set;
//   2. the two box tests (they alone decide pairs of one-point grids);
//   3. pairs of at most `lane_limit` point pairs are decided by the lane
//      itself.
// The pairs still open are then taken one at a time by the whole warp: the
// exact test over core points in 32 x 32 tiles (lane l holds a point of s_j,
// points of s_i are broadcast), stopping at the first pair within eps.  Pairs
// of two small sets (both at most `small_set` points) are decided in full;
// any other pair gets `budget` diagonal tiles (distinct chunks of both sets),
// which finds a witness for nearly every pair that has many, and is otherwise
// handed to the block-level FastMerging kernel -- in particular a few points
// against thousands, where one scan of the large set usually decides.  Hard
// pairs of wave 1 are stored after wave 0's.
template <int D, bool CAP>
__global__ void __launch_bounds__(256, 4)  // latency-bound: four blocks per SM (64 registers)
    merge_list_kernel(const Inst* __restrict__ ins, Flat f, long long total, int wave, int budget, int lane_limit,
                      int small_set) {
    total = flat_total(f);
    constexpr int DP = Padded<D>::value;
    const int lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    FlatCursor cur;
    int acc_inst = -1;
    unsigned acc_pairs = 0;  // candidate pairs taken, flushed per instance
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        cur.seek(f, w);
        const int inst = f.idx[cur.k];
        const Inst& I = ins[inst];
        if (inst != acc_inst) {
            if (acc_inst >= 0 && lane == 0 && acc_pairs) atomicAdd(ins[acc_inst].small + kSmPairsT, (int)acc_pairs);
            acc_inst = inst;
            acc_pairs = 0;
        }
        const bool ldf = I.p.ldf != 0;
        if (ldf && wave == 1) continue;
        const long long slot = w - cur.lo;
        const int c = ldf ? I.ldf_grid[slot] : (int)slot;
        const int* core_start = I.core_start;
        const int mc = core_start[c + 1] - core_start[c];
        if (mc == 0) continue;
        const int d = I.p.d;
        const long long eps2 = I.p.eps2;
        int* parent = I.parent;
        const int cap = I.p.uf_cap;
        unsigned long long* const stv = I.stats;
        const int gl = lane < d ? I.cell_coord[(long long)c * d + lane] : 0;
        const int t_begin = I.nbr_start[c];
        const int t_end = t_begin + I.nbr_fwd[c];  // the forward part: pairs (c, j), j >= c
        const int hard_base = wave == 0 ? 0 : I.small[kSmHard0];
        // list entries and their core counts are loaded ahead (the entries two
        // chunks, the counts one chunk before use), so that their latency
        // overlaps the current chunk's union-find lookups
        const int* nbr = I.nbr;
        auto entry = [&](int t) { return t < t_end ? __ldg(nbr + t) : c; };
        auto cores = [&](int j) { return j != c ? __ldg(core_start + j + 1) - __ldg(core_start + j) : 0; };
        int j_next = entry(t_begin + lane);
        int m_next = cores(j_next);
        int j_after = entry(t_begin + 32 + lane);
        for (int t0 = t_begin; t0 < t_end; t0 += 32) {
            // ---- the lane's candidate pair (c, j2)
            const int j2 = j_next, mj = m_next;
            j_next = j_after;
            m_next = cores(j_after);
            j_after = entry(t0 + 64 + lane);
            bool keep;
            if (ldf) {
                keep = mj > 0;  // j2 != c (the self entry counts as no core points)
            } else {
                bool touching = true;
                for (int j = 0; j < d; ++j) {
                    const int gj = __shfl_sync(kFull, gl, j);
                    const int dl = I.cell_coord[(long long)j2 * d + j] - gj;
                    if (dl > 1 || dl < -1) touching = false;
                }
                keep = j2 > c && mj > 0 && touching == (wave == 0);
            }
            bool open = false;
            int outcome = -1;    // statistics: the slot that decided the lane's pair
            unsigned ndist = 0;  // statistics: distances this lane evaluated
            if (keep) {
                const int ra = uf_find<CAP>(parent, c, cap), rb = uf_find<CAP>(parent, j2, cap);
                if (ra < 0 || rb < 0) {
                    set_status(I, kDevTimeout);
                } else if (ra == rb) {
                    outcome = kStSkipped;
                } else {
                    const int dec =
                        box_decision<D>(I.bbox + (long long)c * 2 * D, I.bbox + (long long)j2 * 2 * D, eps2);
                    bool yes = dec == 1;
                    outcome = dec == 1 ? kStBoxYes : dec == 0 ? kStBoxNo : kStLane;
                    if (dec < 0) {
                        if ((long long)mc * mj <= lane_limit) {
                            const int* A = core_rows(I, c, DP);
                            const int* B = core_rows(I, j2, DP);
                            for (int u = 0; u < mc && !yes; ++u) {
                                int P[D];
#pragma unroll
                                for (int j = 0; j < D; ++j) P[j] = A[(long long)u * DP + j];
                                for (int v = 0; v < mj; ++v) {
                                    int Q[D];
#pragma unroll
                                    for (int j = 0; j < D; ++j) Q[j] = B[(long long)v * DP + j];
                                    ++ndist;
                                    if (sqdist<D>(P, Q) <= eps2) {
                                        yes = true;
                                        break;
                                    }
                                }
                            }
                        } else {
                            open = true;
                            outcome = -1;
                        }
                    }
                    if (yes && !uf_union<CAP>(parent, c, j2, cap)) set_status(I, kDevTimeout);
                }
            }
            acc_pairs += __popc(__ballot_sync(kFull, keep));
            if (stv) {
                stat_add(stv, kStPairs, keep ? 1 : 0);
                if (outcome >= 0) stat_add(stv, outcome, 1);
                stat_add(stv, kStDistMerge, ndist);
            }
            // ---- the open pairs, one at a time, by the whole warp
            unsigned pend = __ballot_sync(kFull, open);
            while (pend) {
                const int src = __ffs(pend) - 1;
                pend &= pend - 1;
                const int py = __shfl_sync(kFull, j2, src);
                int same = 0;
                if (lane == 0) {
                    const int ra = uf_find<CAP>(parent, c, cap), rb = uf_find<CAP>(parent, py, cap);
                    if (ra < 0 || rb < 0) set_status(I, kDevTimeout);
                    same = ra == rb;
                }
                if (__shfl_sync(kFull, same, 0)) {
                    if (lane == 0) stat_add(stv, kStSkipped, 1);
                    continue;
                }
                const int* A = core_rows(I, c, DP);
                const int* B = core_rows(I, py, DP);
                const int mi = mc;
                const int mjj = core_start[py + 1] - core_start[py];
                const int na = (mi + 31) >> 5, nb = (mjj + 31) >> 5;
                const long long tiles = (long long)na * nb;
                const bool exhaustive = mi <= small_set && mjj <= small_set;
                const long long limit = exhaustive ? tiles : (tiles < budget ? tiles : budget);
                bool yes = false;
                unsigned long long tile_dist = 0;
                for (long long tt = 0; tt < limit; ++tt) {
                    const int ta = exhaustive ? (int)(tt / nb) : (int)(tt % na);
                    const int tb = (int)(tt % nb);
                    const int a0 = ta << 5, b0 = tb << 5;
                    const int ca = min(32, mi - a0);
                    int P[D], Q[D];
                    const bool vq = b0 + lane < mjj;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        P[j] = lane < ca ? A[(long long)(a0 + lane) * DP + j] : 0;
                        Q[j] = vq ? B[(long long)(b0 + lane) * DP + j] : 0;
                    }
                    bool hit = false;
                    tile_dist += (unsigned long long)ca * (unsigned long long)min(32, mjj - b0);
                    for (int u = 0; u < ca; ++u) {
                        int pt[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) pt[j] = __shfl_sync(kFull, P[j], u);
                        hit |= vq && sqdist<D>(pt, Q) <= eps2;
                    }
                    if (__any_sync(kFull, hit)) {
                        yes = true;
                        break;
                    }
                }
                const bool handed = !yes && limit < tiles;
                if (lane == 0) {
                    stat_add(stv, handed ? kStHanded : kStWarp, 1);
                    stat_add(stv, kStDistMerge, tile_dist);
                    if (yes) {
                        if (!uf_union<CAP>(parent, c, py, cap)) set_status(I, kDevTimeout);
                    } else if (handed) {
                        I.hard[hard_base + atomicAdd(I.small + kSmHard0 + wave, 1)] = make_int2(c, py);
                    }
                }
            }
        }
    }
    if (acc_inst >= 0 && lane == 0 && acc_pairs) atomicAdd(ins[acc_inst].small + kSmPairsT, (int)acc_pairs);
}

cudaError_t launch_merge_list(const Inst* ins, Flat cells, long long total, int wave, int d, int budget,
                              int lane_limit, int small_set, bool cap, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long b = (total * 32 + 255) / 256;
    if (b > kPersistBlocks) b = kPersistBlocks;
    switch (d) {
#define GD_MW(DD)                                                                                                    \
    case DD:                                                                                                         \
        if (cap)                                                                                                     \
            merge_list_kernel<DD, true><<<(int)b, 256, 0, st>>>(ins, cells, total, wave, budget, lane_limit,       \
                                                                 small_set);                                       \
        else                                                                                                         \
            merge_list_kernel<DD, false><<<(int)b, 256, 0, st>>>(ins, cells, total, wave, budget, lane_limit,      \
                                                                  small_set);                                      \
        break;
        GD_MW(1) GD_MW(2) GD_MW(3) GD_MW(4) GD_MW(5) GD_MW(6) GD_MW(7) GD_MW(8)
#undef GD_MW
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------- FastMerging, per block
// Alg. 5 for one pair per block, exact:
//   p starts at the point of s_i nearest to the centre of s_j's box;
//   q = argmin over s_j of dist(p, .); yes if dist(p, q) <= eps;
//   otherwise prune s_i around p (Alg. 4), take p = argmin over the rest of
//   s_i of dist(., q), test, prune s_j around q, and repeat;
//   no as soon as a pruning empties a set (Thm. 2: only points with no
//   partner within eps are ever removed).
// Alg. 4 removes x from the set pruned around pivot p (nearest partner q,
// dist(p, q) > eps) when
//   - triangle: dist(x, p) < dist(p, q) - eps, decided in exact integers;
//   - angle (Def. 8, Thm. 1): the angle between pq and px exceeds
//     lambda = max over the other set's live points y of
//     arcsin(eps / |py|) + angle(pq, py).
// The angle test runs in single precision on exact int64 inputs (squared
// lengths and dot products, each rounded once to float) and prunes only with
// a margin: cos(angle(pq, px)) < cos(lambda) - kAngleMargin, and never when
// some lambda_y may reach pi (cos is decreasing only on [0, pi]).  Every
// quantity is a handful of correctly rounded IEEE operations (+, -, *, /,
// sqrt: relative error at most 2^-24 each; Higham, "Accuracy and Stability
// of Numerical Algorithms", 2nd ed., Sec. 2.2 and Lemma 3.1) on values of
// magnitude at most 1, so the computed cosines are within 1e-6 of the exact
// ones; the margin of 1e-4 makes every angle prune one the exact test would
// also make.  Pruning less never changes the answer (Thm. 2), only the
// number of rounds.  (Single precision: this GPU's double-precision rate is
// a small fraction of its single-precision rate.)
// s_i is the smaller set.  Each pruning is fused with the next argmin, so a
// round is three passes over live points (the angle bound, then the pruning
// with the argmin).  Every round removes p from s_i and q from s_j, so the
// loop ends after at most min(m_i, m_j) rounds.  The live sets are bitmaps
// (one word per 32 points) in the block's slice of the scratch.

constexpr float kAngleMargin = 1e-4f;
constexpr float kNoAngle = -4.0f;  // cos(lambda) sentinel: no angle pruning

__device__ __forceinline__ bool triangle_trivial(long long A, long long B, long long eps2) {
    // x is trivial iff sqrt(A) + sqrt(eps2) < sqrt(B)
    //   <=> B - A - eps2 > 0 and 4*A*eps2 < (B - A - eps2)^2   (B > eps2)
    const long long t = B - A - eps2;
    if (t <= 0) return false;
    const unsigned __int128 lhs = (unsigned __int128)4 * (unsigned long long)A * (unsigned long long)eps2;
    const unsigned __int128 rhs = (unsigned __int128)(unsigned long long)t * (unsigned long long)t;
    return lhs < rhs;
}

struct BestPt {
    long long d;
    int i;
};

__device__ __forceinline__ BestPt better(BestPt a, BestPt b) {
    if (b.d < a.d || (b.d == a.d && b.i < a.i)) return b;
    return a;
}

constexpr int kFmBlock = 256;
constexpr int kFmWarps = kFmBlock / 32;

// Block-wide argmin and live count; every thread gets the result.
__device__ __forceinline__ BestPt block_best(BestPt v, int cnt, BestPt* sb, int* sc, int* total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        BestPt u;
        u.d = __shfl_down_sync(kFull, v.d, o);
        u.i = __shfl_down_sync(kFull, v.i, o);
        v = better(v, u);
        cnt += __shfl_down_sync(kFull, cnt, o);
    }
    if (lane == 0) {
        sb[warp] = v;
        sc[warp] = cnt;
    }
    __syncthreads();
    BestPt r = sb[0];
    int c = sc[0];
#pragma unroll
    for (int w = 1; w < kFmWarps; ++w) {
        r = better(r, sb[w]);
        c += sc[w];
    }
    *total = c;
    __syncthreads();
    return r;
}

// Block-wide minimum of a float; every thread gets it.
__device__ __forceinline__ float block_min(float v, float* sd) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_down_sync(kFull, v, o));
    if (lane == 0) sd[warp] = v;
    __syncthreads();
    float r = sd[0];
#pragma unroll
    for (int w = 1; w < kFmWarps; ++w) r = fminf(r, sd[w]);
    __syncthreads();
    return r;
}

template <int D, int DP>
__device__ __forceinline__ void load_pt(const int* __restrict__ S, int k, int* x) {
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = S[(long long)k * DP + j];
}

template <int D>
__device__ __forceinline__ long long sqdist_ll(const int* a, const long long* b) {
    long long s = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const long long t = (long long)a[j] - b[j];
        s += t * t;
    }
    return s;
}

// (u - o) . (v - o) for integer points; |result| < 2^62 (Cauchy-Schwarz and
// the coordinate range check d * R^2 < 2^62).
template <int D>
__device__ __forceinline__ long long dot_from(const long long* o, const long long* u, const int* v) {
    long long s = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) s += (u[j] - o[j]) * ((long long)v[j] - o[j]);
    return s;
}

// cos(lambda) of the angle test for pruning around pivot p with nearest
// partner q (|pq|^2 = a2 > eps2): the minimum over the live points y of the
// other set S of cos(arcsin(eps / |py|) + angle(pq, py)), or kNoAngle when
// some lambda_y may reach pi.
template <int D, int DP>
__device__ float fm_cos_lambda(const int* __restrict__ S, int m, const unsigned* live, const long long* p,
                               const long long* q, long long a2, long long eps2, float* sd,
                               unsigned long long* ndist) {
    const int lane = lane_id();
    const float a = sqrtf((float)a2), eps = sqrtf((float)eps2);
    float best = 2.0f;
    int nlive = 0;
    for (int base = 0; base < m; base += kFmBlock) {
        const int k = base + threadIdx.x;
        const unsigned word = k < m ? live[k >> 5] : 0u;
        if ((word >> lane) & 1u) {
            int y[D];
            load_pt<D, DP>(S, k, y);
            const long long b2 = sqdist_ll<D>(y, p);  // >= a2 > eps2 (q is p's nearest)
            const long long dt = dot_from<D>(p, q, y);
            const float b = sqrtf((float)b2);
            const float sin_a = eps / b, cos_a = sqrtf((float)(b2 - eps2)) / b;
            float cos_t = (float)dt / (a * b);
            cos_t = fminf(1.0f, fmaxf(-1.0f, cos_t));
            const float sin_t = sqrtf(fmaxf(0.0f, 1.0f - cos_t * cos_t));
            // lambda_y < pi  <=>  cos(theta) + cos(alpha) > 0
            const float v = (cos_t + cos_a > kAngleMargin) ? cos_a * cos_t - sin_a * sin_t : kNoAngle;
            best = fminf(best, v);
            ++nlive;
        }
    }
    if (ndist) {
        nlive = __reduce_add_sync(kFull, nlive);
        if (lane == 0) atomicAdd(ndist, (unsigned long long)nlive);
    }
    return block_min(best, sd);
}

// One pass over a live set S (bitmap `live`, m points): optionally prune
// around pivot `piv` (nearest partner `near` of the other set at squared
// distance B, cos(lambda) = cl), and return the argmin of the distance to
// `near` over the points kept, plus their count.  Without pruning, `near` is
// only the target of the argmin.
template <int D, int DP, bool PRUNE>
__device__ BestPt fm_pass(const int* __restrict__ S, int m, unsigned* live, const long long* piv, long long B,
                          const long long* near, float cl, long long eps2, BestPt* sb, int* sc, int* count,
                          int* pruned_tri, int* pruned_ang, unsigned long long* ndist) {
    const int lane = lane_id();
    BestPt best{0x7fffffffffffffffll, 0x7fffffff};
    int cnt = 0, ntri = 0, nang = 0;
    const float sqB = PRUNE ? sqrtf((float)B) : 0.0f;
    for (int base = 0; base < m; base += kFmBlock) {
        const int k = base + threadIdx.x;
        // the 32 lanes of a warp hold one bitmap word's 32 points; lane 0 has
        // the lowest, so the word exists whenever lane 0 is inside the set
        const unsigned word = k < m ? live[k >> 5] : 0u;
        bool alive = (word >> lane) & 1u;
        int x[D];
        if (alive) {
            load_pt<D, DP>(S, k, x);
            if (PRUNE) {
                const long long A = sqdist_ll<D>(x, piv);
                if (triangle_trivial(A, B, eps2)) {
                    alive = false;
                    ++ntri;
                } else if (cl > kNoAngle && A > 0) {
                    const float cg = (float)dot_from<D>(piv, near, x) / (sqB * sqrtf((float)A));
                    if (cg < cl - kAngleMargin) {
                        alive = false;
                        ++nang;
                    }
                }
            }
        }
        if (PRUNE) {
            const unsigned nw = __ballot_sync(kFull, alive);
            if (lane == 0 && k < m && nw != word) live[k >> 5] = nw;
        }
        if (alive) {
            cnt++;
            best = better(best, BestPt{sqdist_ll<D>(x, near), k});
        }
    }
    if (pruned_tri) {
        // statistics: a pruning pass evaluates the distance to the pivot for
        // every live point and to the target for every kept one
        const int nlive = __reduce_add_sync(kFull, cnt + ntri + nang);
        const int nkept = __reduce_add_sync(kFull, cnt);
        ntri = __reduce_add_sync(kFull, ntri);
        nang = __reduce_add_sync(kFull, nang);
        if (lane == 0) {
            atomicAdd(pruned_tri, ntri);
            atomicAdd(pruned_ang, nang);
            atomicAdd(ndist, (unsigned long long)(PRUNE ? nlive + nkept : nkept));
        }
    }
    return block_best(best, cnt, sb, sc, count);
}

template <int D, bool CAP>
__global__ void __launch_bounds__(kFmBlock, 3) merge_block_kernel(const Inst* __restrict__ ins, Flat f, int wave,
                                                               unsigned* scratch, int wpb) {
    constexpr int DP = Padded<D>::value;
    __shared__ BestPt sb[kFmWarps];
    __shared__ int sc[kFmWarps];
    __shared__ float sd[kFmWarps];
    __shared__ int s_same;
    __shared__ int s_tri, s_ang;  // statistics: points pruned by each test
    __shared__ unsigned long long s_dist;  // statistics: distances evaluated
    unsigned* live_a = scratch + (long long)blockIdx.x * 2 * wpb;
    unsigned* live_b = live_a + wpb;
    const long long total = flat_total(f);
    for (long long h = blockIdx.x; h < total; h += gridDim.x) {
        const int kk = flat_find(f, h);
        const Inst& I = ins[f.idx[kk]];
        const long long eps2 = I.p.eps2;
        const long long yes2 = I.p.eps2_yes;  // eps2, or (eps + delta)^2 in approximate FastMerging
        const int base = wave == 0 ? 0 : I.small[kSmHard0];
        const int2 pr = I.hard[base + (h - f.off[kk])];
        int* parent = I.parent;
        unsigned long long* const stv = I.stats;
        if (threadIdx.x == 0) {
            const int ra = uf_find<CAP>(parent, pr.x, I.p.uf_cap), rb = uf_find<CAP>(parent, pr.y, I.p.uf_cap);
            if (ra < 0 || rb < 0) set_status(I, kDevTimeout);
            s_same = ra == rb;
            s_tri = 0;
            s_ang = 0;
            s_dist = 0;
        }
        __syncthreads();
        const bool same = s_same;
        __syncthreads();
        if (same) {
            if (threadIdx.x == 0) stat_add(stv, kStSkipped, 1);
            continue;
        }
        int* const ptri = stv ? &s_tri : nullptr;
        int* const pang = stv ? &s_ang : nullptr;
        unsigned long long* const pdist = stv ? &s_dist : nullptr;

        // s_i is the smaller set: each round removes at least its pivot, and
        // a small set is usually emptied by the first pruning
        const int* core_start = I.core_start;
        int gi = pr.x, gj = pr.y;
        if (core_start[gi + 1] - core_start[gi] > core_start[gj + 1] - core_start[gj]) {
            gi = pr.y;
            gj = pr.x;
        }
        const int* A = core_rows(I, gi, DP);
        const int* B = core_rows(I, gj, DP);
        const int ma = core_start[gi + 1] - core_start[gi];
        const int mb = core_start[gj + 1] - core_start[gj];
        const int wa = (ma + 31) >> 5, wb = (mb + 31) >> 5;
        if (wa > wpb || wb > wpb) {
            // the block's bitmaps (sized from an earlier call's largest grid)
            // are too small: the call is run again with exact sizes
            if (threadIdx.x == 0) set_status(I, kDevOverflow);
            __syncthreads();
            continue;
        }
        for (int w = threadIdx.x; w < wa; w += kFmBlock)
            live_a[w] = (w < wa - 1 || (ma & 31) == 0) ? 0xffffffffu : ((1u << (ma & 31)) - 1u);
        for (int w = threadIdx.x; w < wb; w += kFmBlock)
            live_b[w] = (w < wb - 1 || (mb & 31) == 0) ? 0xffffffffu : ((1u << (mb & 31)) - 1u);
        __syncthreads();

        long long piv[D], tgt[D];
        const int* bj = I.bbox + (long long)gj * 2 * D;
#pragma unroll
        for (int j = 0; j < D; ++j) tgt[j] = ((long long)bj[j] + bj[D + j]) / 2;
        int cnt;
        BestPt bp = fm_pass<D, DP, false>(A, ma, live_a, nullptr, 0, tgt, 0.0f, eps2, sb, sc, &cnt, ptri, pang, pdist);
        int px[D];
        load_pt<D, DP>(A, bp.i, px);
#pragma unroll
        for (int j = 0; j < D; ++j) piv[j] = px[j];
        BestPt bq = fm_pass<D, DP, false>(B, mb, live_b, nullptr, 0, piv, 0.0f, eps2, sb, sc, &cnt, ptri, pang, pdist);
        bool yes = false;
        int kappa = 1;  // rounds: one per nearest point q found in s_j
        for (int round = 0; round <= ma + mb; ++round) {
            if (bq.d <= yes2) {
                yes = true;
                break;
            }
            // prune s_i around p (nearest partner q at distance^2 bq.d), then p' = argmin over s_i of dist(., q)
            int qx[D];
            load_pt<D, DP>(B, bq.i, qx);
            long long qv[D];
#pragma unroll
            for (int j = 0; j < D; ++j) qv[j] = qx[j];
            float cl = fm_cos_lambda<D, DP>(B, mb, live_b, piv, qv, bq.d, eps2, sd, pdist);
            bp = fm_pass<D, DP, true>(A, ma, live_a, piv, bq.d, qv, cl, eps2, sb, sc, &cnt, ptri, pang, pdist);
            if (cnt == 0) break;
            if (bp.d <= yes2) {
                yes = true;
                break;
            }
            load_pt<D, DP>(A, bp.i, px);
#pragma unroll
            for (int j = 0; j < D; ++j) piv[j] = px[j];
            // prune s_j around q (nearest partner p' at distance^2 bp.d), then q' = argmin over s_j of dist(p', .)
            cl = fm_cos_lambda<D, DP>(A, ma, live_a, qv, piv, bp.d, eps2, sd, pdist);
            bq = fm_pass<D, DP, true>(B, mb, live_b, qv, bp.d, piv, cl, eps2, sb, sc, &cnt, ptri, pang, pdist);
            if (cnt == 0) break;
            ++kappa;
        }
        if (threadIdx.x == 0) {
            if (yes && !uf_union<CAP>(parent, pr.x, pr.y, I.p.uf_cap)) set_status(I, kDevTimeout);
            if (stv) {
                stat_add(stv, yes ? kStFmYes : kStFmNo, 1);
                stat_add(stv, kStKappa + min(kappa, (int)kKappaBins) - 1, 1);
                stat_add(stv, kStFmTriangle, (unsigned long long)s_tri);
                stat_add(stv, kStFmAngle, (unsigned long long)s_ang);
                stat_add(stv, kStDistFm, s_dist);
            }
        }
        __syncthreads();
    }
}


cudaError_t launch_merge_block(const Inst* ins, Flat hard, int wave, int d, int blocks, unsigned* scratch, int wpb,
                               bool cap, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    switch (d) {
#define GD_MB(DD)                                                                                       \
    case DD:                                                                                            \
        if (cap)                                                                                        \
            merge_block_kernel<DD, true><<<blocks, kFmBlock, 0, st>>>(ins, hard, wave, scratch, wpb);  \
        else                                                                                            \
            merge_block_kernel<DD, false><<<blocks, kFmBlock, 0, st>>>(ins, hard, wave, scratch, wpb); \
        break;
        GD_MB(1) GD_MB(2) GD_MB(3) GD_MB(4) GD_MB(5) GD_MB(6) GD_MB(7) GD_MB(8)
#undef GD_MB
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
