// Grid construction over a batch: bounds (mn_j of Eq. 1) and the
// non-empty-grid compaction of Alg. 1, plus the segmented scan and device-side
// flat offsets every stage uses.  Identifiers and the sort are in sort.cu.
#include <climits>

#include "gd_internal.cuh"

namespace gd {

// ------------------------------------------------------- segmented scan
// Three phases: per-tile sums, one block per segment scanning its tiles'
// sums, per-tile scan.  A tile never spans two segments.  A segment's tiles
// are laid out for its length bound; with a device-side length the tiles
// past it hold nothing, and the tile kernels loop over the tiles from a
// bounded grid, so unused tiles cost one test each.

constexpr int kScanBlock = 256;
constexpr int kScanItems = kScanTile / kScanBlock;
constexpr int kScanGrid = 152 * 8;  // blocks of the tile kernels (grid-stride over tiles)

__device__ __forceinline__ int seg_of_tile(const ScanSeg* segs, int K, long long b) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].blk0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kScanBlock) seg_reduce_kernel(const ScanSeg* __restrict__ segs, int K,
                                                                long long total_tiles, int* __restrict__ bsum) {
    __shared__ int sm[33];
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const ScanSeg sg = segs[seg_of_tile(segs, K, t)];
        const long long len = seg_len(sg);
        const long long base = (t - sg.blk0) * (long long)kScanTile;
        if (base >= len) {  // past the segment's length: block-uniform
            if (threadIdx.x == 0) bsum[t] = 0;
            continue;
        }
        const long long at = base + (long long)threadIdx.x * kScanItems;
        int s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i)
            if (at + i < len) s += sg.in[at + i];
        int total;
        block_exclusive_scan(s, sm, &total);
        if (threadIdx.x == 0) bsum[t] = total;
    }
}

// One block per segment: exclusive scan of its tiles' sums in place; the
// segment total goes to out[len].
__global__ void __launch_bounds__(1024) seg_top_kernel(const ScanSeg* __restrict__ segs, int* __restrict__ bsum,
                                                       long long total_tiles) {
    __shared__ int sm[33];
    const ScanSeg sg = segs[blockIdx.x];
    const long long len = seg_len(sg);
    long long end = (blockIdx.x + 1 < gridDim.x) ? segs[blockIdx.x + 1].blk0 : total_tiles;
    end = min(end, sg.blk0 + (len + kScanTile - 1) / kScanTile);
    int carry = 0;
    for (long long base = sg.blk0; base < end; base += 1024) {
        const long long k = base + threadIdx.x;
        const int v = k < end ? bsum[k] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sm, &total);
        if (k < end) bsum[k] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        sg.out[len] = carry;
        if (sg.tot) *sg.tot = carry;
    }
}

__global__ void __launch_bounds__(kScanBlock) seg_down_kernel(const ScanSeg* __restrict__ segs, int K,
                                                              long long total_tiles, const int* __restrict__ bsum) {
    __shared__ int sm[33];
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const ScanSeg sg = segs[seg_of_tile(segs, K, t)];
        const long long len = seg_len(sg);
        const long long base = (t - sg.blk0) * (long long)kScanTile;
        if (base >= len) continue;
        const long long at = base + (long long)threadIdx.x * kScanItems;
        int v[kScanItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (at + i < len) ? sg.in[at + i] : 0;
            s += v[i];
        }
        int total;
        int run = bsum[t] + block_exclusive_scan(s, sm, &total);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (at + i < len) sg.out[at + i] = run;
            run += v[i];
        }
    }
}

// One block per segment scans it in chunks of 1024 x 8 elements, carrying the
// running total (for short segments: one launch instead of three).
constexpr int kScanOneItems = 8;
__global__ void __launch_bounds__(1024) seg_single_kernel(const ScanSeg* __restrict__ segs) {
    __shared__ int sm[33];
    const ScanSeg sg = segs[blockIdx.x];
    const long long len = seg_len(sg);
    int carry = 0;
    for (long long base = 0; base < len; base += 1024 * kScanOneItems) {
        const long long at = base + (long long)threadIdx.x * kScanOneItems;
        int v[kScanOneItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kScanOneItems; ++i) {
            v[i] = at + i < len ? sg.in[at + i] : 0;
            s += v[i];
        }
        int total;
        int run = carry + block_exclusive_scan(s, sm, &total);
#pragma unroll
        for (int i = 0; i < kScanOneItems; ++i) {
            if (at + i < len) sg.out[at + i] = run;
            run += v[i];
        }
        carry += total;
    }
    if (threadIdx.x == 0) {
        sg.out[len] = carry;
        if (sg.tot) *sg.tot = carry;
    }
}

cudaError_t scan_segments(const ScanSeg* segs, int K, long long total_tiles, int* tmp, cudaStream_t st,
                          long long longest) {
    if (K <= 0) return cudaSuccess;
    if (longest >= 0 && longest <= kScanOneLaunch) {
        seg_single_kernel<<<K, 1024, 0, st>>>(segs);
        GD_COUNT_LAUNCH();
        return cudaGetLastError();
    }
    const int grid = (int)(total_tiles < kScanGrid ? (total_tiles > 0 ? total_tiles : 1) : kScanGrid);
    if (total_tiles > 0) {
        seg_reduce_kernel<<<grid, kScanBlock, 0, st>>>(segs, K, total_tiles, tmp);
        GD_COUNT_LAUNCH();
    }
    seg_top_kernel<<<K, 1024, 0, st>>>(segs, tmp, total_tiles);
    GD_COUNT_LAUNCH();
    if (total_tiles > 0) {
        seg_down_kernel<<<grid, kScanBlock, 0, st>>>(segs, K, total_tiles, tmp);
        GD_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

// ------------------------------------------------------ flat offsets

__global__ void count_flat_kernel(const Inst* __restrict__ ins, const int* __restrict__ idx, int K, int slot,
                                  long long* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    off[0] = 0;
    for (int k = 0; k < K; ++k) {
        run += ins[idx[k]].small[slot];
        off[k + 1] = run;
    }
}

cudaError_t count_flat(const Inst* ins, const int* idx, int K, int slot, long long* off, cudaStream_t st) {
    count_flat_kernel<<<1, 32, 0, st>>>(ins, idx, K, slot, off);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

__global__ void count_flats_kernel(const Inst* __restrict__ ins, const FlatSpec* __restrict__ specs, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const FlatSpec sp = specs[t];
        long long run = 0;
        sp.off[0] = 0;
        for (int k = 0; k < sp.m; ++k) {
            run += ins[sp.idx[k]].small[sp.slot];
            sp.off[k + 1] = run;
        }
    }
}

cudaError_t count_flats(const Inst* ins, const FlatSpec* specs, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_flats_kernel<<<(n + 63) / 64, 64, 0, st>>>(ins, specs, n);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- layout

__device__ __forceinline__ int bit_length_u64(unsigned long long v) { return v ? 64 - __clzll(v) : 0; }

__global__ void layout_kernel(Inst* __restrict__ ins, int K) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        Inst& I = ins[k];
        Params& p = I.p;
        unsigned long long rmax = 0;
        int total_bits = 0;
        for (int j = 0; j < p.d; ++j) {
            const long long lo = I.small[kSmMnmx + j], up = I.small[kSmMnmx + kMaxD + j];
            const unsigned long long rj = (unsigned long long)(up - lo);
            if (rj > rmax) rmax = rj;
            p.mn[j] = (int)lo;
            p.bits[j] = bit_length_u64(rj / (unsigned long long)p.s);
            total_bits += p.bits[j];
        }
        for (int j = p.d - 1, sh = 0; j >= 0; --j) {
            p.shift[j] = sh;
            sh += p.bits[j];
        }
        p.key_bits = total_bits;
        I.small[kSmKeyBits] = total_bits;
        unsigned st = 0;
        // d * rmax^2 >= 2^62, in 128 bits
        const unsigned long long r2lo = rmax * rmax, r2hi = __umul64hi(rmax, rmax);
        const unsigned long long dlo = r2lo * (unsigned long long)p.d;
        const unsigned long long dhi = r2hi * (unsigned long long)p.d + __umul64hi(r2lo, (unsigned long long)p.d);
        if (dhi != 0 || dlo >= (1ull << 62) || total_bits > 128) st |= kDevRange;
        // the plan's passes cover the key; the key class holds it
        const int cap = I.passes * I.digit_bits;
        const bool fits = total_bits <= cap &&
                          (p.key_class == 2 ? total_bits <= 128
                                            : (p.key_class == 1 ? total_bits <= 64 : total_bits + p.pack_bits <= 64));
        if (!fits) st |= kDevReplan;
        if (st) atomicOr(reinterpret_cast<unsigned*>(I.small + kSmStatus), st);
    }
}

cudaError_t launch_layout(Inst* ins, int K, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    layout_kernel<<<(K + 63) / 64, 64, 0, st>>>(ins, K);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bounds

// Per-dimension min and max (mn_j of Eq. 1).  Each warp takes a contiguous
// chunk of the flat point space (lanes on consecutive points, so rows are read
// coalesced); a lane accumulates in registers while its points stay in one
// instance and flushes with atomics when it moves to the next one (rare: only
// at instance boundaries inside the chunk).  At the end, a warp whose lanes
// all hold the same instance reduces with shuffles and applies one atomic per
// dimension, and the block merges its warps' results before the atomics.
// The small blocks' mnmx must hold INT_MAX / INT_MIN first.
template <int D>
__device__ __forceinline__ void bounds_flush(const Inst& I, const int* mn, const int* mx) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
        atomicMin(I.small + kSmMnmx + j, mn[j]);
        atomicMax(I.small + kSmMnmx + kMaxD + j, mx[j]);
    }
}

// Over the instances of dimension D.
constexpr int kBoundsWarps = 8;  // 256 threads

template <int D>
__global__ void __launch_bounds__(kBoundsWarps * 32) bounds_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5);
    const long long per = (((total + nwarps - 1) / nwarps) + 31) & ~31ll;
    const long long beg = wid * per, end = min(total, beg + per);
    int mn[D], mx[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        mn[j] = INT_MAX;
        mx[j] = INT_MIN;
    }
    FlatCursor cur;
    int kk = -1;  // instance index of the accumulated values
    const int* X = nullptr;
    long long i = beg + lane_id();
    while (i < end) {
        if (cur.seek(f, i)) {
            if (kk >= 0) bounds_flush<D>(ins[kk], mn, mx);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                mn[j] = INT_MAX;
                mx[j] = INT_MIN;
            }
            kk = f.idx[cur.k];
            X = ins[kk].X;
        }
        // the lane's points of this instance, four rows in flight at a time
        const long long stop = min(end, cur.hi);
        for (; i < stop; i += 4 * 32) {
            int v[4][D];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long q = i + u * 32;
                const int* row = X + (q - cur.lo) * D;
#pragma unroll
                for (int j = 0; j < D; ++j) v[u][j] = q < stop ? __ldg(row + j) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * 32 < stop) {
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        mn[j] = min(mn[j], v[u][j]);
                        mx[j] = max(mx[j], v[u][j]);
                    }
                }
        }
        if (i >= stop && stop < end) i = stop + ((i - stop) & 31);
    }
    // warp, then block: the atomics of a block's warps that hold one instance
    // are merged, so that few atomics meet on the same addresses
    __shared__ int s_k[kBoundsWarps], s_mn[kBoundsWarps][D], s_mx[kBoundsWarps][D];
    const int w = threadIdx.x >> 5;
    const unsigned uniform = __match_any_sync(kFull, kk);
    if (uniform == kFull) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            mn[j] = __reduce_min_sync(kFull, mn[j]);
            mx[j] = __reduce_max_sync(kFull, mx[j]);
        }
        if (lane_id() == 0) {
            s_k[w] = kk;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                s_mn[w][j] = mn[j];
                s_mx[w][j] = mx[j];
            }
        }
    } else {
        if (kk >= 0) bounds_flush<D>(ins[kk], mn, mx);
        if (lane_id() == 0) s_k[w] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int k0 = -1;
        for (int v = 0; v < kBoundsWarps; ++v) {
            const int k = s_k[v];
            if (k < 0) continue;
            if (k != k0) {
                if (k0 >= 0) bounds_flush<D>(ins[k0], mn, mx);
                k0 = k;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    mn[j] = s_mn[v][j];
                    mx[j] = s_mx[v][j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    mn[j] = min(mn[j], s_mn[v][j]);
                    mx[j] = max(mx[j], s_mx[v][j]);
                }
            }
        }
        if (k0 >= 0) bounds_flush<D>(ins[k0], mn, mx);
    }
}

cudaError_t launch_bounds(const Inst* ins, Flat pts, long long total, int d, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    switch (d) {
#define GD_BK(DD) \
    case DD: bounds_kernel<DD><<<(int)blocks, 256, 0, st>>>(ins, pts, total); break;
        GD_BK(1) GD_BK(2) GD_BK(3) GD_BK(4) GD_BK(5) GD_BK(6) GD_BK(7) GD_BK(8)
#undef GD_BK
        default: return cudaErrorInvalidValue;
    }
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------ compaction
// Alg. 1's scan over the sorted points: a grid starts where the key changes.
// Flat space: compaction tiles of kCompactTile points of each instance.

constexpr int kCompactBlock = 256;
constexpr int kCompactItems = kCompactTile / kCompactBlock;

__device__ __forceinline__ bool key_eq(unsigned long long a, unsigned long long b) { return a == b; }
__device__ __forceinline__ bool key_eq(const Key2& a, const Key2& b) { return a.lo == b.lo && a.hi == b.hi; }

__device__ __forceinline__ unsigned key_field(unsigned long long k, int sh, int bits) {
    return bits == 0 ? 0u : (unsigned)((k >> sh) & ((1ull << bits) - 1ull));
}
__device__ __forceinline__ unsigned key_field(const Key2& k, int sh, int bits) {
    if (bits == 0) return 0u;
    unsigned long long v;
    if (sh >= 64) {
        v = k.hi >> (sh - 64);
    } else {
        v = k.lo >> sh;
        if (sh > 0) v |= k.hi << (64 - sh);
    }
    return (unsigned)(v & ((1ull << bits) - 1ull));
}

// The sorted keys/values of an instance: the sort leaves them in A after an
// even number of passes, in B after an odd number.
template <typename K>
__device__ __forceinline__ const K* sorted_keys(const Inst& I) {
    return (const K*)((I.passes & 1) ? I.keyB : I.keyA);
}
__device__ __forceinline__ int* sorted_vals(const Inst& I) { return (I.passes & 1) ? I.valB : I.valA; }

// The grid key of sorted position q (packed keys carry the point index in
// their low pack_bits bits).
template <typename K, bool PACKED> __device__ __forceinline__ K grid_key(const K* keys, long long q, int pb) {
    if constexpr (PACKED)
        return keys[q] >> pb;
    else
        return keys[q];
}

// Both kernels take a tile's positions warp by warp: warp w owns
// kCompactItems * 32 consecutive positions and item i of lane l is position
// wbase + i * 32 + l, so every load and store of a warp instruction is
// contiguous; a grid start is a lane whose key differs from the position
// before it, and the grid ids follow from ballots of those flags.
constexpr int kCompactWarps = kCompactBlock / 32;

template <typename K, bool PACKED>
__device__ __forceinline__ bool grid_starts(const K* keys, long long q, int n, int pb) {
    return q < n && (q == 0 || !key_eq(grid_key<K, PACKED>(keys, q, pb), grid_key<K, PACKED>(keys, q - 1, pb)));
}

template <typename K, bool PACKED>
__global__ void __launch_bounds__(kCompactBlock) compact_count_kernel(const Inst* __restrict__ ins, Flat f) {
    __shared__ int s_cnt[kCompactWarps];
    const int k = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[k]];
    const long long tile = blockIdx.x - f.off[k];
    const int n = I.p.n;
    const K* keys = sorted_keys<K>(I);
    const int pb = I.p.pack_bits;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const long long wbase = tile * kCompactTile + (long long)warp * 32 * kCompactItems;
    int c = 0;
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) c += grid_starts<K, PACKED>(keys, wbase + i * 32 + lane, n, pb);
    c = __reduce_add_sync(kFull, (unsigned)c);
    if (lane == 0) s_cnt[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
#pragma unroll
        for (int w = 0; w < kCompactWarps; ++w) total += s_cnt[w];
        I.bcnt[tile] = total;
    }
}

// Writes cell_start, identifiers (decoded from the key), pt_cell and the
// grid-order coordinates Xs (gathered through the sorted permutation, or
// rebuilt from the in-cell offsets; packed keys also write the permutation
// out).
template <typename K, bool PACKED>
__global__ void __launch_bounds__(kCompactBlock) compact_write_kernel(const Inst* __restrict__ ins, Flat f) {
    __shared__ int s_cnt[kCompactWarps];
    const int k = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[k]];
    const long long tile = blockIdx.x - f.off[k];
    const int n = I.p.n, d = I.p.d, dp = I.p.dp;
    const K* keys = sorted_keys<K>(I);
    int* vals = sorted_vals(I);
    const int pb = I.p.pack_bits;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const long long wbase = tile * kCompactTile + (long long)warp * 32 * kCompactItems;
    // The items' sources (random reads) are all requested before the block
    // exchange, so that their latency overlaps it.  With in-cell offset words
    // the random read is that word (4 bytes of an array a quarter or less the
    // size of the rows, which the cache keeps) and the row is rebuilt from
    // the identifiers: x_j = mn_j + id_j * s + offset_j.
    const bool rebuild = PACKED && I.p.xoff_w >= 0;
    const int* xoff = in_cell_offsets(I);
    unsigned starts[kCompactItems];
    int src[kCompactItems];
    int4 row4[kCompactItems];
    unsigned ow[kCompactItems];
    int c = 0;
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) {
        const long long q = wbase + i * 32 + lane;
        starts[i] = __ballot_sync(kFull, grid_starts<K, PACKED>(keys, q, n, pb));
        c += __popc(starts[i]);
        src[i] = 0;
        ow[i] = 0;
        row4[i] = make_int4(0, 0, 0, 0);
        if (q < n) {
            if constexpr (PACKED)
                src[i] = (int)(keys[q] & ((1ull << pb) - 1ull));
            else
                src[i] = vals[q];
            if (rebuild) {
                if (I.p.xoff_w > 0) ow[i] = (unsigned)__ldg(xoff + src[i]);
            } else if (dp == 4) {
                const int* row = I.X + (long long)src[i] * d;
                row4[i].x = __ldg(row);
                if (d > 1) row4[i].y = __ldg(row + 1);
                if (d > 2) row4[i].z = __ldg(row + 2);
                if (d > 3) row4[i].w = __ldg(row + 3);
            }
        }
    }
    if (lane == 0) s_cnt[warp] = c;
    __syncthreads();
    // id of the grid holding the position before the warp's first
    int cid = I.bcnt[tile] - 1;
#pragma unroll
    for (int w = 0; w < kCompactWarps; ++w)
        if (w < warp) cid += s_cnt[w];
    const unsigned le = lanemask_lt() | (1u << lane);
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) {
        const long long q = wbase + i * 32 + lane;
        const int my = cid + __popc(starts[i] & le);
        cid += __popc(starts[i]);
        if (q >= n) continue;
        if ((starts[i] >> lane) & 1u) {
            I.cell_start[my] = (int)q;
            const K key = grid_key<K, PACKED>(keys, q, pb);
            for (int j = 0; j < d; ++j)
                I.cell_coord[(long long)my * d + j] = (int)key_field(key, I.p.shift[j], I.p.bits[j]);
        }
        // streaming stores (evict first): the outputs are written once here,
        // and the offset words still to be read stay in the cache
        __stcs(I.pt_cell + q, my);
        if constexpr (PACKED) __stcs(vals + q, src[i]);
        const int* row = I.X + (long long)src[i] * d;
        int* out = I.Xs + q * dp;
        if (rebuild) {
            // unsigned arithmetic: x - mn_j < 2^32 and the sum wraps back to x
            const K key = grid_key<K, PACKED>(keys, q, pb);
            const int w = I.p.xoff_w;
            const unsigned om = w > 0 ? (1u << w) - 1u : 0u;
            int v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = 0;
                if (j < d)
                    v[j] = (int)((unsigned)I.p.mn[j] + key_field(key, I.p.shift[j], I.p.bits[j]) * (unsigned)I.p.s +
                                 (w > 0 ? (ow[i] >> (j * w)) & om : 0u));
            }
            if (dp == 8) {
                __stcs(reinterpret_cast<int4*>(out), make_int4(v[0], v[1], v[2], v[3]));
                __stcs(reinterpret_cast<int4*>(out) + 1, make_int4(v[4], v[5], v[6], v[7]));
            } else if (dp == 4) {
                __stcs(reinterpret_cast<int4*>(out), make_int4(v[0], v[1], v[2], v[3]));
            } else if (dp == 2) {
                __stcs(reinterpret_cast<int2*>(out), make_int2(v[0], v[1]));
            } else {
                __stcs(out, v[0]);
            }
        } else if (dp == 4) {
            *reinterpret_cast<int4*>(out) = row4[i];
        } else {
            for (int j = 0; j < dp; ++j) out[j] = j < d ? __ldg(row + j) : 0;
        }
        if (q == n - 1) {
            I.cell_start[my + 1] = n;
            I.small[kSmCells] = my + 1;
        }
    }
}

cudaError_t launch_compact_count(const Inst* ins, Flat tiles, long long total, int key_class, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (key_class == 0)
        compact_count_kernel<unsigned long long, true><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    else if (key_class == 1)
        compact_count_kernel<unsigned long long, false><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    else
        compact_count_kernel<Key2, false><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_compact_write(const Inst* ins, Flat tiles, long long total, int key_class, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (key_class == 0)
        compact_write_kernel<unsigned long long, true><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    else if (key_class == 1)
        compact_write_kernel<unsigned long long, false><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    else
        compact_write_kernel<Key2, false><<<(unsigned)total, kCompactBlock, 0, st>>>(ins, tiles);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Largest grid of each instance (bounds the merge's bitmaps).  The flat
// space is the instances' points, an upper bound of their grids: a warp-sized
// grid-stride loop reads the sizes of grids c < C (C read on the device) and
// steps over the rest of an instance, reduces the sizes in the warp and
// applies one atomic.  small[kSmMaxCell] must be 0 first.
__global__ void cell_max_kernel(const Inst* __restrict__ ins, Flat f, long long total) {
    total = flat_total(f);
    const long long stride = (long long)gridDim.x * blockDim.x;
    FlatCursor cur;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total;) {
        const long long i = base + lane_id();
        int kk = -1, size = 0;
        long long past = -1;  // end of this lane's instance once its grids are behind
        if (i < total) {
            cur.seek(f, i);
            kk = f.idx[cur.k];
            const Inst& I = ins[kk];
            const long long c = i - cur.lo;
            if (c < I.small[kSmCells])
                size = I.cell_start[c + 1] - I.cell_start[c];
            else
                past = cur.hi;
        }
        // the next position of this warp's stride, past the rest of lane 0's
        // instance when lane 0 is already beyond that instance's grids
        long long next = base + stride;
        const long long hi0 = __shfl_sync(kFull, past, 0);
        if (hi0 > next) next += (hi0 - next + stride - 1) / stride * stride;
        const int k0 = __shfl_sync(kFull, kk, 0);
        if (__all_sync(kFull, kk == k0)) {
            const int m = __reduce_max_sync(kFull, (unsigned)size);
            if (lane_id() == 0 && k0 >= 0 && m > 0) atomicMax(ins[k0].small + kSmMaxCell, m);
        } else if (kk >= 0 && size > 0) {
            atomicMax(ins[kk].small + kSmMaxCell, size);
        }
        base = next;
    }
}

cudaError_t launch_cell_max(const Inst* ins, Flat pts, long long total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > kPersistBlocks) blocks = kPersistBlocks;
    cell_max_kernel<<<(int)blocks, 256, 0, st>>>(ins, pts, total);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
