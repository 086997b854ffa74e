// Grid construction: bounds, identifiers (Eq. 1), LSD radix sort and the
// non-empty-grid compaction of Alg. 1, plus a device-wide exclusive scan.
#include <climits>

#include "gd_internal.cuh"

namespace gd {

// ------------------------------------------------------------------ scan
// Three phases: per-tile sums, one-block scan of the sums, per-tile scan.

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

size_t scan_tmp_ints(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 2; }

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int* __restrict__ in, long long n,
                                                                 int* __restrict__ bsum) {
    __shared__ int sm[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int total;
    block_exclusive_scan(s, sm, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_top_kernel(int* __restrict__ bsum, int nb) {
    __shared__ int sm[33];
    int carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int k = base + threadIdx.x;
        int v = k < nb ? bsum[k] : 0;
        int total;
        int ex = block_exclusive_scan(v, sm, &total);
        if (k < nb) bsum[k] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(const int* in, int* out, long long n,
                                                               const int* __restrict__ bsum, int nb) {
    __shared__ int sm[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int total;
    int run = bsum[blockIdx.x] + block_exclusive_scan(s, sm, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

cudaError_t scan_exclusive(const int* in, int* out, long long n, int* tmp, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
    const int nb = (int)((n + kScanTile - 1) / kScanTile);
    scan_reduce_kernel<<<nb, kScanBlock, 0, st>>>(in, n, tmp);
    GD_COUNT_LAUNCH();
    scan_top_kernel<<<1, 1024, 0, st>>>(tmp, nb);
    GD_COUNT_LAUNCH();
    scan_down_kernel<<<nb, kScanBlock, 0, st>>>(in, out, n, tmp, nb);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bounds

__global__ void init_bounds_kernel(int* mnmx) {
    if (threadIdx.x < kMaxD) {
        mnmx[threadIdx.x] = INT_MAX;
        mnmx[kMaxD + threadIdx.x] = INT_MIN;
    }
}

cudaError_t launch_init_bounds(int* mnmx, cudaStream_t st) {
    init_bounds_kernel<<<1, 32, 0, st>>>(mnmx);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Per-dimension min and max (mn_j of Eq. 1), reduced per warp then per block,
// then one atomic per block and dimension.
__global__ void __launch_bounds__(256) bounds_kernel(const int* __restrict__ X, int n, int d, int* mnmx) {
    int mn[kMaxD], mx[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        mn[j] = INT_MAX;
        mx[j] = INT_MIN;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int* row = X + i * d;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j)
            if (j < d) {
                int v = __ldg(row + j);
                mn[j] = min(mn[j], v);
                mx[j] = max(mx[j], v);
            }
    }
    __shared__ int smn[8][kMaxD], smx[8][kMaxD];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[j] = min(mn[j], __shfl_xor_sync(kFull, mn[j], o));
            mx[j] = max(mx[j], __shfl_xor_sync(kFull, mx[j], o));
        }
        if (lane == 0) {
            smn[warp][j] = mn[j];
            smx[warp][j] = mx[j];
        }
    }
    __syncthreads();
    if (threadIdx.x < d) {
        int a = INT_MAX, b = INT_MIN;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = min(a, smn[w][threadIdx.x]);
            b = max(b, smx[w][threadIdx.x]);
        }
        atomicMin(mnmx + threadIdx.x, a);
        atomicMax(mnmx + kMaxD + threadIdx.x, b);
    }
}

cudaError_t launch_bounds(const int* X, int n, int d, int* mnmx, cudaStream_t st) {
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    bounds_kernel<<<blocks, 256, 0, st>>>(X, n, d, mnmx);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------- quantise

__device__ __forceinline__ unsigned identifier(int x, int mn, long long s) {
    // (x - mn) fits in 32 unsigned bits; an identifier is at most 2^31 - 1
    // because d * range^2 < 2^62 is checked before this runs.
    unsigned long long diff = (unsigned)(x - mn);
    return (unsigned)(diff / (unsigned long long)s);
}

__global__ void __launch_bounds__(256) quantise1_kernel(const int* __restrict__ X, Params p,
                                                        unsigned long long* __restrict__ keys,
                                                        int* __restrict__ vals) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const int* row = X + i * p.d;
        unsigned long long k = 0;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j)
            if (j < p.d) k |= (unsigned long long)identifier(__ldg(row + j), p.mn[j], p.s) << p.shift[j];
        keys[i] = k;
        vals[i] = (int)i;
    }
}

__device__ __forceinline__ void or_shifted(Key2& k, unsigned long long v, int sh) {
    if (sh >= 64) {
        k.hi |= v << (sh - 64);
    } else {
        k.lo |= v << sh;
        if (sh > 0) k.hi |= v >> (64 - sh);
    }
}

__global__ void __launch_bounds__(256) quantise2_kernel(const int* __restrict__ X, Params p, Key2* __restrict__ keys,
                                                        int* __restrict__ vals) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const int* row = X + i * p.d;
        Key2 k{0ull, 0ull};
#pragma unroll
        for (int j = 0; j < kMaxD; ++j)
            if (j < p.d) or_shifted(k, identifier(__ldg(row + j), p.mn[j], p.s), p.shift[j]);
        keys[i] = k;
        vals[i] = (int)i;
    }
}

cudaError_t launch_quantise(const int* X, const Params& p, void* keys, int* vals, cudaStream_t st) {
    int blocks = (p.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (p.key_words == 1)
        quantise1_kernel<<<blocks, 256, 0, st>>>(X, p, (unsigned long long*)keys, vals);
    else
        quantise2_kernel<<<blocks, 256, 0, st>>>(X, p, (Key2*)keys, vals);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
// Stable LSD sort over 8-bit digits.  Per pass: a per-tile digit histogram
// (digit-major table), an exclusive scan of the table, and a scatter that
// ranks each tile stably in shared memory (warp match + per-warp counters)
// and then writes digit runs out contiguously.

constexpr int kRadixBits = 8;
constexpr int kBuckets = 1 << kRadixBits;
constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;

template <typename K> struct KeyTraits;
template <> struct KeyTraits<unsigned long long> {
    static constexpr int kItems = 16;
    __device__ static __forceinline__ unsigned digit(unsigned long long k, int sh) {
        return (unsigned)(k >> sh) & (kBuckets - 1);
    }
};
template <> struct KeyTraits<Key2> {
    static constexpr int kItems = 8;
    __device__ static __forceinline__ unsigned digit(const Key2& k, int sh) {
        unsigned long long v;
        if (sh >= 64) {
            v = k.hi >> (sh - 64);
        } else {
            v = k.lo >> sh;
            if (sh > 64 - kRadixBits) v |= k.hi << (64 - sh);
        }
        return (unsigned)v & (kBuckets - 1);
    }
};

template <typename K> constexpr int sort_tile() { return kSortBlock * KeyTraits<K>::kItems; }

size_t radix_tmp_ints(int n, int key_words) {
    const int tile = key_words == 1 ? sort_tile<unsigned long long>() : sort_tile<Key2>();
    const long long tiles = (n + tile - 1) / tile;
    const long long table = tiles * kBuckets;
    return (size_t)(table + 1) + scan_tmp_ints(table);
}

template <typename K>
__global__ void __launch_bounds__(kSortBlock) radix_hist_kernel(const K* __restrict__ keys, int n, int shift,
                                                                int* __restrict__ table, int tiles) {
    constexpr int kItems = KeyTraits<K>::kItems;
    __shared__ int h[kSortWarps][kBuckets];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kBuckets; i += kSortBlock) (&h[0][0])[i] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * sort_tile<K>();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        long long k = base + i * kSortBlock + threadIdx.x;
        if (k < n) atomicAdd(&h[warp][KeyTraits<K>::digit(keys[k], shift)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += kSortBlock) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += h[w][b];
        table[(long long)b * tiles + blockIdx.x] = s;
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortBlock) radix_scatter_kernel(const K* __restrict__ keys_in,
                                                                   const int* __restrict__ vals_in,
                                                                   K* __restrict__ keys_out, int* __restrict__ vals_out,
                                                                   int n, int shift, const int* __restrict__ table,
                                                                   int tiles) {
    constexpr int kItems = KeyTraits<K>::kItems;
    constexpr int kTile = sort_tile<K>();
    constexpr int kExchBytes = kTile * (sizeof(K) > sizeof(int) ? sizeof(K) : sizeof(int));
    __shared__ __align__(16) unsigned char exch[kExchBytes];
    __shared__ int wcount[kSortWarps][kBuckets];
    __shared__ int dstart[kBuckets];  // first tile-local position of each digit
    __shared__ int goff[kBuckets];    // global offset of this tile's run of each digit
    __shared__ int sm[33];

    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kTile;
    const int count = (int)min((long long)kTile, (long long)n - base);

    for (int i = threadIdx.x; i < kSortWarps * kBuckets; i += kSortBlock) (&wcount[0][0])[i] = 0;
    for (int b = threadIdx.x; b < kBuckets; b += kSortBlock) goff[b] = table[(long long)b * tiles + blockIdx.x];
    __syncthreads();

    // Warp w owns the consecutive items [w*32*kItems, (w+1)*32*kItems) of the
    // tile; item i of lane l is at w*32*kItems + i*32 + l (index order).
    K key[kItems];
    int rank[kItems];
    unsigned dig[kItems];
    const int wbase = warp * 32 * kItems;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        const bool valid = t < count;
        if (valid) key[i] = keys_in[base + t];
        dig[i] = valid ? KeyTraits<K>::digit(key[i], shift) : (unsigned)(kBuckets + lane);
        const unsigned peers = __match_any_sync(kFull, dig[i]);
        int before = 0;
        if (valid) before = wcount[warp][dig[i]];
        __syncwarp();
        if (valid && lane == (int)(__ffs(peers) - 1)) wcount[warp][dig[i]] = before + __popc(peers);
        __syncwarp();
        rank[i] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();

    // Per digit: exclusive prefix over warps, then over digits.
    int tot = 0;
    if (threadIdx.x < kBuckets) {
        const int b = threadIdx.x;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            int c = wcount[w][b];
            wcount[w][b] = tot;
            tot += c;
        }
    }
    int all;
    int ex = block_exclusive_scan(threadIdx.x < kBuckets ? tot : 0, sm, &all);
    if (threadIdx.x < kBuckets) dstart[threadIdx.x] = ex;
    __syncthreads();

    // Keys through shared memory into tile-local digit order, then out.
    K* skeys = reinterpret_cast<K*>(exch);
    int pos[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        if (t < count) {
            pos[i] = dstart[dig[i]] + wcount[warp][dig[i]] + rank[i];
            skeys[pos[i]] = key[i];
        }
    }
    __syncthreads();
    int dst[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = i * kSortBlock + threadIdx.x;
        if (t < count) {
            K k = skeys[t];
            unsigned b = KeyTraits<K>::digit(k, shift);
            dst[i] = goff[b] + (t - dstart[b]);
            keys_out[dst[i]] = k;
        }
    }
    __syncthreads();
    int* svals = reinterpret_cast<int*>(exch);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        if (t < count) svals[pos[i]] = vals_in[base + t];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = i * kSortBlock + threadIdx.x;
        if (t < count) vals_out[dst[i]] = svals[t];
    }
}

template <typename K>
static cudaError_t radix_sort_t(K* ka, int* va, K* kb, int* vb, int n, int key_bits, int* tmp, cudaStream_t st,
                                int* result_in_b) {
    constexpr int kTile = sort_tile<K>();
    const int tiles = (n + kTile - 1) / kTile;
    const long long table_n = (long long)tiles * kBuckets;
    int* table = tmp;
    int* scan_tmp = tmp + table_n + 1;
    K* src_k = ka;
    int* src_v = va;
    K* dst_k = kb;
    int* dst_v = vb;
    int flips = 0;
    for (int shift = 0; shift < key_bits; shift += kRadixBits) {
        radix_hist_kernel<K><<<tiles, kSortBlock, 0, st>>>(src_k, n, shift, table, tiles);
        GD_COUNT_LAUNCH();
        cudaError_t e = scan_exclusive(table, table, table_n, scan_tmp, st);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<K><<<tiles, kSortBlock, 0, st>>>(src_k, src_v, dst_k, dst_v, n, shift, table, tiles);
        GD_COUNT_LAUNCH();
        K* tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        int* tv = src_v;
        src_v = dst_v;
        dst_v = tv;
        flips ^= 1;
    }
    *result_in_b = flips;
    return cudaGetLastError();
}

cudaError_t radix_sort(void* keys_a, int* vals_a, void* keys_b, int* vals_b, int n, int key_words, int key_bits,
                       int* tmp, cudaStream_t st, int* result_in_b) {
    *result_in_b = 0;
    if (n <= 1 || key_bits <= 0) return cudaSuccess;
    if (key_words == 1)
        return radix_sort_t((unsigned long long*)keys_a, vals_a, (unsigned long long*)keys_b, vals_b, n, key_bits,
                            tmp, st, result_in_b);
    return radix_sort_t((Key2*)keys_a, vals_a, (Key2*)keys_b, vals_b, n, key_bits, tmp, st, result_in_b);
}

// ------------------------------------------------------------ compaction
// Alg. 1's scan over the sorted points: a grid starts where the key changes.

constexpr int kCompactBlock = 256;
constexpr int kCompactItems = 4;
constexpr int kCompactTile = kCompactBlock * kCompactItems;

size_t compact_tmp_ints(int n) { return (size_t)((n + kCompactTile - 1) / kCompactTile) + 1 + scan_tmp_ints(n); }

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

template <typename K>
__global__ void __launch_bounds__(kCompactBlock) cell_count_kernel(const K* __restrict__ keys, int n,
                                                                   int* __restrict__ bcnt) {
    __shared__ int sm[33];
    const long long base = (long long)blockIdx.x * kCompactTile + (long long)threadIdx.x * kCompactItems;
    int c = 0;
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) {
        long long k = base + i;
        if (k < n && (k == 0 || !key_eq(keys[k], keys[k - 1]))) c++;
    }
    int total;
    block_exclusive_scan(c, sm, &total);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = total;
}

template <typename K>
__global__ void __launch_bounds__(kCompactBlock) cell_write_kernel(Params p, const int* __restrict__ X,
                                                                   const K* __restrict__ keys,
                                                                   const int* __restrict__ vals,
                                                                   const int* __restrict__ boff,
                                                                   int* __restrict__ cell_start,
                                                                   int* __restrict__ cell_coord,
                                                                   int* __restrict__ pt_cell, int* __restrict__ Xs,
                                                                   int* __restrict__ num_cells) {
    __shared__ int sm[33];
    const int n = p.n, d = p.d, dp = p.dp;
    const long long base = (long long)blockIdx.x * kCompactTile + (long long)threadIdx.x * kCompactItems;
    bool f[kCompactItems];
    int c = 0;
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) {
        long long k = base + i;
        f[i] = k < n && (k == 0 || !key_eq(keys[k], keys[k - 1]));
        c += f[i];
    }
    int total;
    int cid = boff[blockIdx.x] + block_exclusive_scan(c, sm, &total) - 1;
#pragma unroll
    for (int i = 0; i < kCompactItems; ++i) {
        const long long k = base + i;
        if (k >= n) break;
        if (f[i]) {
            cid++;
            cell_start[cid] = (int)k;
            const K key = keys[k];
            for (int j = 0; j < d; ++j) cell_coord[(long long)cid * d + j] = (int)key_field(key, p.shift[j], p.bits[j]);
        }
        pt_cell[k] = cid;
        const int src = vals[k];
        const int* row = X + (long long)src * d;
        int* out = Xs + k * dp;
        for (int j = 0; j < dp; ++j) out[j] = j < d ? __ldg(row + j) : 0;
        if (k == n - 1) {
            cell_start[cid + 1] = n;
            *num_cells = cid + 1;
        }
    }
}

cudaError_t launch_compact(const Params& p, const int* X, const void* keys, const int* vals, int* tmp,
                           int* cell_start, int* cell_coord, int* pt_cell, int* Xs, int* num_cells, cudaStream_t st) {
    const int nb = (p.n + kCompactTile - 1) / kCompactTile;
    int* bcnt = tmp;
    int* scan_tmp = tmp + nb + 1;
    if (p.key_words == 1)
        cell_count_kernel<<<nb, kCompactBlock, 0, st>>>((const unsigned long long*)keys, p.n, bcnt);
    else
        cell_count_kernel<<<nb, kCompactBlock, 0, st>>>((const Key2*)keys, p.n, bcnt);
    GD_COUNT_LAUNCH();
    cudaError_t e = scan_exclusive(bcnt, bcnt, nb, scan_tmp, st);
    if (e != cudaSuccess) return e;
    if (p.key_words == 1)
        cell_write_kernel<<<nb, kCompactBlock, 0, st>>>(p, X, (const unsigned long long*)keys, vals, bcnt, cell_start,
                                                        cell_coord, pt_cell, Xs, num_cells);
    else
        cell_write_kernel<<<nb, kCompactBlock, 0, st>>>(p, X, (const Key2*)keys, vals, bcnt, cell_start, cell_coord,
                                                        pt_cell, Xs, num_cells);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
