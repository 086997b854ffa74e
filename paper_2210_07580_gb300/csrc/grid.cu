// Grid construction: bounds (mn_j of Eq. 1) and the non-empty-grid
// compaction of Alg. 1, plus a device-wide exclusive scan.  The identifiers
// and the sort are in sort.cu.
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
