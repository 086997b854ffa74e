// Grid identifiers (Eq. 1) and the stable LSD radix sort of Alg. 1.
//
// The paper sorts by counting sort one dimension at a time; here the
// identifiers are packed into one 64- or 128-bit key (dimension 1 most
// significant, so key order is the lexicographic order of Alg. 1) and sorted
// by digits of up to 9 bits:
//   1. quantise_hist: computes every key and, in the same pass, the global
//      histogram of every digit position;
//   2. digit_scan: exclusive scan of each digit position's histogram;
//   3. one onesweep pass per digit position: each block takes the next tile
//      (dynamic tile ids), ranks its keys stably in shared memory, publishes
//      its per-digit counts and finds the counts of all earlier tiles by a
//      decoupled look-back, then writes each digit run out contiguously.
// A pass reads and writes every key and value once.  Look-back waits are
// bounded: a block only ever waits for tiles handed out before its own, and
// gives up with kDevTimeout after a fixed number of polls.
#include "gd_internal.cuh"

namespace gd {

constexpr int kMaxDigitBits = 9;
constexpr int kMaxBuckets = 1 << kMaxDigitBits;
constexpr int kOsBlock = 256;
constexpr int kOsWarps = kOsBlock / 32;
constexpr unsigned kFlagAgg = 1u, kFlagInc = 2u;
constexpr int kMaxPolls = 1 << 22;

template <typename K> struct SortKey;
template <> struct SortKey<unsigned long long> {
    static constexpr int kItems = 16;
    __device__ static __forceinline__ unsigned digit(unsigned long long k, int sh, unsigned mask) {
        return (unsigned)(k >> sh) & mask;
    }
};
template <> struct SortKey<Key2> {
    static constexpr int kItems = 8;
    __device__ static __forceinline__ unsigned digit(const Key2& k, int sh, unsigned mask) {
        unsigned long long v;
        if (sh >= 64) {
            v = k.hi >> (sh - 64);
        } else {
            v = k.lo >> sh;
            if (sh > 0) v |= k.hi << (64 - sh);
        }
        return (unsigned)v & mask;
    }
};

template <typename K> __host__ __device__ constexpr int os_tile() { return kOsBlock * SortKey<K>::kItems; }

SortPlan sort_plan(int n, int key_words, int key_bits) {
    SortPlan sp;
    sp.passes = key_bits <= 0 ? 0 : (key_bits + kMaxDigitBits - 1) / kMaxDigitBits;
    sp.bits = sp.passes == 0 ? 0 : (key_bits + sp.passes - 1) / sp.passes;
    sp.buckets = 1 << sp.bits;
    sp.tile = key_words == 1 ? os_tile<unsigned long long>() : os_tile<Key2>();
    sp.tiles = (n + sp.tile - 1) / sp.tile;
    return sp;
}

// Layout of the sort's workspace (ints): hist [P][R], digit_start [P][R],
// tile counters [P], status [P][tiles][R] (64-bit words).
size_t radix_tmp_ints(int n, int key_words, int key_bits) {
    const SortPlan sp = sort_plan(n, key_words, key_bits);
    const size_t pr = (size_t)sp.passes * sp.buckets;
    return 2 * pr + (size_t)sp.passes + 8 + 2 * (size_t)sp.passes * sp.tiles * sp.buckets + 64;
}

struct SortTmp {
    int* hist;
    int* dstart;
    int* counters;
    unsigned long long* status;
};

static SortTmp sort_tmp(int* tmp, const SortPlan& sp) {
    SortTmp t;
    const size_t pr = (size_t)sp.passes * sp.buckets;
    t.hist = tmp;
    t.dstart = tmp + pr;
    t.counters = tmp + 2 * pr;
    size_t off = 2 * pr + sp.passes + 8;
    off = (off + 1) & ~(size_t)1;  // 8-byte alignment (tmp is 256-byte aligned)
    t.status = reinterpret_cast<unsigned long long*>(tmp + off);
    return t;
}

// ------------------------------------------------------------- quantise

__device__ __forceinline__ unsigned identifier(int x, int mn, long long s) {
    // (x - mn) fits in 32 unsigned bits; an identifier is at most 2^31 - 1
    // because d * range^2 < 2^62 is checked before this runs.
    const unsigned long long diff = (unsigned)(x - mn);
    return (unsigned)(diff / (unsigned long long)s);
}

__device__ __forceinline__ void pack_key(unsigned long long& k, unsigned v, int sh) {
    k |= (unsigned long long)v << sh;
}
__device__ __forceinline__ void pack_key(Key2& k, unsigned v, int sh) {
    const unsigned long long w = v;
    if (sh >= 64) {
        k.hi |= w << (sh - 64);
    } else {
        k.lo |= w << sh;
        if (sh > 0) k.hi |= w >> (64 - sh);
    }
}
__device__ __forceinline__ void zero_key(unsigned long long& k) { k = 0; }
__device__ __forceinline__ void zero_key(Key2& k) { k.lo = k.hi = 0; }

// Keys, values (input index) and the histogram of every digit position.
// Runs of equal digits inside a warp are counted once (warp match), which
// keeps shared-memory atomics cheap on clustered data.
template <typename K>
__global__ void __launch_bounds__(256) quantise_hist_kernel(const int* __restrict__ X, Params p, K* __restrict__ keys,
                                                            int* __restrict__ vals, int* __restrict__ hist,
                                                            int passes, int bits) {
    extern __shared__ int sh_hist[];  // [passes][1 << bits]
    const int R = 1 << bits;
    const unsigned mask = (unsigned)R - 1u;
    for (int i = threadIdx.x; i < passes * R; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    const int lane = lane_id();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = ((long long)p.n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < p.n;
        K k;
        zero_key(k);
        if (valid) {
            const int* row = X + i * p.d;
#pragma unroll
            for (int j = 0; j < kMaxD; ++j)
                if (j < p.d) pack_key(k, identifier(__ldg(row + j), p.mn[j], p.s), p.shift[j]);
            keys[i] = k;
            vals[i] = (int)i;
        }
        for (int ps = 0; ps < passes; ++ps) {
            const unsigned dg = valid ? SortKey<K>::digit(k, ps * bits, mask) : (unsigned)R + lane;
            const unsigned peers = __match_any_sync(kFull, dg);
            if (valid && lane == (int)(__ffs(peers) - 1)) atomicAdd(&sh_hist[ps * R + dg], __popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * R; i += blockDim.x)
        if (sh_hist[i]) atomicAdd(hist + i, sh_hist[i]);
}

__global__ void digit_scan_kernel(const int* __restrict__ hist, int* __restrict__ dstart, int R) {
    __shared__ int sm[33];
    const int ps = blockIdx.x;
    int carry = 0;
    for (int base = 0; base < R; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const int v = b < R ? hist[ps * R + b] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sm, &total);
        if (b < R) dstart[ps * R + b] = carry + ex;
        carry += total;
    }
}

// ------------------------------------------------------------- onesweep

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename K>
__global__ void __launch_bounds__(kOsBlock, 3) onesweep_kernel(const K* __restrict__ keys_in,
                                                            const int* __restrict__ vals_in, K* __restrict__ keys_out,
                                                            int* __restrict__ vals_out, int n, int shift, int bits,
                                                            const int* __restrict__ dstart_g,
                                                            unsigned long long* status, int* tile_counter,
                                                            unsigned* err) {
    constexpr int kItems = SortKey<K>::kItems;
    constexpr int kTile = os_tile<K>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << bits;
    const unsigned mask = (unsigned)R - 1u;
    // layout: exchange keys [kTile] K, exchange vals [kTile] int,
    //         wcount [kOsWarps][R], dstart [R], goff [R]
    K* skeys = reinterpret_cast<K*>(smem);
    int* svals = reinterpret_cast<int*>(smem + sizeof(K) * kTile);
    int* wcount = svals + kTile;
    int* ldstart = wcount + kOsWarps * R;
    int* goff = ldstart + R;
    __shared__ int sm[33];
    __shared__ int s_tile;

    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
    for (int i = threadIdx.x; i < kOsWarps * R; i += kOsBlock) wcount[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const long long base = (long long)tile * kTile;
    const int count = (int)min((long long)kTile, (long long)n - base);

    // Warp w owns items [w*32*kItems, (w+1)*32*kItems) of the tile in index
    // order; item i of lane l is at w*32*kItems + i*32 + l.
    K key[kItems];
    int val[kItems];
    int rk[kItems];  // rank within the warp (low 16 bits) | digit << 16
    const int wbase = warp * 32 * kItems;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        if (t < count) {
            key[i] = keys_in[base + t];
            val[i] = vals_in[base + t];
        }
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        const bool valid = t < count;
        const unsigned dg = valid ? SortKey<K>::digit(key[i], shift, mask) : (unsigned)R + lane;
        const unsigned peers = __match_any_sync(kFull, dg);
        int before = 0;
        if (valid) before = wcount[warp * R + dg];
        __syncwarp();
        if (valid && lane == (int)(__ffs(peers) - 1)) wcount[warp * R + dg] = before + __popc(peers);
        __syncwarp();
        rk[i] = (before + __popc(peers & lanemask_lt())) | (int)(dg << 16);
    }
    __syncthreads();

    // per digit: exclusive prefix over warps and the tile's count of it;
    // then the exclusive prefix over digits (local start of each digit run).
    // Thread t owns the `per` consecutive digits starting at t * per.
    {
        const int per = (R + kOsBlock - 1) / kOsBlock;  // 1 or 2 (R <= 512)
        int tots[(kMaxBuckets + kOsBlock - 1) / kOsBlock];
        int sum = 0;
#pragma unroll
        for (int u = 0; u < (kMaxBuckets + kOsBlock - 1) / kOsBlock; ++u) {
            tots[u] = 0;
            const int b = threadIdx.x * per + u;
            if (u < per && b < R) {
                int tot = 0;
#pragma unroll
                for (int w = 0; w < kOsWarps; ++w) {
                    const int c = wcount[w * R + b];
                    wcount[w * R + b] = tot;
                    tot += c;
                }
                goff[b] = tot;  // tile count of digit b, published by the look-back
                tots[u] = tot;
                sum += tot;
            }
        }
        int all;
        int ex = block_exclusive_scan(sum, sm, &all);
#pragma unroll
        for (int u = 0; u < (kMaxBuckets + kOsBlock - 1) / kOsBlock; ++u) {
            const int b = threadIdx.x * per + u;
            if (u < per && b < R) {
                ldstart[b] = ex;
                ex += tots[u];
            }
        }
        __syncthreads();
    }

    // decoupled look-back: one thread per digit
    for (int b = threadIdx.x; b < R; b += kOsBlock) {
        const unsigned own = (unsigned)goff[b];
        unsigned long long* my = status + (long long)tile * R + b;
        unsigned excl = 0;
        if (tile == 0) {
            st_relaxed(my, ((unsigned long long)kFlagInc << 32) | own);
        } else {
            st_relaxed(my, ((unsigned long long)kFlagAgg << 32) | own);
            int t = tile - 1;
            int polls = 0;
            while (true) {
                const unsigned long long v = ld_relaxed(status + (long long)t * R + b);
                const unsigned flag = (unsigned)(v >> 32);
                if (flag == 0u) {
                    if (++polls > kMaxPolls) {
                        atomicOr(err, kDevTimeout);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                excl += (unsigned)v;
                if (flag == kFlagInc || t == 0) break;
                --t;
            }
            st_relaxed(my, ((unsigned long long)kFlagInc << 32) | (excl + own));
        }
        goff[b] = dstart_g[b] + (int)excl;
    }
    __syncthreads();

    // keys and values into tile-local digit order through shared memory
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = wbase + i * 32 + lane;
        if (t < count) {
            const int dg = rk[i] >> 16;
            const int pos = ldstart[dg] + wcount[warp * R + dg] + (rk[i] & 0xffff);
            skeys[pos] = key[i];
            svals[pos] = val[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = i * kOsBlock + threadIdx.x;
        if (t < count) {
            const K k = skeys[t];
            const unsigned dg = SortKey<K>::digit(k, shift, mask);
            const int dst = goff[dg] + (t - ldstart[dg]);
            keys_out[dst] = k;
            vals_out[dst] = svals[t];
        }
    }
}

template <typename K> static size_t onesweep_smem(int R) {
    return sizeof(K) * os_tile<K>() + sizeof(int) * os_tile<K>() + sizeof(int) * (kOsWarps * R + 2 * R);
}

template <typename K>
static cudaError_t quantise_t(const int* X, const Params& p, K* ka, int* va, int* tmp, cudaStream_t st) {
    const SortPlan sp = sort_plan(p.n, p.key_words, p.key_bits);
    const SortTmp t = sort_tmp(tmp, sp);
    const int R = sp.buckets;
    if (sp.passes > 0) {
        cudaError_t e = cudaMemsetAsync(t.hist, 0, sizeof(int) * (size_t)sp.passes * R, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.counters, 0, sizeof(int) * sp.passes, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(t.status, 0, sizeof(unsigned long long) * (size_t)sp.passes * sp.tiles * R, st);
        if (e != cudaSuccess) return e;
    }
    int blocks = (p.n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    quantise_hist_kernel<K><<<blocks, 256, sizeof(int) * (size_t)sp.passes * R, st>>>(X, p, ka, va, t.hist,
                                                                                       sp.passes, sp.bits);
    GD_COUNT_LAUNCH();
    if (sp.passes > 0) {
        digit_scan_kernel<<<sp.passes, 256, 0, st>>>(t.hist, t.dstart, R);
        GD_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

template <typename K>
static cudaError_t passes_t(const Params& p, K* ka, int* va, K* kb, int* vb, int* tmp, unsigned* err, cudaStream_t st,
                            int* result_in_b) {
    const SortPlan sp = sort_plan(p.n, p.key_words, p.key_bits);
    const SortTmp t = sort_tmp(tmp, sp);
    const int R = sp.buckets;
    *result_in_b = 0;
    if (sp.passes == 0 || p.n <= 1) return cudaSuccess;
    const size_t smem = onesweep_smem<K>(R);
    cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    K* src_k = ka;
    int* src_v = va;
    K* dst_k = kb;
    int* dst_v = vb;
    for (int ps = 0; ps < sp.passes; ++ps) {
        onesweep_kernel<K><<<sp.tiles, kOsBlock, smem, st>>>(src_k, src_v, dst_k, dst_v, p.n, ps * sp.bits, sp.bits,
                                                             t.dstart + ps * R,
                                                             t.status + (size_t)ps * sp.tiles * R,
                                                             t.counters + ps, err);
        GD_COUNT_LAUNCH();
        K* tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        int* tv = src_v;
        src_v = dst_v;
        dst_v = tv;
        *result_in_b ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t quantise_hist(const int* X, const Params& p, void* keys_a, int* vals_a, int* tmp, cudaStream_t st) {
    if (p.key_words == 1) return quantise_t(X, p, (unsigned long long*)keys_a, vals_a, tmp, st);
    return quantise_t(X, p, (Key2*)keys_a, vals_a, tmp, st);
}

cudaError_t sort_passes(const Params& p, void* keys_a, int* vals_a, void* keys_b, int* vals_b, int* tmp, unsigned* err,
                        cudaStream_t st, int* result_in_b) {
    if (p.key_words == 1)
        return passes_t(p, (unsigned long long*)keys_a, vals_a, (unsigned long long*)keys_b, vals_b, tmp, err, st,
                        result_in_b);
    return passes_t(p, (Key2*)keys_a, vals_a, (Key2*)keys_b, vals_b, tmp, err, st, result_in_b);
}

}  // namespace gd
