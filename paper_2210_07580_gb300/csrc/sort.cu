// Grid identifiers (Eq. 1) and the stable LSD radix sort of Alg. 1.
//
// The paper sorts by counting sort one dimension at a time; here the
// identifiers are packed into one 64- or 128-bit key (dimension 1 most
// significant, so key order is the lexicographic order of Alg. 1) and sorted
// by digits of up to 9 bits:
//   1. quantise_hist: computes every key and, in the same pass, the
//      histogram of every digit position;
//   2. digit_scan: exclusive scan of each digit position's histogram;
//   3. one onesweep pass per digit position: each block takes the next tile
//      (dynamic tile ids), ranks its keys stably in shared memory, publishes
//      its per-digit counts and finds the counts of all earlier tiles of its
//      instance by a decoupled look-back, then writes each digit run out
//      contiguously.
// A pass reads and writes every key and value once.  When the key and the
// point index fit in 64 bits together, the index rides in the low bits of the
// key (no separate values): a pass then moves 16 bytes per point, not 24,
// and since the passes are stable and look only at key digits, the order is
// the same.  Look-back waits are
// bounded: a block only ever waits for tiles handed out before its own (tile
// ids are taken in order from one counter over the whole batch), and gives
// up with kDevTimeout after a fixed number of polls.
#include <atomic>

#include "gd_internal.cuh"

namespace gd {

constexpr int kMaxDigitBits = 9;
constexpr int kMaxBuckets = 1 << kMaxDigitBits;
constexpr int kOsBlock = 256;
constexpr int kOsWarps = kOsBlock / 32;
constexpr unsigned kFlagAgg = 1u, kFlagInc = 2u;
constexpr int kMaxPolls = 1 << 22;
constexpr int kLookback = 8;

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

// Layout of one instance's sort workspace (ints): hist [P][R],
// dstart [P][R], tile counters [P], status [P][tiles][R] (64-bit words).
// Everything but dstart must be zero before quantise_hist runs.
size_t sort_tmp_ints(int n, int key_words, int key_bits) {
    const SortPlan sp = sort_plan(n, key_words, key_bits);
    const size_t pr = (size_t)sp.passes * sp.buckets;
    return 2 * pr + (size_t)sp.passes + 8 + 2 * (size_t)sp.passes * sp.tiles * sp.buckets + 64;
}

void sort_tmp_layout(int* base, int n, int key_words, int key_bits, int** hist, int** dstart, int** counters,
                     unsigned long long** status, size_t* zero_ints) {
    const SortPlan sp = sort_plan(n, key_words, key_bits);
    const size_t pr = (size_t)sp.passes * sp.buckets;
    // hist, counters and status first (one region to clear), dstart last
    *hist = base;
    *counters = base + pr;
    size_t off = pr + sp.passes + 8;
    off = (off + 1) & ~(size_t)1;  // 8-byte alignment (base is 256-byte aligned)
    *status = reinterpret_cast<unsigned long long*>(base + off);
    off += 2 * (size_t)sp.passes * sp.tiles * sp.buckets;
    *zero_ints = off;
    *dstart = base + off;
}

// ------------------------------------------------------------- quantise

__device__ __forceinline__ unsigned identifier(int x, int mn, unsigned long long s_mul) {
    // (x - mn) fits in 32 unsigned bits; an identifier is at most 2^31 - 1
    // because d * range^2 < 2^62 is checked before this runs.  The division
    // by the cell side is a multiply-high (Params::s_mul).
    const unsigned diff = (unsigned)(x - mn);
    return s_mul ? (unsigned)__umul64hi(s_mul, (unsigned long long)diff) : diff;
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

// One block per tile of kQuantTile points of one instance: keys, values
// (input index) and the tile's histogram of every digit position, added to
// the instance's histograms.  Runs of equal digits over consecutive lanes are
// counted once, which keeps shared-memory atomics cheap on clustered data.
template <typename K, bool PACKED>
__global__ void __launch_bounds__(256) quantise_hist_kernel(const Inst* __restrict__ ins, Flat f) {
    extern __shared__ int sh_hist[];  // [passes][1 << bits]
    const int k = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[k]];
    const long long tile = blockIdx.x - f.off[k];
    const int passes = I.passes, bits = I.digit_bits;
    const int R = 1 << bits;
    const unsigned mask = (unsigned)R - 1u;
    for (int i = threadIdx.x; i < passes * R; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    const int lane = lane_id();
    const Params& p = I.p;
    const int n = p.n, d = p.d;
    K* keys = (K*)I.keyA;
    for (int r = 0; r < kQuantTile; r += 256) {
        const long long i = tile * kQuantTile + r + threadIdx.x;
        const bool valid = i < n;
        K key;
        zero_key(key);
        if (valid) {
            const int* row = I.X + i * d;
#pragma unroll
            for (int j = 0; j < kMaxD; ++j)
                if (j < d) pack_key(key, identifier(__ldg(row + j), p.mn[j], p.s_mul), p.shift[j]);
            if constexpr (PACKED) {
                // key above the point index: one word carries both
                keys[i] = (unsigned long long)key << p.pack_bits | (unsigned long long)i;
            } else {
                keys[i] = key;
                I.valA[i] = (int)i;
            }
        }
        for (int ps = 0; ps < passes; ++ps) {
            // runs of equal digits over consecutive lanes (clustered inputs
            // give long runs) are added once, by their first lane
            const unsigned dg = valid ? SortKey<K>::digit(key, ps * bits, mask) : (unsigned)R + lane;
            const unsigned prev = __shfl_up_sync(kFull, dg, 1);
            const bool start = lane == 0 || dg != prev;
            const unsigned starts = __ballot_sync(kFull, start);
            if (valid && start) {
                const unsigned above = starts & ~((2u << lane) - 1u);
                const int next = above ? __ffs(above) - 1 : 32;
                atomicAdd(&sh_hist[ps * R + dg], next - lane);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * R; i += blockDim.x)
        if (sh_hist[i]) atomicAdd(I.sort_hist + i, sh_hist[i]);
}

// One block per (instance, pass): exclusive scan of the pass's histogram.
__global__ void digit_scan_kernel(const Inst* __restrict__ ins, const int* __restrict__ idx) {
    __shared__ int sm[33];
    const Inst& I = ins[idx[blockIdx.x]];
    const int ps = blockIdx.y;
    if (ps >= I.passes) return;
    const int R = 1 << I.digit_bits;
    int carry = 0;
    for (int base = 0; base < R; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const int v = b < R ? I.sort_hist[ps * R + b] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sm, &total);
        if (b < R) I.sort_dstart[ps * R + b] = carry + ex;
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

template <typename K, bool PACKED>
__global__ void __launch_bounds__(kOsBlock, PACKED ? 3 : 2)
    onesweep_kernel(const Inst* __restrict__ ins, Flat f, int pass, int* flat_counter) {
    constexpr int kItems = SortKey<K>::kItems;
    constexpr int kTile = os_tile<K>();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sm[33];
    __shared__ int s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(flat_counter, 1);
    __syncthreads();
    const int ft = s_tile;
    const int kk = flat_find(f, ft);
    const Inst& I = ins[f.idx[kk]];
    const int tile = ft - (int)f.off[kk];
    const int n = I.p.n, bits = I.digit_bits, shift = pass * bits + (PACKED ? I.p.pack_bits : 0);
    const int R = 1 << bits;
    const unsigned mask = (unsigned)R - 1u;
    const K* keys_in = (const K*)((pass & 1) ? I.keyB : I.keyA);
    K* keys_out = (K*)((pass & 1) ? I.keyA : I.keyB);
    const int* vals_in = (pass & 1) ? I.valB : I.valA;
    int* vals_out = (pass & 1) ? I.valA : I.valB;
    const int* dstart_g = I.sort_dstart + pass * R;
    unsigned long long* status = I.sort_status + (size_t)pass * I.tiles * R;

    // layout: exchange keys [kTile] K, exchange vals [kTile] int,
    //         wcount [kOsWarps][R], ldstart [R], goff [R]
    K* skeys = reinterpret_cast<K*>(smem);
    int* svals = reinterpret_cast<int*>(smem + sizeof(K) * kTile);
    int* wcount = svals + (PACKED ? 0 : kTile);
    int* ldstart = wcount + kOsWarps * R;
    int* goff = ldstart + R;

    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kOsWarps * R; i += kOsBlock) wcount[i] = 0;
    __syncthreads();
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
            if constexpr (!PACKED) val[i] = vals_in[base + t];
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
        constexpr int kPerMax = (kMaxBuckets + kOsBlock - 1) / kOsBlock;
        int tots[kPerMax];
        int sum = 0;
#pragma unroll
        for (int u = 0; u < kPerMax; ++u) {
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
        for (int u = 0; u < kPerMax; ++u) {
            const int b = threadIdx.x * per + u;
            if (u < per && b < R) {
                ldstart[b] = ex;
                ex += tots[u];
            }
        }
        __syncthreads();
    }

    // decoupled look-back: one thread per digit, reading kLookback earlier
    // tiles per round trip (loads of consecutive digits are coalesced) and
    // adding their counts up to the nearest inclusive one (tile 0's always is)
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
                unsigned long long v[kLookback];
#pragma unroll
                for (int j = 0; j < kLookback; ++j)
                    v[j] = t - j >= 0 ? ld_relaxed(status + (long long)(t - j) * R + b) : 0ull;
                int used = 0;
                bool done = false;
#pragma unroll
                for (int j = 0; j < kLookback; ++j) {
                    if (done || used < j) break;  // stop at the first unpublished tile
                    const unsigned flag = (unsigned)(v[j] >> 32);
                    if (flag == 0u) break;
                    excl += (unsigned)v[j];
                    used = j + 1;
                    if (flag == kFlagInc) done = true;
                }
                if (done) break;
                t -= used;
                if (used == 0) {
                    if (++polls > kMaxPolls) {
                        set_status(I, kDevTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
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
            if constexpr (!PACKED) svals[pos] = val[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int t = i * kOsBlock + threadIdx.x;
        if (t < count) {
            const K k2 = skeys[t];
            const unsigned dg = SortKey<K>::digit(k2, shift, mask);
            const int dst = goff[dg] + (t - ldstart[dg]);
            keys_out[dst] = k2;
            if constexpr (!PACKED) vals_out[dst] = svals[t];
        }
    }
}

template <typename K, bool PACKED> static size_t onesweep_smem(int R) {
    return sizeof(K) * os_tile<K>() + (PACKED ? 0 : sizeof(int) * os_tile<K>()) + sizeof(int) * (kOsWarps * R + 2 * R);
}

cudaError_t launch_quantise_hist(const Inst* ins, Flat qtiles, long long total, int key_class, int max_hist_ints,
                                 cudaStream_t st) {
    const long long tiles = total;
    if (tiles <= 0) return cudaSuccess;
    const size_t smem = sizeof(int) * (size_t)(max_hist_ints > 0 ? max_hist_ints : 1);
    if (key_class == 0)
        quantise_hist_kernel<unsigned long long, true><<<(unsigned)tiles, 256, smem, st>>>(ins, qtiles);
    else if (key_class == 1)
        quantise_hist_kernel<unsigned long long, false><<<(unsigned)tiles, 256, smem, st>>>(ins, qtiles);
    else
        quantise_hist_kernel<Key2, false><<<(unsigned)tiles, 256, smem, st>>>(ins, qtiles);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_digit_scan(const Inst* ins, const int* idx, int K, int max_passes, cudaStream_t st) {
    if (K <= 0 || max_passes <= 0) return cudaSuccess;
    digit_scan_kernel<<<dim3(K, max_passes), 256, 0, st>>>(ins, idx);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

template <typename K, bool PACKED>
static cudaError_t onesweep_launch(const Inst* ins, Flat tiles, long long total, int pass, int max_buckets,
                                   int* flat_counter, cudaStream_t st) {
    const size_t smem = onesweep_smem<K, PACKED>(max_buckets);
    onesweep_kernel<K, PACKED><<<(unsigned)total, kOsBlock, smem, st>>>(ins, tiles, pass, flat_counter);
    return cudaSuccess;
}

cudaError_t prepare_onesweep() {
    static std::atomic<unsigned long long> done{0};  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(onesweep_kernel<unsigned long long, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)onesweep_smem<unsigned long long, true>(kMaxBuckets));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(onesweep_kernel<unsigned long long, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<unsigned long long, false>(kMaxBuckets));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(onesweep_kernel<Key2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<Key2, false>(kMaxBuckets));
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

cudaError_t launch_onesweep(const Inst* ins, Flat tiles, long long total, int key_class, int pass, int max_buckets,
                            int* flat_counter, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    cudaError_t e;
    if (key_class == 0)
        e = onesweep_launch<unsigned long long, true>(ins, tiles, total, pass, max_buckets, flat_counter, st);
    else if (key_class == 1)
        e = onesweep_launch<unsigned long long, false>(ins, tiles, total, pass, max_buckets, flat_counter, st);
    else
        e = onesweep_launch<Key2, false>(ins, tiles, total, pass, max_buckets, flat_counter, st);
    if (e != cudaSuccess) return e;
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace gd
