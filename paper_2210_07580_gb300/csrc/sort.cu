// Grid identifiers (Eq. 1) and the stable LSD radix sort of Alg. 1.
//
// The paper sorts by counting sort one dimension at a time; here the
// identifiers are packed into one 64- or 128-bit key (dimension 1 most
// significant, so key order is the lexicographic order of Alg. 1) and sorted
// by digits of up to 9 bits.  Quantisation computes the keys; then every
// digit position is one pass of three steps over tiles of consecutive keys:
//   1. upsweep: each tile's digit histogram;
//   2. tile scan: per digit, exclusive offsets over the tiles (within chunks
//      of tiles, then over the chunks) and the digit starts, the exclusive
//      scan of the digit totals;
//   3. downsweep: each tile ranks its keys stably in shared memory and writes
//      each digit run to its start plus the tile's offset.
// No tile waits for another.  When the key and the point index fit in 64
// bits together, the index rides in the low bits of the key (no separate
// values): a pass then moves 8 bytes per point each way, not 12, and since
// the passes are stable and look only at key digits, the order is the same.
#include <atomic>
#include <type_traits>

#include "gd_internal.cuh"

namespace gd {

constexpr int kMaxDigitBits = 9;
constexpr int kMaxBuckets = 1 << kMaxDigitBits;
constexpr int kOsBlock = 256;
constexpr int kOsWarps = kOsBlock / 32;

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

// One instance's sort workspace (ints): per-tile digit counts (then offsets
// within the tile's chunk) [tiles][R], per-chunk digit totals (then offsets
// over the chunks) [chunks][R], digit starts [R].  Nothing needs clearing:
// every pass writes all of it before reading it.
static size_t sort_chunks(const SortPlan& sp) { return (size_t)(sp.tiles + kSortChunk - 1) / kSortChunk; }

size_t sort_tmp_ints(int n, int key_words, int key_bits) {
    const SortPlan sp = sort_plan(n, key_words, key_bits);
    return ((size_t)sp.tiles + sort_chunks(sp)) * sp.buckets + (size_t)sp.buckets + 64;
}

void sort_tmp_layout(int* base, int n, int key_words, int key_bits, int** tcnt, int** ctot, int** dstart) {
    const SortPlan sp = sort_plan(n, key_words, key_bits);
    *tcnt = base;
    *ctot = base + (size_t)sp.tiles * sp.buckets;
    *dstart = *ctot + sort_chunks(sp) * sp.buckets;
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

// One block per tile of kQuantTile points of one instance: the keys and (for
// unpacked keys) the values, the input index; for packed keys whose in-cell
// offsets fit a word (Params::xoff_w > 0), that word.  For 64-bit keys a quantise tile
// is a sort tile, so the block also writes the tile's histogram of the first
// digit position (the first pass then needs no upsweep).
template <typename K, bool PACKED>
__global__ void __launch_bounds__(256) quantise_kernel(const Inst* __restrict__ ins, Flat f) {
    constexpr bool kHist = os_tile<K>() == kQuantTile;
    __shared__ int hist[kHist ? kMaxBuckets : 1];
    const int k = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[k]];
    const long long tile = blockIdx.x - f.off[k];
    const Params& p = I.p;
    const int n = p.n, d = p.d;
    const int R = 1 << I.digit_bits;
    const unsigned mask = (unsigned)R - 1u;
    const bool hist_on = kHist && I.passes > 0;
    if (hist_on) {
        for (int b = threadIdx.x; b < R; b += 256) hist[b] = 0;
        __syncthreads();
    }
    const int lane = lane_id();
    K* keys = (K*)I.keyA;
    for (int r = 0; r < kQuantTile; r += 256) {
        const long long i = tile * kQuantTile + r + threadIdx.x;
        const bool valid = i < n;
        K key;
        zero_key(key);
        if (valid) {
            const int* row = I.X + i * d;
            unsigned xoff = 0;
#pragma unroll
            for (int j = 0; j < kMaxD; ++j)
                if (j < d) {
                    const int x = __ldcs(row + j);
                    const unsigned id = identifier(x, p.mn[j], p.s_mul);
                    pack_key(key, id, p.shift[j]);
                    if constexpr (PACKED)
                        if (p.xoff_w > 0) xoff |= ((unsigned)(x - p.mn[j]) - id * (unsigned)p.s) << (j * p.xoff_w);
                }
            if constexpr (PACKED) {
                // key above the point index: one word carries both
                keys[i] = (unsigned long long)key << p.pack_bits | (unsigned long long)i;
                if (p.xoff_w > 0) __stcs(in_cell_offsets(I) + i, (int)xoff);  // read after the sort
            } else {
                keys[i] = key;
                I.valA[i] = (int)i;
            }
        }
        if (hist_on) {
            // runs of equal digits over consecutive lanes are added once
            const unsigned dg = valid ? SortKey<K>::digit(key, 0, mask) : (unsigned)R + lane;
            const unsigned prev = __shfl_up_sync(kFull, dg, 1);
            const bool start = lane == 0 || dg != prev;
            const unsigned starts = __ballot_sync(kFull, start);
            if (valid && start) {
                const unsigned above = starts & ~((2u << lane) - 1u);
                atomicAdd(&hist[dg], (above ? __ffs(above) - 1 : 32) - lane);
            }
        }
    }
    if (hist_on) {
        __syncthreads();
        int* out = I.sort_tcnt + tile * R;
        for (int b = threadIdx.x; b < R; b += 256) out[b] = hist[b];
    }
}

// ------------------------------------------------------------- one pass

template <typename K, bool PACKED> __device__ __forceinline__ int pass_shift(const Inst& I, int pass) {
    return pass * I.digit_bits + (PACKED ? I.p.pack_bits : 0);
}

// Upsweep: the digit histogram of each tile (one block per tile) into
// sort_tcnt[tile][*].  Runs of equal digits over consecutive lanes are added
// once, which keeps the shared-memory atomics cheap on clustered data.
template <typename K, bool PACKED>
__global__ void __launch_bounds__(kOsBlock) upsweep_kernel(const Inst* __restrict__ ins, Flat f, int pass) {
    constexpr int kTile = os_tile<K>();
    __shared__ int hist[kMaxBuckets];
    const int kk = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[kk]];
    const int tile = blockIdx.x - (int)f.off[kk];
    const int R = 1 << I.digit_bits, shift = pass_shift<K, PACKED>(I, pass);
    const unsigned mask = (unsigned)R - 1u;
    for (int b = threadIdx.x; b < R; b += kOsBlock) hist[b] = 0;
    __syncthreads();
    const K* keys = (const K*)((pass & 1) ? I.keyB : I.keyA);
    const long long base = (long long)tile * kTile;
    const int count = (int)min((long long)kTile, (long long)I.p.n - base);
    const int lane = lane_id();
    // all of the thread's digits first (their loads in flight together)
    constexpr int kItems = kTile / kOsBlock;
    unsigned dgs[kItems];
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
        const int t = u * kOsBlock + threadIdx.x;
        dgs[u] = t < count ? SortKey<K>::digit(keys[base + t], shift, mask) : (unsigned)R + lane;
    }
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
        const bool valid = u * kOsBlock + (int)threadIdx.x < count;
        const unsigned dg = dgs[u];
        const unsigned prev = __shfl_up_sync(kFull, dg, 1);
        const bool start = lane == 0 || dg != prev;
        const unsigned starts = __ballot_sync(kFull, start);
        if (valid && start) {
            const unsigned above = starts & ~((2u << lane) - 1u);
            atomicAdd(&hist[dg], (above ? __ffs(above) - 1 : 32) - lane);
        }
    }
    __syncthreads();
    int* out = I.sort_tcnt + (long long)tile * R;
    for (int b = threadIdx.x; b < R; b += kOsBlock) out[b] = hist[b];
}

// Tile scan: one block per chunk of kSortChunk consecutive tiles, a thread
// per digit: the digit's exclusive offsets over the chunk's tiles, in place
// (the rows are read and written whole, so every access is contiguous), and
// the chunk's digit totals.  The block that finishes an instance's last chunk
// (counted in small[kSmSortChunks]) turns the chunk totals into offsets over
// the chunks and writes the digit starts: the exclusive scan of the digit
// totals.  A tile's offset of digit b is then
// dstart[b] + ctot[chunk][b] + tcnt[tile][b].  No block waits for another.
constexpr int kTileScanBlock = kMaxBuckets;

__global__ void __launch_bounds__(kTileScanBlock) tile_scan_kernel(const Inst* __restrict__ ins, Flat f, int pass) {
    __shared__ int sm[33];
    __shared__ int s_last;
    const int kk = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[kk]];
    if (pass >= I.passes) return;  // block-uniform
    const int c = blockIdx.x - (int)f.off[kk];
    const int R = 1 << I.digit_bits, tiles = I.tiles;
    const int nch = (tiles + kSortChunk - 1) / kSortChunk;
    const int b = threadIdx.x;
    const int t0 = c * kSortChunk, rows = min(kSortChunk, tiles - t0);
    int* tcnt = I.sort_tcnt;
    int* ctot = I.sort_ctot;
    if (b < R) {
        int v[kSortChunk];
#pragma unroll
        for (int i = 0; i < kSortChunk; ++i) v[i] = i < rows ? tcnt[(long long)(t0 + i) * R + b] : 0;
        int run = 0;
#pragma unroll
        for (int i = 0; i < kSortChunk; ++i)
            if (i < rows) {
                tcnt[(long long)(t0 + i) * R + b] = run;
                run += v[i];
            }
        ctot[(long long)c * R + b] = run;
    }
    // the last chunk done: its block sees every chunk's totals
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(I.small + kSmSortChunks, 1) == nch - 1;
    __syncthreads();
    if (!s_last) return;
    int run = 0;
    if (b < R) {
        for (int c0 = 0; c0 < nch; c0 += kSortChunk) {
            int v[kSortChunk];
#pragma unroll
            for (int i = 0; i < kSortChunk; ++i) v[i] = c0 + i < nch ? __ldcg(ctot + (long long)(c0 + i) * R + b) : 0;
#pragma unroll
            for (int i = 0; i < kSortChunk; ++i)
                if (c0 + i < nch) {
                    ctot[(long long)(c0 + i) * R + b] = run;
                    run += v[i];
                }
        }
    }
    int total;
    const int ex = block_exclusive_scan(b < R ? run : 0, sm, &total);
    if (b < R) I.sort_dstart[b] = ex;
    if (threadIdx.x == 0) I.small[kSmSortChunks] = 0;  // the next pass counts again
}

// Downsweep: one block per tile ranks its keys stably in shared memory and
// writes each digit run to (digit start + the tile's offset of the digit).
template <typename K, bool PACKED>
__global__ void __launch_bounds__(kOsBlock, PACKED ? 3 : 2)
    downsweep_kernel(const Inst* __restrict__ ins, Flat f, int pass) {
    constexpr int kItems = SortKey<K>::kItems;
    constexpr int kTile = os_tile<K>();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sm[33];
    const int kk = flat_find(f, blockIdx.x);
    const Inst& I = ins[f.idx[kk]];
    const int tile = blockIdx.x - (int)f.off[kk];
    const int n = I.p.n, shift = pass_shift<K, PACKED>(I, pass);
    const int R = 1 << I.digit_bits;
    const unsigned mask = (unsigned)R - 1u;
    const K* keys_in = (const K*)((pass & 1) ? I.keyB : I.keyA);
    K* keys_out = (K*)((pass & 1) ? I.keyA : I.keyB);
    const int* vals_in = (pass & 1) ? I.valB : I.valA;
    int* vals_out = (pass & 1) ? I.valA : I.valB;

    // layout: exchange keys [kTile] K, exchange vals [kTile] int (unpacked),
    //         wcount [kOsWarps][R], ldstart [R], goff [R]
    K* skeys = reinterpret_cast<K*>(smem);
    int* svals = reinterpret_cast<int*>(smem + sizeof(K) * kTile);
    int* wcount = svals + (PACKED ? 0 : kTile);
    int* ldstart = wcount + kOsWarps * R;
    int* goff = ldstart + R;

    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kOsWarps * R; i += kOsBlock) wcount[i] = 0;
    // the tile's global start of each digit
    const int* ctot = I.sort_ctot + (long long)(tile / kSortChunk) * R;
    for (int b = threadIdx.x; b < R; b += kOsBlock)
        goff[b] = I.sort_dstart[b] + ctot[b] + I.sort_tcnt[(long long)tile * R + b];
    __syncthreads();
    const long long base = (long long)tile * kTile;
    const int count = (int)min((long long)kTile, (long long)n - base);

    // Full tiles (all but an instance's last) run a copy of the body in which
    // every bound check is known to hold.
    auto run = [&](auto full) {
        const int cnt = decltype(full)::value ? kTile : count;
        // Warp w owns items [w*32*kItems, (w+1)*32*kItems) of the tile in index
        // order; item i of lane l is at w*32*kItems + i*32 + l.
        K key[kItems];
        [[maybe_unused]] int val[PACKED ? 1 : kItems];  // index values (unpacked keys only)
        int rk[kItems];  // rank within the warp (low 16 bits) | digit << 16
        const int wbase = warp * 32 * kItems;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int t = wbase + i * 32 + lane;
            if (t < cnt) {
                key[i] = keys_in[base + t];
                if constexpr (!PACKED) val[i] = vals_in[base + t];
            }
        }
        const int bits = I.digit_bits;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int t = wbase + i * 32 + lane;
            const bool valid = t < cnt;
            const unsigned dg = valid ? SortKey<K>::digit(key[i], shift, mask) : (unsigned)R + lane;
            // lanes with the same digit: one ballot per digit bit (a constant
            // cost, where a match instruction's grows with the distinct digits)
            unsigned peers = cnt == kTile ? kFull : __ballot_sync(kFull, valid);
            if (!valid) peers = 1u << lane;
#pragma unroll
            for (int b = 0; b < kMaxDigitBits; ++b) {
                if (b >= bits) break;
                const bool on = (dg >> b) & 1u;
                const unsigned bal = __ballot_sync(kFull, on);
                peers &= on ? bal : ~bal;
            }
            int before = 0;
            if (valid) before = wcount[warp * R + dg];
            __syncwarp();
            if (valid && lane == (int)(__ffs(peers) - 1)) wcount[warp * R + dg] = before + __popc(peers);
            __syncwarp();
            rk[i] = (before + __popc(peers & lanemask_lt())) | (int)(dg << 16);
        }
        __syncthreads();

        // per digit: exclusive prefix over warps; then the exclusive prefix over
        // digits (local start of each digit run).  Thread t owns the `per`
        // consecutive digits starting at t * per.
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

        // keys and values into tile-local digit order through shared memory
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int t = wbase + i * 32 + lane;
            if (t < cnt) {
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
            if (t < cnt) {
                const K k2 = skeys[t];
                const unsigned dg = SortKey<K>::digit(k2, shift, mask);
                const int dst = goff[dg] + (t - ldstart[dg]);
                keys_out[dst] = k2;
                if constexpr (!PACKED) vals_out[dst] = svals[t];
            }
        }
    };
    if (count == kTile)
        run(std::true_type{});
    else
        run(std::false_type{});
}

template <typename K, bool PACKED> static size_t downsweep_smem(int R) {
    return sizeof(K) * os_tile<K>() + (PACKED ? 0 : sizeof(int) * os_tile<K>()) + sizeof(int) * (kOsWarps * R + 2 * R);
}

// ------------------------------------------------------------- launches

cudaError_t launch_quantise(const Inst* ins, Flat qtiles, long long total, int key_class, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (key_class == 0)
        quantise_kernel<unsigned long long, true><<<(unsigned)total, 256, 0, st>>>(ins, qtiles);
    else if (key_class == 1)
        quantise_kernel<unsigned long long, false><<<(unsigned)total, 256, 0, st>>>(ins, qtiles);
    else
        quantise_kernel<Key2, false><<<(unsigned)total, 256, 0, st>>>(ins, qtiles);
    GD_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t prepare_sort() {
    static std::atomic<unsigned long long> done{0};  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(downsweep_kernel<unsigned long long, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)downsweep_smem<unsigned long long, true>(kMaxBuckets));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(downsweep_kernel<unsigned long long, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)downsweep_smem<unsigned long long, false>(kMaxBuckets));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(downsweep_kernel<Key2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)downsweep_smem<Key2, false>(kMaxBuckets));
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

void record_event(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

template <typename K, bool PACKED>
static void pass_launch(const Inst* ins, Flat tiles, long long total, Flat chunks, long long chunk_total, int pass,
                        int max_buckets, cudaStream_t st, cudaEvent_t ev_a, cudaEvent_t ev_b) {
    if (pass > 0 || os_tile<K>() != kQuantTile) {  // quantisation wrote the first histograms
        upsweep_kernel<K, PACKED><<<(unsigned)total, kOsBlock, 0, st>>>(ins, tiles, pass);
        GD_COUNT_LAUNCH();
    }
    tile_scan_kernel<<<(unsigned)chunk_total, kTileScanBlock, 0, st>>>(ins, chunks, pass);
    GD_COUNT_LAUNCH();
    if (ev_a) record_event(ev_a, st);
    downsweep_kernel<K, PACKED><<<(unsigned)total, kOsBlock, downsweep_smem<K, PACKED>(max_buckets), st>>>(ins, tiles,
                                                                                                      pass);
    GD_COUNT_LAUNCH();
    if (ev_b) record_event(ev_b, st);
}

cudaError_t launch_sort_pass(const Inst* ins, Flat tiles, long long total, Flat chunks, long long chunk_total,
                             int key_class, int pass, int max_buckets, cudaStream_t st, cudaEvent_t ev_a,
                             cudaEvent_t ev_b) {
    if (total <= 0 || tiles.K <= 0 || chunk_total <= 0) return cudaSuccess;
    if (key_class == 0)
        pass_launch<unsigned long long, true>(ins, tiles, total, chunks, chunk_total, pass, max_buckets, st, ev_a,
                                              ev_b);
    else if (key_class == 1)
        pass_launch<unsigned long long, false>(ins, tiles, total, chunks, chunk_total, pass, max_buckets, st, ev_a,
                                               ev_b);
    else
        pass_launch<Key2, false>(ins, tiles, total, chunks, chunk_total, pass, max_buckets, st, ev_a, ev_b);
    return cudaGetLastError();
}

}  // namespace gd
