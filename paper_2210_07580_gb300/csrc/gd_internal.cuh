// Internal declarations shared by the CUDA translation units of libgdbscan.
//
// Every stage runs over a batch of K independent DBSCAN instances (K = 1 for
// gd_dbscan).  An instance is described by an Inst record in device memory
// (its parameters and workspace pointers); a launch covers a flat space of
// items -- the points, grids, pairs ... of all instances concatenated -- and
// each thread, warp or block finds its instance from the space's offset table.
//
// Pipeline of one instance:
//   bounds -> identifiers (Eq. 1) + digit histograms -> radix sort (Alg. 1)
//   -> grid compaction + coordinate gather (Alg. 1) -> grid-tree levels
//   (Alg. 2) -> neighbour-grid walk (Alg. 3) -> core points (G13 rule,
//   Section 3.2) -> core-point packing -> core-grid merge (Def. 6-7, Alg. 4-5)
//   with union-find (LDF variant, Section 5.2) -> cluster ids -> labels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gd {

constexpr int kMaxD = 8;
// Largest stencil radius r = 1 + (isqrt(eps2) - 1) / s with s = 1 + isqrt(eps2 / d):
// s > sqrt(eps2 / d) gives (isqrt(eps2) - 1) / s < sqrt(d), so r <= 1 + floor(sqrt(8)) = 3.
constexpr int kMaxR = 3;
// Size buckets of instances (points): <= 2^12, 2^15, 2^18, 2^21, larger.
constexpr int kSizeBuckets = 5;
inline int size_bucket(long long n) {
    return n <= (1 << 12) ? 0 : n <= (1 << 15) ? 1 : n <= (1 << 18) ? 2 : n <= (1 << 21) ? 3 : 4;
}
constexpr unsigned kFull = 0xffffffffu;

// Bits of an instance's device status word (OR-ed by kernels).
//   kDevTimeout  a bounded union-find loop ran out (GD_ETIMEOUT);
//   kDevOverflow a buffer sized from an earlier call was too small (the
//                neighbour lists or FastMerging bitmaps): the result is not
//                valid and the call is run again with exact sizes;
//   kDevReplan   the grid key layout of the data does not fit the launch
//                plan reused from an earlier call: likewise;
//   kDevRange    d * R^2 >= 2^62 or a key wider than 128 bits (GD_ERANGE).
enum : unsigned { kDevTimeout = 1u, kDevOverflow = 2u, kDevReplan = 4u, kDevRange = 8u };

// Retry cap for the lock-free union-find loops: far above any legitimate
// number of CAS retries, so reaching it means something is wrong; the kernel
// then records kDevTimeout and gives up instead of spinning.  A context can
// lower it (gd_set_retry_limit, for tests of that path): Params::uf_cap.
constexpr int kMaxUfRetries = 1 << 20;

// Per-instance parameters, fixed once the bounds are known.
struct Params {
    int n;            // points
    int d;            // dimensions (1..8)
    int dp;           // padded row stride of the grid-order coordinates (1,2,4,8)
    long long eps2;   // squared radius (clamped below 2^62)
    // FastMerging's "yes" radius^2: eps2 (exact), or larger for approximate
    // FastMerging (the Remark after Alg. 5), which accepts a pair within
    // eps + delta and prunes as the exact one does
    long long eps2_yes;
    int minpts;
    long long s;      // integer cell side: largest s with d*(s-1)^2 <= eps2
    // floor(x / s) for 32-bit x as the high word of s_mul * x (s_mul =
    // floor((2^64 - 1) / s) + 1; exact for every 32-bit x and 2 <= s < 2^32:
    // Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019);
    // 0 when s = 1
    unsigned long long s_mul;
    long long r;      // largest |delta| per dimension whose gap alone is <= eps
    int key_bits;     // total bits of the packed grid key
    int key_words;    // 1 or 2 64-bit words
    // Sort key class: 0 = one 64-bit word holding the key above the point
    // index (pack_bits low bits; no separate values), 1 = 64-bit key plus
    // index values, 2 = 128-bit key plus index values.
    int key_class;
    int pack_bits;
    // Width of each dimension's in-cell offset (x - mn) - id * s when the d
    // offsets of a point fit one 32-bit word (packed keys only), else -1.
    // Quantisation then writes that word per point, and the compaction
    // rebuilds each grid-order row from its identifiers and the word instead
    // of gathering the input row.
    int xoff_w;
    int ldf;          // merge order: 0 = touching pairs first, 1 = low density first (Section 5.2)
    int uf_cap;       // iterations a union-find loop may take before it gives up
    int mn[kMaxD];    // per-dimension minimum coordinate
    int bits[kMaxD];  // bits of each identifier in the key
    int shift[kMaxD]; // bit offset of identifier j (dimension 0 most significant)
};

// 128-bit grid key for identifiers wider than 64 bits in total.
struct Key2 {
    unsigned long long lo, hi;
};

// Slots of an instance's small device block (ints).
enum SmallSlot {
    kSmMnmx = 0,        // [16] per-dimension min then max
    kSmCells = 16,      // C
    kSmStatus = 17,     // status bits
    kSmMaxCell = 18,    // largest grid
    kSmNnbr = 19,       // neighbour-list length
    kSmNonfull = 20,    // points of non-full grids
    kSmPairsT = 21,     // candidate pairs taken by the merge
    kSmHard0 = 23,      // pairs handed to FastMerging, wave 0
    kSmHard1 = 24,      // ... wave 1
    kSmPool = 26,       // [2] instance 0 only: 64-bit neighbour-pool counter
    kSmKeyClass = 28,   // the sort plan: key class,
    kSmKeyBits = 29,    // ... key bits (the device's layout when it computes it),
    kSmKeyWords = 30,   // ... key words
    kSmLevelCount = 32, // [8] nodes per grid-tree level
    kSmSortChunks = 40, // sort tile scan: chunks of the current pass done (the last one resets it)
    kSmallInts = 64
};

// Run statistics (gd_set_stats): 64-bit counters per instance, kept only when
// the context asks for them (Inst::stats non-null).  Slot names are in
// kStatNames (api.cu); kStKappa is a histogram of FastMerging rounds.
enum StatSlot {
    kStPairs = 0,      // candidate pairs of neighbouring core grids
    kStSkipped,        // ... skipped: the two grids were already in one set
    kStBoxNo,          // ... decided "no" by the gap between the core boxes
    kStBoxYes,         // ... decided "yes" by the core boxes' farthest corners
    kStLane,           // ... decided by one lane's exact loop
    kStWarp,           // ... decided by the warp's exact tiles
    kStHanded,         // ... handed to FastMerging (Alg. 5)
    kStFmYes,          // FastMerging answers
    kStFmNo,
    kStFmTriangle,     // points FastMerging removed by the triangle test (Alg. 4)
    kStFmAngle,        // points it removed by the angle test (Alg. 4, Def. 8)
    kStNonfull,        // points of non-full grids (their core flag is counted)
    kStCountRows,      // rows of neighbour grids a count would stage once per non-full grid
    kStDistCore,       // exact squared distances evaluated: core counting,
    kStDistMerge,      // ... merging (lane loops and warp tiles),
    kStDistFm,         // ... FastMerging (every pass, the angle bound included),
    kStDistLabels,     // ... border labels
    kStWalkNodes,      // tree nodes whose key the neighbour walk tested (Alg. 3)
    kStWalkSteps,      // warp steps of the walk (up to 32 node tests each)
    kStKappa,          // [kKappaBins] FastMerging rounds 1, 2, ..., then >= kKappaBins
    kKappaBins = 16,
    kStatCount = kStKappa + kKappaBins
};

__device__ __forceinline__ void stat_add(unsigned long long* stats, int slot, unsigned long long v) {
    if (stats && v) atomicAdd(stats + slot, v);
}

// One instance: parameters and workspace, in device memory.
struct Inst {
    Params p;
    int passes, digit_bits, tiles;  // radix-sort plan
    unsigned long long* stats;      // [kStatCount] or null (statistics off)
    const int* X;
    int* labels;
    unsigned char* is_core;
    int* small;  // [kSmallInts]
    void* keyA;
    void* keyB;
    int* valA;
    int* valB;  // packed keys: the sorted permutation in one of valA/valB, the in-cell offsets in the other
    int* Xs;  // [n][dp] coordinates in grid order
    int* pt_cell;
    unsigned char* core_s;
    int* Xc;  // [n][dp] core points packed per grid
    int* cell_start;
    int* cell_coord;
    int* pbox;  // [C][2d] box of each grid's points: d minima, then d maxima
    int* lv_key[kMaxD];
    int* lv_cb[kMaxD];
    int* lv_E;  // [d][C+1] level scratch
    int* lv_L;  // [C]
    // Neighbour lists: list(c) holds the grids g' >= c the walk found from c
    // (forward part, nbr_fwd[c] entries) followed by the grids g < c whose
    // walks found c (backward part); nbr_bwd counts the backward entries,
    // then (from the list check on) holds the absolute position of the next
    // backward entry of c.
    int* nbr_start;
    int* nbr;
    int* nbr_fwd;
    int* nbr_bwd;
    long long nbr_cap;  // entries the instance's list buffer holds (and its hard-pair buffer)
    int* nf_start;
    int* nf_pts;  // [points counted one by one] their index in grid order (shares lv_E's space)
    int* core_start;
    int* bbox;
    int* ldf_grid;  // low-density-first order: the grid at each slot (core grids by core count first)
    int* ldf_ctr;  // [kLdfBuckets] bucket counts, then cursors
    int2* hard;  // pairs handed to FastMerging: wave 0's, then wave 1's
    int* parent;
    int* cid_root;
    int* cell_cid;
    int* bcnt;  // compaction: per-tile grid starts (scanned)
    int* sort_tcnt;    // [tiles][R] per-tile digit counts, then offsets within the tile's chunk
    int* sort_ctot;    // [chunks][R] per-chunk digit totals, then offsets over the chunks
    int* sort_dstart;  // [R] digit starts of the current pass
};

// Flat item space over the instances of a launch: item i belongs to instance
// idx[k] for off[k] <= i < off[k+1] (off has K+1 entries).  The offsets of a
// space over grids are filled on the device (count_flat), so a kernel takes
// its loop bound from off[K] (flat_total); the `total` a launcher receives
// from the host only sizes the launch (an upper bound).
struct Flat {
    const long long* off;
    const int* idx;
    int K;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Position k in the flat space (largest k with off[k] <= i); off[0] = 0.
__device__ __forceinline__ int flat_find(const Flat& f, long long i) {
    int lo = 0, hi = f.K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(f.off + mid) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long flat_total(const Flat& f) { return __ldg(f.off + f.K); }

// Caches the instance range of the last item, so that a thread walking items
// of one instance does the binary search only when it crosses into another.
struct FlatCursor {
    int k = -1;
    long long lo = 0, hi = 0;
    // Returns true when the instance changed.
    __device__ __forceinline__ bool seek(const Flat& f, long long i) {
        if (i >= lo && i < hi) return false;
        k = flat_find(f, i);
        lo = __ldg(f.off + k);
        hi = __ldg(f.off + k + 1);
        return true;
    }
};

// Exact squared distance of two integer points (int32 coordinates, int64 sum).
template <int D>
__device__ __forceinline__ long long sqdist(const int* a, const int* b) {
    long long s = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        int t = a[j] - b[j];
        s += (long long)t * t;
    }
    return s;
}

// Inclusive warp scan of an int.
__device__ __forceinline__ int warp_inclusive_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

// Exclusive block scan of one int per thread (blockDim.x a multiple of 32,
// at most 1024).  `smem` holds 33 ints.  Returns the exclusive prefix;
// *total receives the block sum (all threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem, int* total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = warp_inclusive_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? smem[lane] : 0;
        int wi = warp_inclusive_scan(w);
        if (lane < nw) smem[lane] = wi - w;
        if (lane == 31) smem[32] = wi;
    }
    __syncthreads();
    int res = smem[warp] + inc - v;
    *total = smem[32];
    __syncthreads();
    return res;
}

// Linking priority of a union-find root: a bijective 32-bit mix of the index
// (the murmur3 finaliser), so distinct roots never tie.
__device__ __forceinline__ unsigned uf_priority(int x) {
    unsigned h = (unsigned)x;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Union-find root with path halving; -1 if the retry cap is reached.  Parents
// are read through L2 (other SMs link roots concurrently) and every halving
// store writes an ancestor, so concurrent finds and unions stay consistent.
// CAP: the loop bound is the run's (lowered) cap; otherwise the built-in
// constant, which keeps the loop the compiler's to schedule (a runtime bound
// measured about 30% slower in the merge).
template <bool CAP = false>
__device__ __forceinline__ int uf_find(int* parent, int x, int cap) {
    for (int it = 0; it < (CAP ? cap : kMaxUfRetries); ++it) {
        const int px = __ldcg(parent + x);
        if (px == x) return x;
        const int gp = __ldcg(parent + px);
        if (gp != px) __stcg(parent + x, gp);
        x = gp;
    }
    return -1;
}

// The root of x without writing anything.  Used where every grid's pointer
// must end at its root: a halving store by one thread can put back an older
// ancestor over the root another thread has just written.
template <bool CAP = false>
__device__ __forceinline__ int uf_find_ro(const int* parent, int x, int cap) {
    for (int it = 0; it < (CAP ? cap : kMaxUfRetries); ++it) {
        const int px = __ldcg(parent + x);
        if (px == x) return x;
        x = px;
    }
    return -1;
}

// The core points of grid c (rows of dp ints): a grid with at least MinPts
// points has only core points (G13 rule) and they stay in place in the
// grid-order coordinates Xs; the core points of other grids are packed in Xc
// from core_start[c].  Either way core_start[c+1] - core_start[c] rows.
__device__ __forceinline__ const int* core_rows(const Inst& I, int c, int dp) {
    const int b = I.cell_start[c];
    return I.cell_start[c + 1] - b >= I.p.minpts ? I.Xs + (long long)b * dp : I.Xc + (long long)I.core_start[c] * dp;
}

// Packed keys: the sort leaves the permutation in valA after an even number
// of passes, in valB after an odd number; the other one holds each point's
// in-cell offset word (input order) from quantisation to the compaction.
__device__ __forceinline__ int* in_cell_offsets(const Inst& I) { return (I.passes & 1) ? I.valA : I.valB; }

__device__ __forceinline__ void set_status(const Inst& I, unsigned bits) {
    atomicOr(reinterpret_cast<unsigned*>(I.small + kSmStatus), bits);
}

template <int D> struct Padded {
    static constexpr int value = D == 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
};

// Persistent grid size for grid-stride kernels.
constexpr int kPersistBlocks = 152 * 16;

// --------------------------------------------------- host-side launchers
// All launchers enqueue on `st` and return cudaGetLastError().  `ins` is the
// device array of Inst records; flat spaces are described by device offset
// tables built by the host (sizes known there) or by count_flat (sizes known
// only on the device).

// Host-side count of kernel launches issued by this thread (reported per run).
extern thread_local long long t_launches;
#define GD_COUNT_LAUNCH() (++::gd::t_launches)

// A segmented exclusive scan: segment k scans in[0..len) into out (in may
// equal out) and writes its total to out[len].  Segments are given by a
// device array of ScanSeg with blk0 = first flat tile of the segment.
struct ScanSeg {
    const int* in;
    int* out;
    long long len;        // the length, or (with len_dev) an upper bound of it
    long long blk0;       // first tile of the segment (tiles counted from len)
    int* tot;             // also receives the segment's total (out[len]), if not null
    const int* len_dev;   // if not null: the length, read on the device
};
__device__ __forceinline__ long long seg_len(const ScanSeg& sg) { return sg.len_dev ? *sg.len_dev : sg.len; }
constexpr int kScanTile = 2048;
// tmp: at least (total tiles + K) ints.  longest: the longest segment's
// length if known (segments of at most kScanOneLaunch elements are scanned
// by one block each in a single launch), else -1.
constexpr long long kScanOneLaunch = 1 << 16;
cudaError_t scan_segments(const ScanSeg* segs, int K, long long total_tiles, int* tmp, cudaStream_t st,
                          long long longest = -1);

// Device-side flat offsets: off[0] = 0, off[k+1] = off[k] + small[slot] of
// instance idx[k].
cudaError_t count_flat(const Inst* ins, const int* idx, int K, int slot, long long* off, cudaStream_t st);
// Several such flat spaces in one launch (one thread each).
struct FlatSpec {
    const int* idx;
    long long* off;
    int m;
    int slot;
};
cudaError_t count_flats(const Inst* ins, const FlatSpec* specs, int n, cudaStream_t st);
// The grid-key layout of each instance from its bounds (Eq. 1 identifiers
// packed, dimension 1 most significant): mn, bits, shift and key_bits in the
// device records.  The launch plan (key class, passes, digit bits) is the
// host's; a layout that does not fit it sets kDevReplan, a range too large
// kDevRange.
cudaError_t launch_layout(Inst* ins, int K, cudaStream_t st);

// Grid construction (grid.cu).
// Over the instances of dimension d.
cudaError_t launch_bounds(const Inst* ins, Flat pts, long long total, int d, cudaStream_t st);
constexpr int kCompactTile = 1024;
cudaError_t launch_compact_count(const Inst* ins, Flat tiles, long long total, int key_class, cudaStream_t st);
cudaError_t launch_compact_write(const Inst* ins, Flat tiles, long long total, int key_class, cudaStream_t st);
// Over the flat space of points.
cudaError_t launch_cell_max(const Inst* ins, Flat pts, long long total, cudaStream_t st);

// Identifiers and the radix sort (sort.cu).
struct SortPlan {
    int passes;   // digit positions
    int bits;     // bits per digit (<= 9)
    int buckets;  // 1 << bits
    int tile;     // keys per sort tile
    int tiles;
};
SortPlan sort_plan(int n, int key_words, int key_bits);
// ints of workspace for one instance's sort (tile histograms, digit totals
// and starts); layout in sort.cu.
size_t sort_tmp_ints(int n, int key_words, int key_bits);
void sort_tmp_layout(int* base, int n, int key_words, int key_bits, int** tcnt, int** ctot, int** dstart);
constexpr int kQuantTile = 4096;  // points per quantise block
// Keys (and, unpacked, index values) of every point, over quantisation tiles.
cudaError_t launch_quantise(const Inst* ins, Flat tiles, long long total, int key_class, cudaStream_t st);
// Sets the downsweep kernels' shared-memory limit on the current device (once
// per device; before any stream capture).
cudaError_t prepare_sort();
// One radix-sort pass (upsweep, tile scan, downsweep) of digit position
// `pass` over the sort tiles of the instances of one key class; `chunks` is
// the flat space of their tile-scan chunks (kSortChunk tiles each).  ev_a /
// ev_b, when set, are recorded just before and after the downsweep.
constexpr int kSortChunk = 32;
cudaError_t launch_sort_pass(const Inst* ins, Flat tiles, long long total, Flat chunks, long long chunk_total,
                             int key_class, int pass, int max_buckets, cudaStream_t st, cudaEvent_t ev_a = nullptr,
                             cudaEvent_t ev_b = nullptr);
// Records ev on st; inside a stream capture, as an external graph node.
void record_event(cudaEvent_t ev, cudaStream_t st);

// Grid-tree levels and neighbour walk (neighbors.cu).
cudaError_t launch_point_boxes(const Inst* ins, Flat cells, long long total, cudaStream_t st);
cudaError_t launch_level_diff(const Inst* ins, Flat cells, long long total, cudaStream_t st);
cudaError_t launch_level_flag(const Inst* ins, Flat cells, long long total, int level, cudaStream_t st);
cudaError_t launch_level_write(const Inst* ins, Flat cells, long long total, cudaStream_t st);
// Single-pass neighbour walk: the walk counts and, in the same pass, appends
// each query's neighbours to a pool in runs of at most kPoolRun (segments;
// long runs keep the shared counter's atomics few); after
// the counts are scanned, the segments are scattered into the lists.  One
// 64-bit counter hands out both: pool entries in its low kPoolBits bits,
// segments above them.  A pool that overflows is discarded (the lists are then
// filled by a second walk).
constexpr int kPoolBits = 37;
constexpr int kPoolRun = 96;
struct PoolSeg {
    long long pos;  // first pool entry
    int inst;       // instance (index into the Inst array)
    int c;          // query grid
    int off;        // offset of the run in the grid's list
    int len;        // 1..kPoolRun
};
struct WalkPool {
    int* data;
    PoolSeg* seg;
    unsigned long long* ctr;
    long long cap, seg_cap;
};
enum WalkMode { kWalkCount = 0, kWalkFill = 1, kWalkPool = 2 };
cudaError_t launch_walk(const Inst* ins, Flat cells, long long total, int mode, WalkPool pool, int blocks,
                        bool small_eps, int d, cudaStream_t st);
// The pool's runs into the lists (nothing when the pool overflowed; the
// filling walk, kWalkFill, runs only then -- or always without a pool).
cudaError_t launch_pool_scatter(const Inst* ins, WalkPool pool, cudaStream_t st);
// Lists whose total exceeds the instance's nbr_cap are given up (emptied,
// kDevOverflow).
cudaError_t launch_nbr_check(const Inst* ins, Flat cells, long long total, cudaStream_t st);
// After a counting or pooled walk: nbr_start[c] = forward + backward entries
// (scanned next), backward counts reset to serve as placement cursors.
cudaError_t launch_nbr_total(const Inst* ins, Flat cells, long long total, cudaStream_t st);

// Core points (core.cu).
cudaError_t launch_core_full(const Inst* ins, Flat cells, long long total, cudaStream_t st);
cudaError_t launch_nf_index(const Inst* ins, Flat cells, long long total, cudaStream_t st);
cudaError_t launch_nonfull_count(const Inst* ins, Flat cells, long long total, cudaStream_t st);
// Statistics only: non-full points and the rows a per-grid count would stage.
cudaError_t launch_core_stats(const Inst* ins, Flat cells, long long total, cudaStream_t st);
// Non-full points of instances with dimension d (flat offsets on the device).
cudaError_t launch_core_point(const Inst* ins, Flat nf_pts, int d, int band_limit, cudaStream_t st);
// Non-full grids of instances with dimension d, one warp per grid (the grids
// of `cells`; full grids are skipped).
cudaError_t launch_core_grid(const Inst* ins, Flat cells, long long total, int d, int band_limit, cudaStream_t st);

// Merging (merge.cu).
cudaError_t launch_core_count(const Inst* ins, Flat cells, long long total, cudaStream_t st);
// Core points of non-full grids packed, and every grid's core box, a thread
// per grid of `cells` (the instances of dimension d).
cudaError_t launch_core_pack(const Inst* ins, Flat cells, long long total, int d, cudaStream_t st);
// Low-density-first order of the grids (instances with p.ldf set): core
// grids by ascending core-point count (buckets: exact counts below 64, then
// powers of two), non-core grids last.
constexpr int kLdfBuckets = 128;
cudaError_t launch_ldf_order(const Inst* ins, const int* idx, int K, Flat cells, long long total, cudaStream_t st);

cudaError_t launch_uf_init(const Inst* ins, Flat cells, long long total, cudaStream_t st);
cudaError_t launch_uf_flatten(const Inst* ins, Flat cells, long long total, bool cap, cudaStream_t st);
// Warp-level test of the candidate pairs of one wave (touching order: 0 =
// touching pairs, 1 = the others; LDF order: wave 0 only), taken from the
// neighbour lists of the grids of `cells` (instances of dimension d);
// undecided pairs go to the instance's hard list.
// (cap: the union-find loops take the run's lowered cap, Params::uf_cap.)
cudaError_t launch_merge_list(const Inst* ins, Flat cells, long long total, int wave, int d, int budget,
                              int lane_limit, int small_set, bool cap, cudaStream_t st);
// FastMerging (Alg. 5) of the hard pairs of one wave: `blocks` blocks, block b
// using the 2 * wpb bitmap words at scratch + 2 * wpb * b (wpb >= the largest
// grid of the batch / 32 + 1).
cudaError_t launch_merge_block(const Inst* ins, Flat hard, int wave, int d, int blocks, unsigned* scratch, int wpb,
                               bool cap, cudaStream_t st);

// Labels (label.cu).
cudaError_t launch_cluster_ids(const Inst* ins, Flat cells, long long total, bool cap, cudaStream_t st);
cudaError_t launch_labels(const Inst* ins, Flat pts, long long total, int d, cudaStream_t st);

}  // namespace gd
