// Internal declarations shared by the CUDA translation units of libgdbscan.
//
// Pipeline (one DBSCAN instance, all arrays device-resident):
//   bounds -> quantise/pack keys (Eq. 1) -> LSD radix sort (Alg. 1)
//   -> grid compaction + coordinate gather (Alg. 1) -> grid-tree levels (Alg. 2)
//   -> neighbour-grid walk (Alg. 3) -> core points (G13 rule, Section 3.2)
//   -> core-point compaction -> core-grid merge (Def. 6-7, Alg. 4-5) with
//   union-find (LDF variant, Section 5.2) -> cluster ids -> border + labels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gd {

constexpr int kMaxD = 8;
constexpr unsigned kFull = 0xffffffffu;

// Bits of the device status word (OR-ed by kernels, read by the host).
enum : unsigned { kDevTimeout = 1u, kDevOverflow = 2u };

// Retry cap for the lock-free union-find loops: far above any legitimate
// number of CAS retries, so reaching it means something is wrong; the kernel
// then records kDevTimeout and gives up instead of spinning.
constexpr int kMaxUfRetries = 1 << 20;

// Per-instance parameters, fixed once the bounds are known.
struct Params {
    int n;            // points
    int d;            // dimensions (1..8)
    int dp;           // padded row stride of the grid-order coordinates (1,2,4,8)
    long long eps2;   // squared radius
    int minpts;
    long long s;      // integer cell side: largest s with d*(s-1)^2 <= eps2
    long long r;      // largest |delta| per dimension whose gap alone is <= eps
    int key_bits;     // total bits of the packed grid key
    int key_words;    // 1 or 2 64-bit words
    int mn[kMaxD];    // per-dimension minimum coordinate
    int bits[kMaxD];  // bits of each identifier in the key
    int shift[kMaxD]; // bit offset of identifier j (dimension 0 most significant)
};

// 128-bit grid key for identifiers wider than 64 bits in total.
struct Key2 {
    unsigned long long lo, hi;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

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
__device__ __forceinline__ int uf_find(int* parent, int x) {
    for (int it = 0; it < kMaxUfRetries; ++it) {
        const int px = __ldcg(parent + x);
        if (px == x) return x;
        const int gp = __ldcg(parent + px);
        if (gp != px) __stcg(parent + x, gp);
        x = gp;
    }
    return -1;
}

// --------------------------------------------------- host-side launchers
// All launchers enqueue on `st` and return cudaGetLastError().

// Host-side count of kernel launches issued by this thread (reported per run).
extern thread_local long long t_launches;
#define GD_COUNT_LAUNCH() (++::gd::t_launches)

// Device-wide exclusive scan of n ints (in may equal out); out[n] = total.
// tmp must hold scan_tmp_ints(n) ints.
size_t scan_tmp_ints(long long n);
cudaError_t scan_exclusive(const int* in, int* out, long long n, int* tmp, cudaStream_t st);

// Grid construction (grid.cu).
cudaError_t launch_init_bounds(int* mnmx, cudaStream_t st);
cudaError_t launch_bounds(const int* X, int n, int d, int* mnmx, cudaStream_t st);
// Identifiers and the radix sort (sort.cu).
struct SortPlan {
    int passes;   // digit positions
    int bits;     // bits per digit (<= 9)
    int buckets;  // 1 << bits
    int tile;     // keys per onesweep tile
    int tiles;
};
SortPlan sort_plan(int n, int key_words, int key_bits);
size_t radix_tmp_ints(int n, int key_words, int key_bits);
// Computes the keys (Eq. 1, packed) and values (input index) into keys_a /
// vals_a, with the histogram of every digit position (into tmp).
cudaError_t quantise_hist(const int* X, const Params& p, void* keys_a, int* vals_a, int* tmp, cudaStream_t st);
// The onesweep passes: sorts (keys_a, vals_a) stably by key; *result_in_b
// tells which buffer pair holds the result.  err receives kDevTimeout if a
// look-back gave up.  tmp must still hold what quantise_hist left there.
cudaError_t sort_passes(const Params& p, void* keys_a, int* vals_a, void* keys_b, int* vals_b, int* tmp, unsigned* err,
                        cudaStream_t st, int* result_in_b);
size_t compact_tmp_ints(int n);
cudaError_t launch_compact(const Params& p, const int* X, const void* keys, const int* vals, int* tmp,
                           int* cell_start, int* cell_coord, int* pt_cell, int* Xs, int* num_cells,
                           cudaStream_t st);

// Grid-tree levels and neighbour walk (neighbors.cu).
struct Levels {
    int* key[kMaxD];          // level j: identifier j of each node
    int* child_begin[kMaxD];  // level j < d-1: first child at level j+1 ([N_j + 1])
    int* count;               // [kMaxD] node counts per level (device)
};
size_t levels_tmp_ints(int C, int d);
cudaError_t build_levels(const Params& p, const int* cell_coord, int C, Levels lv, int* tmp, cudaStream_t st);
cudaError_t launch_walk_count(const Params& p, const int* cell_coord, int C, Levels lv, int* nbr_count,
                              cudaStream_t st);
cudaError_t launch_walk_fill(const Params& p, const int* cell_coord, int C, Levels lv, const int* nbr_start,
                             int* nbr, cudaStream_t st);

// Core points (core.cu).
// nf_start: C+1 ints of workspace (points of non-full grids, scanned).
cudaError_t launch_core(const Params& p, const int* Xs, const int* cell_start, const int* pt_cell,
                        const int* cell_coord, int C, const int* nbr_start, const int* nbr, int* nf_start, int* tmp,
                        unsigned char* core_s, cudaStream_t st);

// Merging (merge.cu).
cudaError_t launch_core_count(const Params& p, const unsigned char* core_s, const int* cell_start, int C,
                              int* core_cnt, int* bbox, cudaStream_t st);
cudaError_t launch_core_pack(const Params& p, const int* Xs, const unsigned char* core_s, const int* pt_cell,
                             const int* cell_start, const int* core_start, int* Xc, int* bbox, cudaStream_t st);
cudaError_t launch_cell_max(const int* cell_start, int C, int* out, cudaStream_t st);
cudaError_t launch_pair_count(const Params& p, const int* nbr_start, const int* nbr, const int* core_start,
                              const int* cell_coord, int C, int* t_count, int* f_count, cudaStream_t st);
cudaError_t launch_pair_fill(const Params& p, const int* nbr_start, const int* nbr, const int* core_start,
                             const int* cell_coord, int C, const int* t_start, const int* f_start, int2* pairs,
                             cudaStream_t st);
cudaError_t launch_merge_ranges(const int* t_start, const int* f_start, int C, int* range, int* hard_cnt,
                                cudaStream_t st);
cudaError_t launch_uf_init(int* parent, int C, cudaStream_t st);
// Points every grid at its union-find root (no unions may run concurrently).
cudaError_t launch_uf_flatten(int* parent, int C, unsigned* status, cudaStream_t st);
// Default number of FastMerging blocks; each block owns 2 * wpb words of
// `scratch`, wpb = ceil(largest grid / 32) + 1.
int merge_fm_blocks();
// One merge wave (0: touching pairs, 1: the others): warp-level test of every
// pair in range[2*wave .. 2*wave+1], then FastMerging of the pairs it hands on.
cudaError_t launch_merge_wave(const Params& p, int wave, const int2* pairs, const int* range, int max_pairs,
                              const int* Xc, const int* core_start, const int* bbox, int* parent, unsigned* status,
                              int2* hard, int* hard_cnt, unsigned* scratch, int wpb, int fm_blocks,
                              cudaStream_t st);

// Labels (label.cu).
cudaError_t launch_cluster_ids(const Params& p, int* parent, const int* core_start, const int* cell_start,
                               const unsigned char* core_s, const int* perm, int C, int* cid_root,
                               int* cell_cid, cudaStream_t st, unsigned* status);
cudaError_t launch_labels(const Params& p, const int* Xs, const int* cell_start, const int* pt_cell,
                          const unsigned char* core_s, const int* nbr_start, const int* nbr,
                          const int* core_start, const int* Xc, const int* bbox, const int* cell_cid,
                          const int* perm, int* labels, unsigned char* is_core, cudaStream_t st);

}  // namespace gd
