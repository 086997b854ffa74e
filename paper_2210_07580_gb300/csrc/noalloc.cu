// gd_dbscan_noalloc: the exact-DBSCAN pipeline with every scratch buffer taken
// from one fixed, statically sized device array instead of cudaMalloc.
//
// Some callers cannot allocate device memory at the time they need a
// clustering: code running under a memory manager that owns the whole device
// pool, a plugin in a host application that forbids allocations on its hot
// path, or a process whose allocator is already exhausted.  This entry point
// serves them for small inputs (at most GD_NOALLOC_MAX_POINTS points): it
// calls no cudaMalloc, cudaFree, cudaMallocHost or any other allocating
// routine.  It runs the same kernels as gd_dbscan, so its labels equal
// gd_dbscan's bit for bit.
//
// The scratch array below (GD_NOALLOC_SCRATCH_BYTES) exists on every GPU that
// loads this library, for as long as the library stays loaded.
#include <climits>
#include <cstring>
#include <mutex>

#include "gd_internal.cuh"
#include "gdbscan.h"

using namespace gd;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;                  // serialises host callers (they share the array)
void* g_scratch_addr[kMaxDevices];   // device address of the array, per device

int dp_of(int d) { return d == 1 ? 1 : d == 2 ? 2 : d <= 4 ? 4 : 8; }

unsigned long long isqrt64(unsigned long long v) {
    unsigned long long lo = 0, hi = 1ull << 32;
    while (hi - lo > 1) {
        const unsigned long long mid = lo + (hi - lo) / 2;
        if ((unsigned __int128)mid * mid <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Bump allocator over the static array (no device allocation involved).
struct Bump {
    char* base;
    size_t cap, off;
    void* take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        if (off + bytes > cap) return nullptr;
        void* p = base + off;
        off += bytes;
        return p;
    }
};

// There is no context to hold an error message: failures are reported by
// status code only (GD_ECUDA for a failed CUDA call, GD_ENOMEM when the input
// needs more than the static array holds).
#define NA_CUDA(call)                                \
    do {                                             \
        if ((call) != cudaSuccess) return GD_ECUDA;  \
    } while (0)

#define NA_TAKE(ptr, type, bytes)                    \
    do {                                             \
        ptr = (type)bump.take(bytes);                \
        if (!ptr) return GD_ENOMEM;                  \
    } while (0)

// Copy `count` ints from the device into a host array and wait (a pageable
// destination: no pinned staging buffer is allocated).
gd_status fetch(int* host, const int* dev, int count, cudaStream_t st) {
    NA_CUDA(cudaMemcpyAsync(host, dev, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    return GD_OK;
}

#define NA_TRY(call)                  \
    do {                              \
        gd_status s_ = (call);        \
        if (s_ != GD_OK) return s_;   \
    } while (0)

gd_status run_noalloc(char* base, const int32_t* X, int n, int d, long long eps2, int minpts, int32_t* labels,
                      uint8_t* is_core, cudaStream_t st) {
    Bump bump{base, (size_t)GD_NOALLOC_SCRATCH_BYTES, 0};
    int* small;
    NA_TAKE(small, int*, 64 * sizeof(int));
    int* mnmx = small;
    int* num_cells = small + 16;
    unsigned* status = (unsigned*)(small + 17);
    int* max_cell = small + 18;
    int* level_count = small + 24;
    int* mrange = small + 32;
    int* hard_cnt = small + 36;
    int host[64];

    Params p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.d = d;
    p.dp = dp_of(d);
    const long long cap = (1ll << 62) - 1;
    p.eps2 = eps2 > cap ? cap : eps2;
    p.minpts = minpts;
    p.s = 1 + (long long)isqrt64((unsigned long long)p.eps2 / (unsigned long long)d);
    p.r = p.eps2 == 0 ? 0 : 1 + ((long long)isqrt64((unsigned long long)p.eps2) - 1) / p.s;

    NA_CUDA(launch_init_bounds(mnmx, st));
    NA_CUDA(launch_bounds(X, n, d, mnmx, st));
    NA_TRY(fetch(host, mnmx, 16, st));
    unsigned long long rmax = 0;
    int total_bits = 0;
    for (int j = 0; j < d; ++j) {
        const long long lo = host[j], hi = host[kMaxD + j];
        const unsigned long long rj = (unsigned long long)(hi - lo);
        if (rj > rmax) rmax = rj;
        p.mn[j] = (int)lo;
        int b = 0;
        for (unsigned long long v = rj / (unsigned long long)p.s; v; v >>= 1) b++;
        p.bits[j] = b;
        total_bits += b;
    }
    if ((unsigned __int128)d * rmax * rmax >= ((unsigned __int128)1 << 62))
        return GD_ERANGE;
    if (total_bits > 128) return GD_ERANGE;
    for (int j = d - 1, sh = 0; j >= 0; --j) {
        p.shift[j] = sh;
        sh += p.bits[j];
    }
    p.key_bits = total_bits;
    p.key_words = total_bits <= 64 ? 1 : 2;

    // fixed buffers, sized for this n and d
    const size_t N = (size_t)n;
    void *keyA, *keyB;
    int *valA, *valB, *Xs, *pt_cell, *Xc, *cell_start, *cell_coord, *nbr_start, *core_start, *bbox, *pair_start,
        *pair_start_f, *parent, *cid_root, *cell_cid, *tmp;
    unsigned char* core_s;
    NA_TAKE(keyA, void*, N * 8 * p.key_words);
    NA_TAKE(keyB, void*, N * 8 * p.key_words);
    NA_TAKE(valA, int*, N * 4);
    NA_TAKE(valB, int*, N * 4);
    NA_TAKE(Xs, int*, N * p.dp * 4);
    NA_TAKE(pt_cell, int*, N * 4);
    NA_TAKE(core_s, unsigned char*, N);
    NA_TAKE(Xc, int*, N * p.dp * 4);
    NA_TAKE(cell_start, int*, (N + 1) * 4);
    NA_TAKE(cell_coord, int*, N * d * 4);
    Levels lv;
    for (int j = 0; j < kMaxD; ++j) {
        lv.key[j] = nullptr;
        lv.child_begin[j] = nullptr;
        if (j < d) NA_TAKE(lv.key[j], int*, (N + 1) * 4);
        if (j < d - 1) NA_TAKE(lv.child_begin[j], int*, (N + 2) * 4);
    }
    lv.count = level_count;
    NA_TAKE(nbr_start, int*, (N + 1) * 4);
    NA_TAKE(core_start, int*, (N + 1) * 4);
    NA_TAKE(bbox, int*, N * 2 * d * 4);
    NA_TAKE(pair_start, int*, (N + 1) * 4);
    NA_TAKE(pair_start_f, int*, (N + 1) * 4);
    NA_TAKE(parent, int*, N * 4);
    NA_TAKE(cid_root, int*, N * 4);
    NA_TAKE(cell_cid, int*, N * 4);
    size_t t = radix_tmp_ints(n, p.key_words, p.key_bits);
    if (compact_tmp_ints(n) > t) t = compact_tmp_ints(n);
    if (levels_tmp_ints(n, d) > t) t = levels_tmp_ints(n, d);
    if (scan_tmp_ints((long long)n + 1) > t) t = scan_tmp_ints((long long)n + 1);
    NA_TAKE(tmp, int*, t * 4);

    // the status word starts at zero on every call (the array keeps old contents)
    NA_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    int in_b = 0;
    NA_CUDA(quantise_hist(X, p, keyA, valA, tmp, st));
    NA_CUDA(sort_passes(p, keyA, valA, keyB, valB, tmp, status, st, &in_b));
    void* keys = in_b ? keyB : keyA;
    int* perm = in_b ? valB : valA;
    NA_CUDA(launch_compact(p, X, keys, perm, tmp, cell_start, cell_coord, pt_cell, Xs, num_cells, st));
    NA_TRY(fetch(host, num_cells, 1, st));
    const int C = host[0];
    NA_CUDA(launch_cell_max(cell_start, C, max_cell, st));

    NA_CUDA(build_levels(p, cell_coord, C, lv, tmp, st));
    NA_CUDA(launch_walk_count(p, cell_coord, C, lv, nbr_start, st));
    NA_CUDA(scan_exclusive(nbr_start, nbr_start, C, tmp, st));
    NA_TRY(fetch(host, nbr_start + C, 1, st));
    const long long nnbr = (unsigned)host[0];
    NA_TRY(fetch(host, max_cell, 1, st));
    const int wpb = (host[0] + 31) / 32 + 1;
    int* nbr;
    int2 *pairs, *hard;
    unsigned* mscratch;
    NA_TAKE(nbr, int*, (size_t)nnbr * 4 + 16);
    NA_TAKE(pairs, int2*, (size_t)nnbr * 8 + 16);
    NA_TAKE(hard, int2*, (size_t)nnbr * 8 + 16);
    const int fm_blocks = 152;  // fewer FastMerging blocks: their bitmaps come out of the static array
    NA_TAKE(mscratch, unsigned*, (size_t)fm_blocks * 2 * wpb * 4);
    NA_CUDA(launch_walk_fill(p, cell_coord, C, lv, nbr_start, nbr, st));

    NA_CUDA(launch_core(p, Xs, cell_start, pt_cell, cell_coord, C, nbr_start, nbr, pair_start, tmp, core_s, st));
    NA_CUDA(launch_core_count(p, core_s, cell_start, C, core_start, bbox, st));
    NA_CUDA(scan_exclusive(core_start, core_start, C, tmp, st));
    NA_CUDA(launch_core_pack(p, Xs, core_s, pt_cell, cell_start, core_start, Xc, bbox, st));
    NA_CUDA(launch_pair_count(p, nbr_start, nbr, core_start, cell_coord, C, pair_start, pair_start_f, st));
    NA_CUDA(scan_exclusive(pair_start, pair_start, C, tmp, st));
    NA_CUDA(scan_exclusive(pair_start_f, pair_start_f, C, tmp, st));
    NA_CUDA(launch_pair_fill(p, nbr_start, nbr, core_start, cell_coord, C, pair_start, pair_start_f, pairs, st));

    NA_CUDA(launch_uf_init(parent, C, st));
    NA_CUDA(launch_merge_ranges(pair_start, pair_start_f, C, mrange, hard_cnt, st));
    for (int wave = 0; wave < 2; ++wave) {
        NA_CUDA(launch_merge_wave(p, wave, pairs, mrange, (int)nnbr, Xc, core_start, bbox, parent, status, hard,
                                  hard_cnt, mscratch, wpb, fm_blocks, st));
        if (wave == 0) NA_CUDA(launch_uf_flatten(parent, C, status, st));
    }
    NA_CUDA(launch_cluster_ids(p, parent, core_start, cell_start, core_s, perm, C, cid_root, cell_cid, st, status));
    NA_CUDA(launch_labels(p, Xs, cell_start, pt_cell, core_s, nbr_start, nbr, core_start, Xc, bbox, cell_cid, perm,
                          labels, is_core, st));
    NA_TRY(fetch(host, (const int*)status, 1, st));
    if ((unsigned)host[0] & kDevTimeout) return GD_ETIMEOUT;
    return GD_OK;
}

}  // namespace

extern "C" gd_status gd_dbscan_noalloc(const int32_t* X, int64_t n, int d, int64_t eps2, int32_t minpts,
                                       int32_t* labels, uint8_t* is_core, gd_stream_t stream) {
    if (d < 1 || d > kMaxD) return GD_EINVAL;
    if (n < 0) return GD_EINVAL;
    if (n > GD_NOALLOC_MAX_POINTS) return GD_ENOMEM;
    if (eps2 < 0) return GD_EINVAL;
    if (minpts < 1) return GD_EINVAL;
    if (n > 0 && (!X || !labels)) return GD_EINVAL;
    if (n == 0) return GD_OK;

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return GD_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GD_EINVAL;
    if (!g_scratch_addr[dev]) {
        // First call on this device (which is current): look up the device
        // address of the static array.  The host-side symbol is only a
        // stand-in and must never be handed to a kernel.
        void* addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr)
            return GD_ECUDA;
        g_scratch_addr[dev] = addr;
    }
    return run_noalloc((char*)g_scratch_addr[dev], X, (int)n, d, eps2, minpts, labels, is_core,
                       (cudaStream_t)stream);
}
