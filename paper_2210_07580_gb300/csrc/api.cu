// C ABI of libgdbscan: context, workspace and the stage sequence of one
// exact DBSCAN run (Alg. 6 as a sequence of device stages).
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "gd_internal.cuh"
#include "gdbscan.h"

using namespace gd;

namespace gd {
thread_local long long t_launches = 0;
}

namespace {

constexpr int kStages = 11;
const char* const kStageNames[kStages] = {"bounds", "quantise", "sort",  "compact", "levels", "walk",
                                          "core",   "core_pack", "pairs", "merge",   "labels"};

// Small device block: mnmx[16], then scalar counters.
enum SmallSlot {
    kMnmx = 0,        // [16] per-dimension min then max
    kNumCells = 16,   // C
    kStatus = 17,     // device status bits
    kMaxCell = 18,    // largest grid
    kLevelCount = 24, // [8] nodes per grid-tree level
    kRange = 32,      // [4] merge wave ranges
    kHardCnt = 36,    // [2] pairs handed to FastMerging per wave
    kSmallInts = 64
};

struct Work {
    void* keyA;
    void* keyB;
    int* valA;
    int* valB;
    int* Xs;
    int* pt_cell;
    unsigned char* core_s;
    int* Xc;
    int* cell_start;
    int* cell_coord;
    int* lv_key[kMaxD];
    int* lv_cb[kMaxD];
    int* nbr_start;
    int* core_start;
    int* bbox;
    int* pair_start;
    int* pair_start_f;
    int* parent;
    int* cid_root;
    int* cell_cid;
    int* tmp;
};

int padded_dim(int d) { return d == 1 ? 1 : d == 2 ? 2 : d <= 4 ? 4 : 8; }

// Lay the fixed workspace out from `base` (or only size it when base is
// null).  Arrays indexed by grid are sized for n grids, the upper bound.
size_t carve(Work* w, char* base, int64_t n, int d, int key_words, int key_bits) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + 255) & ~(size_t)255;
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t N = (size_t)n, dp = (size_t)padded_dim(d);
    w->keyA = take(N * 8 * key_words);
    w->keyB = take(N * 8 * key_words);
    w->valA = (int*)take(N * 4);
    w->valB = (int*)take(N * 4);
    w->Xs = (int*)take(N * dp * 4);
    w->pt_cell = (int*)take(N * 4);
    w->core_s = (unsigned char*)take(N);
    w->Xc = (int*)take(N * dp * 4);
    w->cell_start = (int*)take((N + 1) * 4);
    w->cell_coord = (int*)take(N * d * 4);
    for (int j = 0; j < kMaxD; ++j) {
        w->lv_key[j] = j < d ? (int*)take((N + 1) * 4) : nullptr;
        w->lv_cb[j] = j < d - 1 ? (int*)take((N + 2) * 4) : nullptr;
    }
    w->nbr_start = (int*)take((N + 1) * 4);
    w->core_start = (int*)take((N + 1) * 4);
    w->bbox = (int*)take(N * 2 * d * 4);
    w->pair_start = (int*)take((N + 1) * 4);
    w->pair_start_f = (int*)take((N + 1) * 4);
    w->parent = (int*)take(N * 4);
    w->cid_root = (int*)take(N * 4);
    w->cell_cid = (int*)take(N * 4);
    size_t t = radix_tmp_ints((int)n, key_words, key_bits);
    t = t > compact_tmp_ints((int)n) ? t : compact_tmp_ints((int)n);
    t = t > levels_tmp_ints((int)n, d) ? t : levels_tmp_ints((int)n, d);
    t = t > scan_tmp_ints(n + 1) ? t : scan_tmp_ints(n + 1);
    w->tmp = (int*)take(t * 4);
    return off + 256;
}

unsigned long long isqrt_u64(unsigned long long v) {
    // largest r with r*r <= v, by bisection on r
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

int bit_length(unsigned long long v) {
    int b = 0;
    while (v) {
        b++;
        v >>= 1;
    }
    return b;
}

struct DevBuf {
    char* ptr = nullptr;
    size_t cap = 0;
};

}  // namespace

struct gd_ctx {
    int device = 0;
    DevBuf arena, nbr, pairs, hard, mscratch, io;
    int* small = nullptr;       // device
    int* host_small = nullptr;  // pinned host mirror
    cudaEvent_t ev[kStages + 1] = {};
    bool timing = false;
    float stage_ms[kStages] = {};
    int nstages = 0;
    std::string err;
    bool have_run = false;
    int64_t sizes[12] = {};
    const void* view_ptr[7] = {};
    size_t view_bytes[7] = {};
};

namespace {

gd_status fail(gd_ctx* ctx, gd_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

gd_status cuda_fail(gd_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, GD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GD_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Grow a device buffer to at least `bytes` (contents are not kept).
gd_status ensure(gd_ctx* ctx, DevBuf& b, size_t bytes, cudaStream_t st) {
    if (b.cap >= bytes) return GD_OK;
    if (b.ptr) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 8 + (1 << 20);
    cudaError_t e = cudaMalloc((void**)&b.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        return fail(ctx, GD_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    b.cap = want;
    return GD_OK;
}

gd_status readback(gd_ctx* ctx, const int* dev, int count, cudaStream_t st) {
    GD_CUDA(cudaMemcpyAsync(ctx->host_small, dev, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
    GD_CUDA(cudaStreamSynchronize(st));
    return GD_OK;
}

gd_status validate(gd_ctx* ctx, const void* X, int64_t n, int d, int64_t eps2, int32_t minpts, const void* labels) {
    if (!ctx) return GD_EINVAL;
    if (d < 1 || d > kMaxD) return fail(ctx, GD_EINVAL, "d must be in [1, 8]");
    if (n < 0 || n >= (int64_t)INT_MAX) return fail(ctx, GD_EINVAL, "n must be in [0, 2^31 - 1)");
    if (eps2 < 0) return fail(ctx, GD_EINVAL, "eps2 must be >= 0");
    if (minpts < 1) return fail(ctx, GD_EINVAL, "minpts must be >= 1");
    if (n > 0 && (!X || !labels)) return fail(ctx, GD_EINVAL, "null pointer with n > 0");
    return GD_OK;
}

#define GD_TRY(call)                      \
    do {                                  \
        gd_status s_ = (call);            \
        if (s_ != GD_OK) return s_;       \
    } while (0)

gd_status run(gd_ctx* ctx, const int32_t* X, int64_t n64, int d, int64_t eps2, int32_t minpts, int32_t* labels,
              uint8_t* is_core, cudaStream_t st) {
    const int n = (int)n64;
    ctx->have_run = false;
    const long long launches0 = t_launches;
    auto mark = [&](int stage) {
        if (ctx->timing) cudaEventRecord(ctx->ev[stage], st);
    };

    Params p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.d = d;
    p.dp = padded_dim(d);
    // Every squared distance is below 2^62 once the range check passes, so a
    // larger eps2 changes nothing; clamping keeps the gap sums in range.
    const long long kEpsCap = (1ll << 62) - 1;
    p.eps2 = eps2 > kEpsCap ? kEpsCap : eps2;
    p.minpts = minpts;
    p.s = 1 + (long long)isqrt_u64((unsigned long long)p.eps2 / (unsigned long long)d);
    p.r = p.eps2 == 0 ? 0 : 1 + ((long long)isqrt_u64((unsigned long long)p.eps2) - 1) / p.s;

    // --- bounds (mn_j of Eq. 1) and the range check
    mark(0);
    GD_CUDA(launch_init_bounds(ctx->small + kMnmx, st));
    GD_CUDA(launch_bounds(X, n, d, ctx->small + kMnmx, st));
    GD_TRY(readback(ctx, ctx->small, kSmallInts, st));
    unsigned long long rmax = 0;
    int total_bits = 0;
    for (int j = 0; j < d; ++j) {
        const long long lo = ctx->host_small[kMnmx + j], hi = ctx->host_small[kMnmx + kMaxD + j];
        const unsigned long long rj = (unsigned long long)(hi - lo);
        if (rj > rmax) rmax = rj;
        p.mn[j] = (int)lo;
        p.bits[j] = bit_length(rj / (unsigned long long)p.s);
        total_bits += p.bits[j];
    }
    if ((unsigned __int128)d * rmax * rmax >= ((unsigned __int128)1 << 62))
        return fail(ctx, GD_ERANGE, "coordinate range too large: d * R^2 >= 2^62");
    if (total_bits > 128) return fail(ctx, GD_ERANGE, "packed grid key needs more than 128 bits");
    {
        int sh = 0;
        for (int j = d - 1; j >= 0; --j) {
            p.shift[j] = sh;
            sh += p.bits[j];
        }
    }
    p.key_bits = total_bits;
    p.key_words = total_bits <= 64 ? 1 : 2;

    Work w;
    const size_t need = carve(&w, nullptr, n, d, p.key_words, p.key_bits);
    GD_TRY(ensure(ctx, ctx->arena, need, st));
    carve(&w, ctx->arena.ptr, n, d, p.key_words, p.key_bits);

    // --- identifiers (Eq. 1) with digit histograms, then the sort (Alg. 1)
    mark(1);
    GD_CUDA(cudaMemsetAsync(ctx->small + kStatus, 0, sizeof(int), st));
    GD_CUDA(quantise_hist(X, p, w.keyA, w.valA, w.tmp, st));
    mark(2);
    int in_b = 0;
    GD_CUDA(sort_passes(p, w.keyA, w.valA, w.keyB, w.valB, w.tmp, (unsigned*)(ctx->small + kStatus), st, &in_b));
    void* keys = in_b ? w.keyB : w.keyA;
    int* perm = in_b ? w.valB : w.valA;

    // --- non-empty grids (Alg. 1)
    mark(3);
    GD_CUDA(launch_compact(p, X, keys, perm, w.tmp, w.cell_start, w.cell_coord, w.pt_cell, w.Xs,
                           ctx->small + kNumCells, st));
    GD_TRY(readback(ctx, ctx->small + kNumCells, 1, st));
    const int C = ctx->host_small[0];
    GD_CUDA(launch_cell_max(w.cell_start, C, ctx->small + kMaxCell, st));

    // --- grid tree levels (Alg. 2) and Nei(g) (Alg. 3)
    mark(4);
    Levels lv;
    for (int j = 0; j < kMaxD; ++j) {
        lv.key[j] = w.lv_key[j];
        lv.child_begin[j] = w.lv_cb[j];
    }
    lv.count = ctx->small + kLevelCount;
    GD_CUDA(build_levels(p, w.cell_coord, C, lv, w.tmp, st));
    mark(5);
    GD_CUDA(launch_walk_count(p, w.cell_coord, C, lv, w.nbr_start, st));
    GD_CUDA(scan_exclusive(w.nbr_start, w.nbr_start, C, w.tmp, st));
    GD_TRY(readback(ctx, w.nbr_start + C, 1, st));
    const long long nnbr = (unsigned)ctx->host_small[0];
    if (nnbr >= INT_MAX) return fail(ctx, GD_ERANGE, "neighbour lists exceed 2^31 entries");
    GD_TRY(ensure(ctx, ctx->nbr, (size_t)nnbr * 4 + 16, st));
    int* nbr = (int*)ctx->nbr.ptr;
    GD_CUDA(launch_walk_fill(p, w.cell_coord, C, lv, w.nbr_start, nbr, st));

    // --- core points (G13 rule)
    mark(6);
    GD_CUDA(launch_core(p, w.Xs, w.cell_start, w.pt_cell, w.cell_coord, C, w.nbr_start, nbr, w.pair_start, w.tmp,
                        w.core_s, st));

    // --- core point sets s_i and their boxes
    mark(7);
    GD_CUDA(launch_core_count(p, w.core_s, w.cell_start, C, w.core_start, w.bbox, st));
    GD_CUDA(scan_exclusive(w.core_start, w.core_start, C, w.tmp, st));
    GD_CUDA(launch_core_pack(p, w.Xs, w.core_s, w.pt_cell, w.cell_start, w.core_start, w.Xc, w.bbox, st));

    // --- candidate pairs of neighbouring core grids (at most nnbr of them):
    //     touching grids first, then the others
    mark(8);
    GD_TRY(ensure(ctx, ctx->pairs, (size_t)nnbr * 8 + 16, st));
    GD_TRY(ensure(ctx, ctx->hard, (size_t)nnbr * 8 + 16, st));
    int2* pairs = (int2*)ctx->pairs.ptr;
    int2* hard = (int2*)ctx->hard.ptr;
    GD_CUDA(launch_pair_count(p, w.nbr_start, nbr, w.core_start, w.cell_coord, C, w.pair_start, w.pair_start_f, st));
    GD_CUDA(scan_exclusive(w.pair_start, w.pair_start, C, w.tmp, st));
    GD_CUDA(scan_exclusive(w.pair_start_f, w.pair_start_f, C, w.tmp, st));
    GD_CUDA(launch_pair_fill(p, w.nbr_start, nbr, w.core_start, w.cell_coord, C, w.pair_start, w.pair_start_f, pairs,
                             st));

    // --- merging (Def. 6-7): two waves, each a warp-level test then
    //     FastMerging (Alg. 5) on the pairs left undecided
    mark(9);
    GD_TRY(readback(ctx, ctx->small + kMaxCell, 1, st));
    const int wpb = (ctx->host_small[0] + 31) / 32 + 1;
    GD_TRY(ensure(ctx, ctx->mscratch, (size_t)merge_fm_blocks() * 2 * wpb * 4, st));
    GD_CUDA(launch_uf_init(w.parent, C, st));
    GD_CUDA(launch_merge_ranges(w.pair_start, w.pair_start_f, C, ctx->small + kRange, ctx->small + kHardCnt, st));
    for (int wave = 0; wave < 2; ++wave) {
        GD_CUDA(launch_merge_wave(p, wave, pairs, ctx->small + kRange, (int)nnbr, w.Xc, w.core_start, w.bbox, w.parent,
                                  (unsigned*)(ctx->small + kStatus), hard, ctx->small + kHardCnt,
                                  (unsigned*)ctx->mscratch.ptr, wpb, merge_fm_blocks(), st));
        if (wave == 0) GD_CUDA(launch_uf_flatten(w.parent, C, (unsigned*)(ctx->small + kStatus), st));
    }

    // --- cluster ids, border points, labels
    mark(10);
    GD_CUDA(launch_cluster_ids(p, w.parent, w.core_start, w.cell_start, w.core_s, perm, C, w.cid_root, w.cell_cid,
                               st, (unsigned*)(ctx->small + kStatus)));
    GD_CUDA(launch_labels(p, w.Xs, w.cell_start, w.pt_cell, w.core_s, w.nbr_start, nbr, w.core_start, w.Xc, w.bbox,
                          w.cell_cid, perm, labels, is_core, st));
    mark(11);
    GD_TRY(readback(ctx, ctx->small, kSmallInts, st));
    const unsigned status = (unsigned)ctx->host_small[kStatus];
    if (status & kDevTimeout) return fail(ctx, GD_ETIMEOUT, "a bounded device wait or retry loop hit its limit");

    if (ctx->timing) {
        for (int s = 0; s < kStages; ++s) cudaEventElapsedTime(&ctx->stage_ms[s], ctx->ev[s], ctx->ev[s + 1]);
        ctx->nstages = kStages;
    }
    // remember the last run for introspection
    const int npairs = ctx->host_small[kRange + 3];
    ctx->sizes[0] = n;
    ctx->sizes[1] = d;
    ctx->sizes[2] = C;
    ctx->sizes[3] = nnbr;
    ctx->sizes[4] = p.s;
    ctx->sizes[5] = p.key_bits;
    ctx->sizes[6] = t_launches - launches0;
    ctx->sizes[7] = npairs;
    {
        const SortPlan sp = sort_plan(n, p.key_words, p.key_bits);
        ctx->sizes[8] = sp.passes;
        ctx->sizes[9] = sp.bits;
    }
    ctx->sizes[10] = (int64_t)ctx->host_small[kHardCnt] + ctx->host_small[kHardCnt + 1];
    ctx->sizes[11] = 0;
    ctx->view_ptr[GD_VIEW_PERM] = perm;
    ctx->view_bytes[GD_VIEW_PERM] = (size_t)n * 4;
    ctx->view_ptr[GD_VIEW_CELL_START] = w.cell_start;
    ctx->view_bytes[GD_VIEW_CELL_START] = (size_t)(C + 1) * 4;
    ctx->view_ptr[GD_VIEW_CELL_COORD] = w.cell_coord;
    ctx->view_bytes[GD_VIEW_CELL_COORD] = (size_t)C * d * 4;
    ctx->view_ptr[GD_VIEW_NBR_START] = w.nbr_start;
    ctx->view_bytes[GD_VIEW_NBR_START] = (size_t)(C + 1) * 4;
    ctx->view_ptr[GD_VIEW_NBR] = nbr;
    ctx->view_bytes[GD_VIEW_NBR] = (size_t)nnbr * 4;
    ctx->view_ptr[GD_VIEW_CORE_SORTED] = w.core_s;
    ctx->view_bytes[GD_VIEW_CORE_SORTED] = (size_t)n;
    ctx->view_ptr[GD_VIEW_CELL_CID] = w.cell_cid;
    ctx->view_bytes[GD_VIEW_CELL_CID] = (size_t)C * 4;
    ctx->have_run = true;
    return GD_OK;
}

}  // namespace

extern "C" {

gd_status gd_create(gd_ctx** out, int device) {
    if (!out) return GD_EINVAL;
    *out = nullptr;
    gd_ctx* ctx = new (std::nothrow) gd_ctx();
    if (!ctx) return GD_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->small, sizeof(int) * kSmallInts);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->host_small, sizeof(int) * kSmallInts);
    for (int i = 0; e == cudaSuccess && i <= kStages; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        gd_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? GD_ENOMEM : GD_ECUDA;
    }
    *out = ctx;
    return GD_OK;
}

void gd_destroy(gd_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (DevBuf* b : {&ctx->arena, &ctx->nbr, &ctx->pairs, &ctx->hard, &ctx->mscratch, &ctx->io})
        if (b->ptr) cudaFree(b->ptr);
    if (ctx->small) cudaFree(ctx->small);
    if (ctx->host_small) cudaFreeHost(ctx->host_small);
    for (int i = 0; i <= kStages; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

size_t gd_workspace_bytes(int64_t n, int d) {
    if (n < 0 || d < 1 || d > kMaxD) return 0;
    Work w;
    return carve(&w, nullptr, n, d, 2, 128) + (size_t)n * 8;
}

gd_status gd_dbscan(gd_ctx* ctx, const int32_t* X, int64_t n, int d, int64_t eps2, int32_t minpts, int32_t* labels,
                    uint8_t* is_core, gd_stream_t stream) {
    GD_TRY(validate(ctx, X, n, d, eps2, minpts, labels));
    ctx->err.clear();
    if (n == 0) return GD_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return run(ctx, X, n, d, eps2, minpts, labels, is_core, (cudaStream_t)stream);
}

gd_status gd_dbscan_host(gd_ctx* ctx, const int32_t* X_host, int64_t n, int d, int64_t eps2, int32_t minpts,
                         int32_t* labels_host, uint8_t* is_core_host, gd_stream_t stream) {
    GD_TRY(validate(ctx, X_host, n, d, eps2, minpts, labels_host));
    ctx->err.clear();
    if (n == 0) return GD_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t xb = (size_t)n * d * 4, lb = (size_t)n * 4, cb = (size_t)n;
    const size_t xo = 0, lo = (xb + 255) & ~(size_t)255, co = (lo + lb + 255) & ~(size_t)255;
    GD_TRY(ensure(ctx, ctx->io, co + cb, st));
    int32_t* Xd = (int32_t*)(ctx->io.ptr + xo);
    int32_t* Ld = (int32_t*)(ctx->io.ptr + lo);
    uint8_t* Cd = (uint8_t*)(ctx->io.ptr + co);
    GD_CUDA(cudaMemcpyAsync(Xd, X_host, xb, cudaMemcpyHostToDevice, st));
    GD_TRY(run(ctx, Xd, n, d, eps2, minpts, Ld, is_core_host ? Cd : nullptr, st));
    GD_CUDA(cudaMemcpyAsync(labels_host, Ld, lb, cudaMemcpyDeviceToHost, st));
    if (is_core_host) GD_CUDA(cudaMemcpyAsync(is_core_host, Cd, cb, cudaMemcpyDeviceToHost, st));
    GD_CUDA(cudaStreamSynchronize(st));
    return GD_OK;
}

const char* gd_status_str(gd_status s) {
    switch (s) {
        case GD_OK: return "ok";
        case GD_EINVAL: return "invalid argument";
        case GD_ERANGE: return "coordinate range or key width out of range";
        case GD_ENOMEM: return "out of memory";
        case GD_ECUDA: return "CUDA error";
        case GD_ETIMEOUT: return "device retry limit reached";
        case GD_EBUSY: return "busy";
    }
    return "unknown status";
}

const char* gd_last_error(const gd_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

gd_status gd_last_sizes(const gd_ctx* ctx, int64_t out[12]) {
    if (!ctx || !out || !ctx->have_run) return GD_EINVAL;
    for (int i = 0; i < 12; ++i) out[i] = ctx->sizes[i];
    return GD_OK;
}

gd_status gd_copy_view(gd_ctx* ctx, gd_view which, void* host_dst, size_t bytes) {
    if (!ctx || !ctx->have_run || (int)which < 0 || (int)which > 6 || (!host_dst && bytes)) return GD_EINVAL;
    if (bytes > ctx->view_bytes[which]) return fail(ctx, GD_EINVAL, "view smaller than requested bytes");
    if (bytes == 0) return GD_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMemcpy(host_dst, ctx->view_ptr[which], bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy (view)");
    return GD_OK;
}

gd_status gd_set_timing(gd_ctx* ctx, int enable) {
    if (!ctx) return GD_EINVAL;
    ctx->timing = enable != 0;
    ctx->nstages = 0;
    return GD_OK;
}

int gd_stage_times(const gd_ctx* ctx, float* ms, const char** names, int max) {
    if (!ctx) return 0;
    int k = ctx->nstages < max ? ctx->nstages : max;
    for (int i = 0; i < k; ++i) {
        if (ms) ms[i] = ctx->stage_ms[i];
        if (names) names[i] = kStageNames[i];
    }
    return k;
}

}  // extern "C"
