// C ABI of libgdbscan: contexts and the entry points, over the batched
// driver (pipeline.cu).  gd_dbscan is a batch of one.
#include <climits>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gdbscan.h"
#include "pipeline.h"

using namespace gd;

namespace gd {
thread_local long long t_launches = 0;
}

namespace {

struct DevBuf {
    char* ptr = nullptr;
    size_t cap = 0;
};
struct HostBuf {
    char* ptr = nullptr;
    size_t cap = 0;
};

// The context's memory: device buffers grown on demand with cudaMalloc (to
// 1/8 more than asked, kept for reuse), pinned host staging likewise.  With
// a cap, a buffer that would take the device bytes held past it is refused
// (GD_ENOMEM) and the buffers held stay as they are.
struct CtxMem : MemProvider {
    DevBuf dev[kMemSlots];
    HostBuf host_[kHostSlots];
    cudaStream_t st = nullptr;
    std::string* err = nullptr;
    double pool_ratio = 0.0, runs_ratio = 0.0;  // most pool entries / runs per point seen
    PlanCache cache;         // plans and sizes of earlier calls, per instance shape
    size_t cap_bytes = 0;    // 0: no cap
    const size_t* extra_held = nullptr;  // other device bytes the context holds (I/O copies)
    int fail_at = 0;         // > 0: the fail_at-th device request from now fails (tests)

    size_t held() const {
        size_t b = extra_held ? *extra_held : 0;
        for (const DevBuf& d : dev) b += d.cap;
        return b;
    }

    bool pool_enabled() override { return true; }
    double pool_per_point() override { return pool_ratio; }
    double runs_per_point() override { return runs_ratio; }
    void note_pool(double entries, double runs) override {
        if (entries > pool_ratio) pool_ratio = entries;
        if (runs > runs_ratio) runs_ratio = runs;
    }
    PlanCache* plans() override { return &cache; }
    void* current(int slot) override { return dev[slot].ptr; }

    gd_status device(int slot, size_t bytes, void** out) override {
        DevBuf& b = dev[slot];
        if (fail_at > 0 && --fail_at == 0) {
            if (err) *err = "device buffer request refused (injected failure)";
            return GD_ENOMEM;
        }
        if (b.cap < bytes) {
            const size_t want0 = bytes + bytes / 8 + (1 << 16);
            if (cap_bytes && held() - b.cap + want0 > cap_bytes) {
                if (err) *err = "device buffer of " + std::to_string(want0) + " bytes exceeds the context's cap";
                return GD_ENOMEM;
            }
            if (b.ptr) {
                if (cudaStreamSynchronize(st) != cudaSuccess) return GD_ECUDA;
                cudaFree(b.ptr);
                b.ptr = nullptr;
                b.cap = 0;
            }
            const size_t want = bytes + bytes / 8 + (1 << 16);
            if (cudaMalloc((void**)&b.ptr, want) != cudaSuccess) {
                cudaGetLastError();
                b.ptr = nullptr;
                if (err) *err = "cudaMalloc of " + std::to_string(want) + " bytes failed";
                return GD_ENOMEM;
            }
            b.cap = want;
        }
        *out = b.ptr;
        return GD_OK;
    }
    gd_status host(int slot, size_t bytes, void** out) override {
        HostBuf& b = host_[slot];
        if (b.cap < bytes) {
            if (b.ptr) {
                if (cudaStreamSynchronize(st) != cudaSuccess) return GD_ECUDA;
                cudaFreeHost(b.ptr);
                b.ptr = nullptr;
                b.cap = 0;
            }
            const size_t want = bytes + bytes / 8 + 4096;
            if (cudaMallocHost((void**)&b.ptr, want) != cudaSuccess) {
                cudaGetLastError();
                b.ptr = nullptr;
                if (err) *err = "cudaMallocHost of " + std::to_string(want) + " bytes failed";
                return GD_ENOMEM;
            }
            b.cap = want;
        }
        *out = b.ptr;
        return GD_OK;
    }
    void release() {
        for (DevBuf& b : dev)
            if (b.ptr) cudaFree(b.ptr);
        for (HostBuf& b : host_)
            if (b.ptr) cudaFreeHost(b.ptr);
        for (DevBuf& b : dev) b = DevBuf();
        for (HostBuf& b : host_) b = HostBuf();
        pool_ratio = runs_ratio = 0.0;
        cache.clear();
    }
};

}  // namespace

struct gd_ctx {
    int device = 0;
    CtxMem mem;
    DevBuf io;  // device copies for gd_dbscan_host
    int uf_cap = 0;  // union-find retry cap (0: built-in)
    cudaEvent_t ev[kStageEvents] = {};
    bool timing = false;
    bool stats = false;
    float stage_ms[kStages + 1] = {};   // the stages, then the sort's downsweeps
    cudaEvent_t sev[2 * kSortEventPairs] = {};
    int nstages = 0;
    std::string err;
    bool have_run = false;
    RunInfo info;
    Tuning tuning;
    PhaseGraphs graphs;
    // graphs cannot be captured from the legacy default stream: such calls
    // run on this stream, ordered after the caller's by events
    cudaStream_t own = nullptr;
    cudaEvent_t own_ev = nullptr, own_done = nullptr;
    // the call queued last and not finished yet: its instances (for a run
    // with exact sizes), the stream it runs on and the caller's stream
    bool pending = false;
    std::vector<gd_instance> pend_inst;
    cudaStream_t pend_st = nullptr, pend_caller = nullptr;
    gd_status deferred = GD_OK;  // first failure of a call finished before gd_sync
    std::string deferred_err;
    // host staging sets (calls alternate) and their last-upload events
    int next_set = 0;
    cudaEvent_t stage_ev[2] = {};
    // results of a host-buffer call still to reach the host: the copies are
    // queued after the run (and queued again after a run with exact sizes)
    struct HostOut {
        bool active = false;
        void* lab = nullptr;
        void* core = nullptr;
        const void* dlab = nullptr;
        const void* dcore = nullptr;
        size_t lb = 0, cb = 0;
        cudaStream_t st = nullptr;
    } out;
};

namespace {

gd_status validate_one(const gd_instance& g, std::string* err) {
    if (g.d < 1 || g.d > kMaxD) return *err = "d must be in [1, 8]", GD_EINVAL;
    if (g.n < 0 || g.n >= (int64_t)INT_MAX) return *err = "n must be in [0, 2^31 - 1)", GD_EINVAL;
    if (g.eps2 < 0) return *err = "eps2 must be >= 0", GD_EINVAL;
    if (g.eps2_yes != 0 && g.eps2_yes < g.eps2) return *err = "eps2_yes must be 0 or >= eps2", GD_EINVAL;
    if (g.minpts < 1) return *err = "minpts must be >= 1", GD_EINVAL;
    if (g.n > 0 && (!g.X || !g.labels)) return *err = "null pointer with n > 0", GD_EINVAL;
    return GD_OK;
}

// The stream a call runs on: the caller's, or (graphs on the legacy
// default stream, which cannot be captured) the context's own, ordered after
// the caller's work by an event.
gd_status call_stream(gd_ctx* ctx, cudaStream_t caller, cudaStream_t* st) {
    *st = caller;
    if (ctx->graphs.enabled && (caller == nullptr || caller == cudaStreamLegacy || caller == cudaStreamPerThread)) {
        if (!ctx->own) {
            if (cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->own_ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->own_done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return ctx->err = "stream creation failed", GD_ECUDA;
            }
        }
        if (cudaEventRecord(ctx->own_ev, caller) != cudaSuccess || cudaStreamWaitEvent(ctx->own, ctx->own_ev, 0) != cudaSuccess)
            return ctx->err = "stream ordering failed", GD_ECUDA;
        *st = ctx->own;
    }
    return GD_OK;
}

// Queues a call (see run_batch); with `allow_async` false it reads its sizes
// back (a run with exact sizes).
gd_status queue(gd_ctx* ctx, int k, const gd_instance* inst, cudaStream_t caller, bool allow_async) {
    cudaStream_t st;
    gd_status s = call_stream(ctx, caller, &st);
    if (s != GD_OK) return s;
    ctx->mem.st = st;
    ctx->mem.err = &ctx->err;
    ctx->info = RunInfo();
    ctx->info.want_stats = ctx->stats;
    ctx->info.uf_cap = ctx->uf_cap;
    const int set = ctx->next_set;
    ctx->next_set ^= 1;
    const long long l0 = t_launches;
    s = run_batch(ctx->mem, k, inst, st, ctx->timing ? ctx->ev : nullptr, &ctx->info, &ctx->tuning, &ctx->graphs,
                  ctx->timing ? ctx->sev : nullptr, StageSet{set, ctx->stage_ev[set]}, allow_async);
    ctx->info.sizes[6] = t_launches - l0;
    if (st != caller && st == ctx->own) {
        // later work on the caller's stream is ordered after the call
        if (cudaEventRecord(ctx->own_done, st) != cudaSuccess || cudaStreamWaitEvent(caller, ctx->own_done, 0) != cudaSuccess)
            if (s == GD_OK) s = (ctx->err = "stream ordering failed", GD_ECUDA);
    }
    if (s != GD_OK) {
        if (ctx->err.empty()) ctx->err = ctx->info.error;
        // what was queued must finish before the buffers are touched again
        cudaStreamSynchronize(st);
        return s;
    }
    ctx->pending = true;
    ctx->pend_inst.assign(inst, inst + k);
    ctx->pend_st = st;
    ctx->pend_caller = caller;
    return GD_OK;
}

// Finishes the pending call: waits for it, reads its status back, runs it
// again with exact sizes if a plan or capacity from an earlier call did not
// fit, and computes the stage times.
gd_status finish(gd_ctx* ctx) {
    if (!ctx->pending) return GD_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->err = "cudaSetDevice failed", GD_ECUDA;
    const int k = (int)ctx->pend_inst.size();
    gd_status s = finish_batch(ctx->mem, k, ctx->pend_inst.data(), ctx->pend_st, &ctx->info);
    bool rerun = false;
    if (s == kGdRerun) {
        ctx->pending = false;
        rerun = true;
        const std::vector<gd_instance> again = ctx->pend_inst;  // queue() replaces pend_inst
        s = queue(ctx, k, again.data(), ctx->pend_caller, false);
        if (s == GD_OK) s = finish_batch(ctx->mem, k, again.data(), ctx->pend_st, &ctx->info);
        if (s == kGdRerun) s = (ctx->info.error = "device buffers overflowed on a run with exact sizes", GD_ECUDA);
    }
    ctx->pending = false;
    if (ctx->out.active) {
        // a host-buffer call: its copies out follow the (last) run
        gd_ctx::HostOut& o = ctx->out;
        if (s == GD_OK && rerun) {
            if (cudaMemcpyAsync(o.lab, o.dlab, o.lb, cudaMemcpyDeviceToHost, o.st) != cudaSuccess ||
                (o.core && cudaMemcpyAsync(o.core, o.dcore, o.cb, cudaMemcpyDeviceToHost, o.st) != cudaSuccess))
                s = (ctx->info.error = "copy out failed", GD_ECUDA);
        }
        if (cudaStreamSynchronize(o.st) != cudaSuccess && s == GD_OK)
            s = (ctx->info.error = "synchronise failed", GD_ECUDA);
        o.active = false;
    }
    if (s != GD_OK) {
        ctx->err = ctx->info.error;
        return s;
    }
    if (ctx->timing) {
        for (int i = 0; i < kStages; ++i) {
            // stages ending at a read-back of sizes have their own end event
            const int end = i == 0 ? kStages + 1 : i == 3 ? kStages + 2 : i == 5 ? kStages + 3 : i + 1;
            cudaEventElapsedTime(&ctx->stage_ms[i], ctx->ev[i], ctx->ev[end]);
        }
        float ds = 0.f;
        for (int i = 0; i < ctx->info.sort_event_pairs; ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ctx->sev[2 * i], ctx->sev[2 * i + 1]);
            ds += t;
        }
        ctx->stage_ms[kStages] = ds;
        ctx->nstages = kStages + 1;
        cudaGetLastError();
    }
    ctx->have_run = true;
    return GD_OK;
}

// A new call: the previous one is finished first (its failure is kept for
// the next gd_sync).
gd_status run_ctx(gd_ctx* ctx, int k, const gd_instance* inst, cudaStream_t st) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->err = "cudaSetDevice failed", GD_ECUDA;
    if (ctx->pending) {
        const gd_status p = finish(ctx);
        if (p != GD_OK && ctx->deferred == GD_OK) {
            ctx->deferred = p;
            ctx->deferred_err = ctx->err;
        }
    }
    ctx->err.clear();
    ctx->have_run = false;
    ctx->nstages = 0;
    return queue(ctx, k, inst, st, true);
}

}  // namespace

extern "C" {

gd_status gd_create(gd_ctx** out, int device, size_t arena_bytes) {
    if (!out) return GD_EINVAL;
    *out = nullptr;
    gd_ctx* ctx = new (std::nothrow) gd_ctx();
    if (!ctx) return GD_ENOMEM;
    ctx->device = device;
    ctx->mem.cap_bytes = arena_bytes;
    ctx->mem.extra_held = &ctx->io.cap;
    cudaError_t e = cudaSetDevice(device);
    for (int i = 0; e == cudaSuccess && i < kStageEvents; ++i) e = cudaEventCreate(&ctx->ev[i]);
    for (int i = 0; e == cudaSuccess && i < 2 * kSortEventPairs; ++i) e = cudaEventCreate(&ctx->sev[i]);
    for (int i = 0; e == cudaSuccess && i < 2; ++i) e = cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming);
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
    ctx->graphs.release();
    if (ctx->own) cudaStreamDestroy(ctx->own);
    if (ctx->own_ev) cudaEventDestroy(ctx->own_ev);
    if (ctx->own_done) cudaEventDestroy(ctx->own_done);
    for (int i = 0; i < 2; ++i)
        if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]);
    ctx->mem.release();
    if (ctx->io.ptr) cudaFree(ctx->io.ptr);
    for (int i = 0; i < kStageEvents; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < 2 * kSortEventPairs; ++i)
        if (ctx->sev[i]) cudaEventDestroy(ctx->sev[i]);
    delete ctx;
}

size_t gd_workspace_bytes(int64_t n, int d) {
    if (n < 0 || n >= (int64_t)INT_MAX || d < 1 || d > kMaxD) return 0;
    // the per-instance arrays (upper bound: 128-bit keys, the most digit
    // passes) plus the batch's small blocks, descriptors and scan scratch
    const size_t N = (size_t)n, dp = d == 1 ? 1 : d == 2 ? 2 : d <= 4 ? 4 : 8;
    size_t b = N * (2 * 16 + 2 * 4 + 2 * dp * 4 + 4 + 1 + 4 * 12 + (size_t)d * 4 * 4 + 4 * (2 * d + 2));
    b += sort_tmp_ints((int)n, 2, 128) * 4 + ((size_t)1 << 20);
    return b;
}

gd_status gd_dbscan(gd_ctx* ctx, const int32_t* X, int64_t n, int d, int64_t eps2, int32_t minpts, int32_t* labels,
                    uint8_t* is_core, gd_stream_t stream) {
    if (!ctx) return GD_EINVAL;
    ctx->err.clear();
    gd_instance g{X, n, d, eps2, minpts, labels, is_core};
    gd_status s = validate_one(g, &ctx->err);
    if (s != GD_OK || n == 0) return s;
    return run_ctx(ctx, 1, &g, (cudaStream_t)stream);
}

gd_status gd_dbscan_batched(gd_ctx* ctx, int k, const gd_instance* inst, gd_stream_t stream) {
    if (!ctx) return GD_EINVAL;
    ctx->err.clear();
    if (k < 0 || (k > 0 && !inst)) return ctx->err = "bad instance array", GD_EINVAL;
    if (k == 0) return GD_OK;
    for (int i = 0; i < k; ++i) {
        gd_status s = validate_one(inst[i], &ctx->err);
        if (s != GD_OK) return ctx->err += " (instance " + std::to_string(i) + ")", s;
        if (inst[i].n == 0) return ctx->err = "empty instance in a batch (instance " + std::to_string(i) + ")", GD_EINVAL;
    }
    return run_ctx(ctx, k, inst, (cudaStream_t)stream);
}

gd_status gd_dbscan_host_async(gd_ctx* ctx, const int32_t* X_host, int64_t n, int d, int64_t eps2, int32_t minpts,
                               int32_t* labels_host, uint8_t* is_core_host, gd_stream_t stream) {
    if (!ctx) return GD_EINVAL;
    ctx->err.clear();
    gd_instance g{X_host, n, d, eps2, minpts, labels_host, is_core_host};
    gd_status s = validate_one(g, &ctx->err);
    if (s != GD_OK || n == 0) return s;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->err = "cudaSetDevice failed", GD_ECUDA;
    // the previous call (and its copies out) are done before the device
    // copies are reused; its failure is kept for the next gd_sync
    if (ctx->pending) {
        const gd_status p = finish(ctx);
        if (p != GD_OK && ctx->deferred == GD_OK) {
            ctx->deferred = p;
            ctx->deferred_err = ctx->err;
        }
        ctx->err.clear();
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t xb = (size_t)n * d * 4, lb = (size_t)n * 4, cb = (size_t)n;
    const size_t lo = (xb + 255) & ~(size_t)255, co = (lo + lb + 255) & ~(size_t)255;
    if (ctx->io.cap < co + cb) {
        if (ctx->mem.cap_bytes && ctx->mem.held() - ctx->io.cap + co + cb > ctx->mem.cap_bytes)
            return ctx->err = "input/output copies exceed the context's cap", GD_ENOMEM;
        if (ctx->io.ptr) {
            cudaStreamSynchronize(st);
            cudaFree(ctx->io.ptr);
            ctx->io = DevBuf();
        }
        if (cudaMalloc((void**)&ctx->io.ptr, co + cb) != cudaSuccess) {
            cudaGetLastError();
            ctx->io = DevBuf();
            return ctx->err = "cudaMalloc of the input/output copies failed", GD_ENOMEM;
        }
        ctx->io.cap = co + cb;
    }
    gd_instance dg{(const int32_t*)ctx->io.ptr, n, d, eps2, minpts, (int32_t*)(ctx->io.ptr + lo),
                   is_core_host ? (uint8_t*)(ctx->io.ptr + co) : nullptr};
    if (cudaMemcpyAsync((void*)dg.X, X_host, xb, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ctx->err = "copy in failed", GD_ECUDA;
    s = run_ctx(ctx, 1, &dg, st);
    if (s != GD_OK) return s;
    // copies out behind the run (queued again by gd_sync if the run must be
    // repeated with exact sizes)
    gd_ctx::HostOut& o = ctx->out;
    o.lab = labels_host;
    o.core = is_core_host;
    o.dlab = dg.labels;
    o.dcore = dg.is_core;
    o.lb = lb;
    o.cb = cb;
    o.st = st;
    o.active = true;
    if (cudaMemcpyAsync(labels_host, dg.labels, lb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (is_core_host && cudaMemcpyAsync(is_core_host, dg.is_core, cb, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        return ctx->err = "copy out failed", GD_ECUDA;
    return GD_OK;
}

gd_status gd_dbscan_host(gd_ctx* ctx, const int32_t* X_host, int64_t n, int d, int64_t eps2, int32_t minpts,
                         int32_t* labels_host, uint8_t* is_core_host, gd_stream_t stream) {
    gd_status s = gd_dbscan_host_async(ctx, X_host, n, d, eps2, minpts, labels_host, is_core_host, stream);
    if (s != GD_OK || n == 0) return s;
    return gd_sync(ctx, stream);
}

size_t gd_ctx_bytes(const gd_ctx* ctx) {
    if (!ctx) return 0;
    size_t b = ctx->io.cap;
    for (const DevBuf& d : ctx->mem.dev) b += d.cap;
    return b;
}

gd_status gd_sync(gd_ctx* ctx, gd_stream_t stream) {
    if (!ctx) return GD_EINVAL;
    (void)stream;  // a context has at most one call in flight: its own stream is known
    gd_status s = finish(ctx);
    if (ctx->deferred != GD_OK) {
        const gd_status d = ctx->deferred;
        ctx->err = ctx->deferred_err;
        ctx->deferred = GD_OK;
        ctx->deferred_err.clear();
        return d;
    }
    return s;
}

gd_status gd_ctx_trim(gd_ctx* ctx) {
    if (!ctx) return GD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return GD_ECUDA;
    finish(ctx);
    if (ctx->mem.st) cudaStreamSynchronize(ctx->mem.st);
    ctx->graphs.release();
    ctx->mem.release();
    if (ctx->io.ptr) cudaFree(ctx->io.ptr);
    ctx->io = DevBuf();
    ctx->have_run = false;
    return GD_OK;
}

gd_status gd_set_graphs(gd_ctx* ctx, int enable) {
    if (!ctx) return GD_EINVAL;
    ctx->graphs.enabled = enable != 0;
    return GD_OK;
}

gd_status gd_graph_stats(const gd_ctx* ctx, int64_t out[3]) {
    if (!ctx || !out) return GD_EINVAL;
    out[0] = ctx->graphs.launches;
    out[1] = ctx->graphs.updates;
    out[2] = ctx->graphs.instantiations;
    return GD_OK;
}

gd_status gd_set_tuning(gd_ctx* ctx, const gd_tuning* entries, int count) {
    if (!ctx) return GD_EINVAL;
    if (count < 0 || count > kMaxTuning || (count > 0 && !entries))
        return ctx->err = "tuning table: bad entry count or pointer", GD_EINVAL;
    for (int i = 0; i < count; ++i) {
        const gd_tuning& t = entries[i];
        if (t.d < 0 || t.d > kMaxD || t.n_max < 0 || !knob_in_range(t.knob, t.value))
            return ctx->err = "tuning table: bad entry " + std::to_string(i), GD_EINVAL;
    }
    for (int i = 0; i < count; ++i) ctx->tuning.e[i] = entries[i];
    ctx->tuning.count = count;
    return GD_OK;
}

gd_status gd_get_knob(const gd_ctx* ctx, int knob, int d, int64_t n, int32_t* value) {
    if (!ctx || !value || knob_default(knob, d) < 0) return GD_EINVAL;
    *value = ctx->tuning.value(knob, d, n);
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

gd_status gd_last_sizes(gd_ctx* ctx, int64_t out[13]) {
    if (!ctx || !out) return GD_EINVAL;
    if (ctx->pending) finish(ctx);
    if (!ctx->have_run) return GD_EINVAL;
    for (int i = 0; i < 13; ++i) out[i] = ctx->info.sizes[i];
    return GD_OK;
}

gd_status gd_copy_view(gd_ctx* ctx, gd_view which, void* host_dst, size_t bytes) {
    if (ctx && ctx->pending) finish(ctx);
    if (!ctx || !ctx->have_run || (int)which < 0 || (int)which > 6 || (!host_dst && bytes)) return GD_EINVAL;
    if (bytes > ctx->info.view_bytes[which]) return ctx->err = "view smaller than requested bytes", GD_EINVAL;
    if (bytes == 0) return GD_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMemcpy(host_dst, ctx->info.view_ptr[which], bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ctx->err = std::string("cudaMemcpy (view): ") + cudaGetErrorString(e), GD_ECUDA;
    return GD_OK;
}

gd_status gd_set_timing(gd_ctx* ctx, int enable) {
    if (!ctx) return GD_EINVAL;
    ctx->timing = enable != 0;
    ctx->nstages = 0;
    return GD_OK;
}

gd_status gd_set_retry_limit(gd_ctx* ctx, int32_t limit) {
    if (!ctx || limit < 0) return GD_EINVAL;
    ctx->uf_cap = limit;
    return GD_OK;
}

gd_status gd_inject_alloc_failure(gd_ctx* ctx, int32_t k) {
    if (!ctx || k < 0) return GD_EINVAL;
    ctx->mem.fail_at = k;
    return GD_OK;
}

gd_status gd_set_stats(gd_ctx* ctx, int enable) {
    if (!ctx) return GD_EINVAL;
    ctx->stats = enable != 0;
    return GD_OK;
}

static const char* const kStatNames[kStatCount] = {
    "pairs", "pairs_skipped", "pairs_box_no", "pairs_box_yes", "pairs_lane", "pairs_warp", "pairs_fastmerging",
    "fm_yes", "fm_no", "fm_pruned_triangle", "fm_pruned_angle", "nonfull_points", "count_rows",
    "dist_core", "dist_merge", "dist_fastmerging", "dist_labels", "walk_nodes", "walk_steps",
    "kappa_1", "kappa_2", "kappa_3", "kappa_4", "kappa_5", "kappa_6", "kappa_7", "kappa_8", "kappa_9",
    "kappa_10", "kappa_11", "kappa_12", "kappa_13", "kappa_14", "kappa_15", "kappa_16_or_more"};

int gd_run_stats(gd_ctx* ctx, int64_t* values, const char** names, int max) {
    if (ctx && ctx->pending) finish(ctx);
    if (!ctx || !ctx->have_run || !ctx->info.have_stats) return 0;
    const int k = kStatCount < max ? kStatCount : max;
    for (int i = 0; i < k; ++i) {
        if (values) values[i] = (int64_t)ctx->info.stats[i];
        if (names) names[i] = kStatNames[i];
    }
    return k;
}

int gd_stage_times(gd_ctx* ctx, float* ms, const char** names, int max) {
    if (!ctx) return 0;
    if (ctx->pending) finish(ctx);
    int k = ctx->nstages < max ? ctx->nstages : max;
    for (int i = 0; i < k; ++i) {
        if (ms) ms[i] = ctx->stage_ms[i];
        if (names) names[i] = i < kStages ? kStageNames[i] : "sort_downsweep";
    }
    return k;
}

}  // extern "C"
