// gd_dbscan_noalloc: the exact-DBSCAN pipeline with every buffer taken from
// one fixed, statically sized device array instead of cudaMalloc.
//
// Some callers cannot allocate device memory at the time they need a
// clustering: code running under a memory manager that owns the whole device
// pool, a plugin in a host application that forbids allocations on its hot
// path, or a process whose allocator is already exhausted.  This entry point
// serves them for small inputs (at most GD_NOALLOC_MAX_POINTS points): it
// calls no cudaMalloc, cudaFree, cudaMallocHost or any other allocating
// routine.  It runs the same driver and kernels as gd_dbscan, so its labels
// equal gd_dbscan's bit for bit.
//
// The device array below (GD_NOALLOC_SCRATCH_BYTES) is backed on a GPU once
// the module holding it is loaded there and stays until the process exits.
// CUDA loads modules lazily by default (CUDA_MODULE_LOADING=LAZY), so that
// happens inside the first call on each device: callers should make one
// warm-up call per device at start-up, before any allocation budget is
// spent and before any stream capture.  The host-side staging it needs is a
// static host array.
#include <cstring>
#include <mutex>

#include "gdbscan.h"
#include "pipeline.h"

using namespace gd;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GD_NOALLOC_SCRATCH_BYTES];

constexpr size_t kHostStaging = 1 << 20;
std::mutex g_mutex;  // serialises host callers (they share both arrays)
alignas(256) unsigned char g_host[kHostSlots][kHostStaging];

// Memory from the static arrays: each slot is carved once per call, in the
// order the driver asks for it; asking again for a slot returns the same
// buffer if it is big enough.  Nothing is ever allocated.
struct StaticMem : MemProvider {
    char* base = nullptr;
    size_t off = 0;
    char* slot_ptr[kMemSlots] = {};
    size_t slot_cap[kMemSlots] = {};

    gd_status device(int slot, size_t bytes, void** out) override {
        if (slot_ptr[slot]) {
            if (slot_cap[slot] < bytes) return GD_ENOMEM;
            *out = slot_ptr[slot];
            return GD_OK;
        }
        off = (off + 255) & ~(size_t)255;
        if (off + bytes > (size_t)GD_NOALLOC_SCRATCH_BYTES) return GD_ENOMEM;
        slot_ptr[slot] = base + off;
        slot_cap[slot] = bytes;
        off += bytes;
        *out = slot_ptr[slot];
        return GD_OK;
    }
    gd_status host(int slot, size_t bytes, void** out) override {
        if (bytes > kHostStaging) return GD_ENOMEM;
        *out = g_host[slot];
        return GD_OK;
    }
    void* current(int slot) override { return slot_ptr[slot]; }
};

// The FastMerging kernel's bitmaps come from the static array too: few blocks.
const Tuning& noalloc_tuning() {
    static Tuning t = [] {
        Tuning u;
        u.e[0] = gd_tuning{GD_KNOB_FM_BLOCKS, 0, INT64_MAX, 152};
        u.count = 1;
        return u;
    }();
    return t;
}

}  // namespace

extern "C" gd_status gd_dbscan_noalloc(const int32_t* X, int64_t n, int d, int64_t eps2, int32_t minpts,
                                       int32_t* labels, uint8_t* is_core, gd_stream_t stream) {
    if (d < 1 || d > 8 || n < 0 || eps2 < 0 || minpts < 1) return GD_EINVAL;
    if (n > GD_NOALLOC_MAX_POINTS) return GD_ENOMEM;
    if (n > 0 && (!X || !labels)) return GD_EINVAL;
    if (n == 0) return GD_OK;

    std::lock_guard<std::mutex> lock(g_mutex);
    // The device address of the static array on the current device.  The
    // host-side symbol is only a stand-in and must never be handed to a
    // kernel.  It is looked up on every call (cheap once the module is
    // loaded), so nothing stale survives a device reset.  The first lookup on
    // a device loads the module and backs the array; if the device cannot
    // back it, that is an out-of-memory condition, not a CUDA fault.
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GD_ENOMEM : GD_ECUDA;
    }
    StaticMem mem;
    mem.base = (char*)addr;
    // The driver clears every piece of device state it reads before it reads
    // it, so nothing left in the array by an earlier call leaks into this one.
    const gd_instance g{X, n, d, eps2, minpts, labels, is_core};
    const cudaStream_t st = (cudaStream_t)stream;
    // Sizes are read back while queueing (there is no plan of earlier calls),
    // so the run never has to be repeated; finish_batch waits for it and
    // reads its status.
    gd_status s = run_batch(mem, 1, &g, st, nullptr, nullptr, &noalloc_tuning(), nullptr, nullptr, StageSet(), false);
    if (s == GD_OK) s = finish_batch(mem, 1, &g, st, nullptr);
    if (s == kGdRerun) s = GD_ECUDA;  // cannot happen with exact sizes
    // A failed run may return with kernels still queued on the stream; they
    // use the shared array, so they must finish before the next caller gets
    // the lock.
    if (s != GD_OK) cudaStreamSynchronize(st);
    return s;
}
