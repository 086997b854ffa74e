// Host-side batched driver of the exact-DBSCAN pipeline (pipeline.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "gd_internal.cuh"
#include "gdbscan.h"

namespace gd {

// Where the driver's memory comes from: a context's growable buffers, or a
// fixed static array (the no-allocation entry point).
enum MemSlot {
    kMemSmall, kMemDesc, kMemArena, kMemScanTmp, kMemNbr, kMemHard, kMemScratch, kMemPool, kMemPoolSeg,
    kMemStats, kMemSlots
};
// Host staging: two sets (calls alternate between them, so that one call's
// uploads may still be pending while the next is built), each a small-block
// mirror plus host work area and a descriptor staging area; plus the area
// the results of a call are read back into.
enum HostSlot { kHostSmall0, kHostDesc0, kHostSmall1, kHostDesc1, kHostFinish, kHostSlots };

// What a context remembers about one instance shape (n, d, eps2) from the
// last call that clustered it: the sort's launch plan and the sizes the data
// needed.  A later call of that shape is queued with this plan and these
// sizes (plus margins) without reading anything back; the device checks that
// the data fit, and a call whose data did not is run again with exact sizes.
struct ShapePlan {
    long long n = -1;
    int d = 0;
    long long eps2 = -1;
    int key_class = 0, key_words = 1, key_bits = 0;
    long long nnbr = 0, maxcell = 0;
    unsigned long long stamp = 0;
};
struct PlanCache {
    static constexpr int kSize = 1024;
    ShapePlan e[kSize];
    unsigned long long clock = 0;
    const ShapePlan* find(long long n, int d, long long eps2) const {
        for (const ShapePlan& p : e)
            if (p.n == n && p.d == d && p.eps2 == eps2) return &p;
        return nullptr;
    }
    ShapePlan* slot(long long n, int d, long long eps2) {
        ShapePlan* old = &e[0];
        for (ShapePlan& p : e) {
            if (p.n == n && p.d == d && p.eps2 == eps2) return &p;
            if (p.stamp < old->stamp) old = &p;
        }
        *old = ShapePlan();
        old->n = n;
        old->d = d;
        old->eps2 = eps2;
        return old;
    }
    void clear() {
        for (ShapePlan& p : e) p = ShapePlan();
    }
};

struct MemProvider {
    virtual ~MemProvider() {}
    // A device buffer of at least `bytes` for the slot (contents are not kept
    // when it has to grow).  GD_ENOMEM if it cannot be had.
    virtual gd_status device(int slot, size_t bytes, void** out) = 0;
    // A host staging buffer (pinned where possible) of at least `bytes`.
    virtual gd_status host(int slot, size_t bytes, void** out) = 0;
    // Single-pass neighbour walk: whether to try it, and the most pool
    // entries and runs per point seen so far (size the pool; 0 = none yet).
    virtual bool pool_enabled() { return false; }
    virtual double pool_per_point() { return 0.0; }
    virtual double runs_per_point() { return 0.0; }
    virtual void note_pool(double, double) {}
    // Plans of earlier calls (null: every call reads its sizes back).
    virtual PlanCache* plans() { return nullptr; }
    // The slot's current buffer, as last handed out (no request is made).
    virtual void* current(int slot) = 0;
};

// Stage timing: when non-null, events[s] is recorded when stage s starts and
// events[kStages] at the end; stages that end at a read-back of sizes
// (bounds, compact, walk) also record events[kStages + 1 + i], i = 0, 1, 2,
// when their last kernel is issued, so that no stage includes host work.
constexpr int kStages = 12;
constexpr int kStageEvents = kStages + 4;
extern const char* const kStageNames[kStages];

// Kernel timing of the sort's downsweeps: when the driver is given sort
// events, it records a pair around each downsweep launch (at most
// kSortEventPairs) and reports how many pairs it used.
constexpr int kSortEventPairs = 48;

// What the driver reports about a run (instance 0 for the views).  Filled in
// two steps: when the run is queued (run_batch) and when its results are
// read back (finish_batch).
struct RunInfo {
    long long sizes[13] = {};
    const void* view_ptr[7] = {};
    size_t view_bytes[7] = {};
    long long launches = 0;
    int sort_event_pairs = 0;
    bool queued_async = false;  // queued without reading sizes back
    // union-find retry cap for the run (0: the built-in kMaxUfRetries)
    int uf_cap = 0;
    // statistics of the run (summed over its instances) when asked for
    bool want_stats = false;
    bool have_stats = false;
    unsigned long long stats[kStatCount] = {};
    std::string error;
};

// Host staging set and the event that marks its last upload, per call.
struct StageSet {
    int set = 0;                 // 0 or 1
    cudaEvent_t done = nullptr;  // recorded after the set's last upload (may be null)
};

// A context's tuning table (knobs of gdbscan.h).
constexpr int kMaxTuning = 1024;
struct Tuning {
    int count = 0;
    gd_tuning e[kMaxTuning];
    // The value of `knob` for a group of dimension d whose largest instance
    // has n points: the first matching entry, else the default.
    int value(int knob, int d, long long n) const;
};
// A knob's built-in value for instances of dimension d.
int knob_default(int knob, int d);
bool knob_in_range(int knob, int value);

// Executable graphs of the driver's launch phases, one per phase, kept by a
// context between calls.  The first phase (bounds) is not captured; each
// later call launches a phase's first long kernels directly, captures the
// rest from its stream and updates the executable graph in place when only
// parameters changed (re-instantiating it when the launch sequence changed),
// then launches it.  Calls with fewer points in all run without graphs.
constexpr long long kGraphMinPoints = 1 << 18;

struct PhaseGraphs {
    bool enabled = false;
    cudaGraphExec_t exec[4] = {};
    long long launches = 0, updates = 0, instantiations = 0;
    void release() {
        for (auto& e : exec)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    }
};

// Queues K instances on `st`.  The result of instance k will be in
// inst[k].labels / is_core (device pointers) once the stream reaches the
// end of the run; finish_batch then reports its status.  With a plan cache
// holding every instance's shape (and `allow_async`), nothing is read back
// while queueing; otherwise the driver waits for the bounds and for the
// neighbour-list sizes.  Returns the first error found while queueing; `info`
// and `tuning` may be null (defaults).
gd_status run_batch(MemProvider& mem, int K, const gd_instance* inst, cudaStream_t st, cudaEvent_t* events,
                    RunInfo* info, const Tuning* tuning, PhaseGraphs* graphs = nullptr,
                    cudaEvent_t* sort_events = nullptr, StageSet stage = StageSet(), bool allow_async = true);

// Waits for the run queued last on `st` by run_batch on this memory, reads
// its status words back and fills the sizes and views of `info`: GD_OK,
// GD_ETIMEOUT or GD_ERANGE; kGdRerun when the run must be queued again with
// exact sizes (a plan or capacity from an earlier call did not fit); the
// plan cache learns the run's sizes.
constexpr gd_status kGdRerun = (gd_status)100;
gd_status finish_batch(MemProvider& mem, int K, const gd_instance* inst, cudaStream_t st, RunInfo* info);

}  // namespace gd
