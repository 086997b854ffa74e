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
enum HostSlot { kHostSmall, kHostDesc, kHostSlots };

struct MemProvider {
    virtual ~MemProvider() {}
    // A device buffer of at least `bytes` for the slot (contents are not kept
    // when it has to grow).  GD_ENOMEM if it cannot be had.
    virtual gd_status device(int slot, size_t bytes, void** out) = 0;
    // A host staging buffer (pinned where possible) of at least `bytes`.
    virtual gd_status host(int slot, size_t bytes, void** out) = 0;
    // Single-pass neighbour walk: whether to try it, and the largest number of
    // neighbour entries per grid seen so far (sizes the pool; 0 = none yet).
    virtual bool pool_enabled() { return false; }
    virtual double nbr_per_grid() { return 0.0; }
    virtual void note_nbr_per_grid(double) {}
};

// Stage timing: when non-null, events[s] is recorded when stage s starts and
// events[kStages] at the end; stages that end at a read-back of sizes
// (bounds, compact, walk) also record events[kStages + 1 + i], i = 0, 1, 2,
// when their last kernel is issued, so that no stage includes host work.
constexpr int kStages = 11;
constexpr int kStageEvents = kStages + 4;
extern const char* const kStageNames[kStages];

// Kernel timing of the sort's downsweeps: when the driver is given sort
// events, it records a pair around each downsweep launch (at most
// kSortEventPairs) and reports how many pairs it used.
constexpr int kSortEventPairs = 48;

// What the driver reports about the run (instance 0 for the views).
struct RunInfo {
    long long sizes[12];
    const void* view_ptr[7];
    size_t view_bytes[7];
    long long launches;
    int sort_event_pairs = 0;
    // union-find retry cap for the run (0: the built-in kMaxUfRetries)
    int uf_cap = 0;
    // statistics of the run (summed over its instances) when asked for
    bool want_stats = false;
    bool have_stats = false;
    unsigned long long stats[kStatCount] = {};
    std::string error;
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

// Executable graphs of the driver's launch phases (the work between two reads
// of sizes), one per phase, kept by a context between calls.  The first phase
// (bounds) is not captured; each later call launches a phase's first long
// kernels directly, captures the rest from its stream and updates the
// executable graph in place when only parameters changed (re-instantiating
// it when the launch sequence changed), then launches it.
// Calls with fewer points in all run without graphs.
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

// Runs K instances.  The result of instance k is in inst[k].labels /
// is_core (device pointers).  Returns the first error; `info` and `tuning`
// may be null (defaults).
gd_status run_batch(MemProvider& mem, int K, const gd_instance* inst, cudaStream_t st, cudaEvent_t* events,
                    RunInfo* info, const Tuning* tuning, PhaseGraphs* graphs = nullptr,
                    cudaEvent_t* sort_events = nullptr);

}  // namespace gd
