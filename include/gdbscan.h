/*
 * gdbscan -- exact Euclidean DBSCAN on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library libgdbscan.so.  The method is GriT-DBSCAN
 * (Huang, Ma, Liu, Liu: "GriT-DBSCAN: A Spatial Clustering Algorithm for Very
 * Large Databases", arXiv 2210.07580): integer grid (Eq. 1, Alg. 1), grid-tree
 * neighbour query (Alg. 2-3), core identification as in G13 (Section 3.2),
 * core-grid merging decided by MinDist <= eps (Def. 6-7; Alg. 4-5) joined by
 * union-find (the LDF variant, Section 5.2) and border assignment (Alg. 6).
 *
 * Result definition (Section 3.1, Defs. 1-5), computed exactly:
 *   - N_eps(p) = { q : dist(p,q) <= eps }, p included; p is core iff
 *     |N_eps(p)| >= minpts.
 *   - Clusters are the connected components of the core points under
 *     dist <= eps.  A cluster's id is the smallest input index among its
 *     core points.
 *   - A non-core point within eps of a core point is a border point and takes
 *     the smallest id among the clusters of those core points; any other
 *     point is noise, label -1.
 *
 * Arithmetic: coordinates are int32; every comparison is the exact int64
 * squared distance against eps2.  For a real radius eps pass
 * eps2 = floor(eps^2): for integer points dist <= eps <=> dist2 <= eps2.
 *
 * Layout: points are row-major int32 [n][d] (point i at X[i*d .. i*d+d-1]).
 * labels is int32 [n], is_core is uint8 [n] (0/1), both in input order.
 *
 * Ownership: the caller owns X, labels and is_core.  A gd_ctx owns its device
 * workspace (grown on demand with cudaMalloc and kept for reuse), a small
 * pinned host staging area and timing events; gd_destroy frees them.  A
 * context is not thread-safe: use one per host thread.
 *
 * Errors: every entry point returns a gd_status; no exception or abort crosses
 * the ABI.  On an error other than GD_OK the outputs are unspecified and
 * gd_last_error() describes the failure.
 */
#ifndef GDBSCAN_H
#define GDBSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gd_ctx gd_ctx;

/* A CUDA stream handle (cudaStream_t); NULL means the legacy default stream. */
typedef void *gd_stream_t;

typedef enum {
    GD_OK = 0,
    GD_EINVAL = 1,   /* bad argument: d outside [1,8], n < 0 or n >= 2^31,
                        eps2 < 0, minpts < 1, NULL pointer with n > 0 */
    GD_ERANGE = 2,   /* d * (max_j (max x_j - min x_j))^2 >= 2^62, or the
                        packed grid key would need more than 128 bits */
    GD_ENOMEM = 3,   /* device or pinned host allocation failed */
    GD_ECUDA = 4,    /* a CUDA runtime call or kernel launch failed */
    GD_ETIMEOUT = 5, /* a bounded device-side retry loop hit its limit */
    GD_EBUSY = 6     /* reserved */
} gd_status;

/* Create a context on CUDA device `device` (made current by the call).
 * *out receives the context, or NULL on failure.  arena_bytes caps the device
 * memory the context may hold (its workspace and, for gd_dbscan_host, the
 * device copies); 0 means no cap.  A call that would need more returns
 * GD_ENOMEM and leaves the context usable with the buffers it held.  (The
 * paper has no counterpart: this is memory management of the GPU library.) */
gd_status gd_create(gd_ctx **out, int device, size_t arena_bytes);

/* Free the context and everything it owns.  NULL is ignored. */
void gd_destroy(gd_ctx *ctx);

/* Upper bound, in bytes, of the device workspace gd_dbscan needs for n points
 * in d dimensions before neighbour lists (which depend on the data: the
 * context grows them on demand).  Used for admission control.  (No
 * counterpart in the paper: memory sizing of the GPU library.) */
size_t gd_workspace_bytes(int64_t n, int d);

/* Exact DBSCAN of the device-resident points X (Section 4.4, Alg. 6: input
 * P, eps, MinPts; output the clustering).  X, labels and is_core are device
 * pointers (is_core may be NULL); labels and is_core must not overlap each
 * other or X (labels also serves as scratch during the call).
 *
 * Asynchronous: the work is queued on `stream` and the call returns; the
 * status of the clustering is deferred to gd_sync, and labels / is_core are
 * final once gd_sync has returned GD_OK (work queued on `stream` after
 * gd_sync sees them; X must stay unchanged until then).  When the context
 * has clustered an instance of the same n, d and eps2 before, the call reads
 * nothing back from the device while queueing; otherwise it waits twice for
 * sizes the data decides (the coordinate bounds, the neighbour-list sizes).
 * A context finishes its previous call before queueing a new one (a failure
 * of that call is reported by the next gd_sync).  The return value reports
 * errors found while queueing (bad arguments, GD_ENOMEM, GD_ECUDA, and
 * GD_ERANGE when the bounds were read back).  n == 0 is a no-op returning
 * GD_OK. */
gd_status gd_dbscan(gd_ctx *ctx, const int32_t *X, int64_t n, int d, int64_t eps2,
                    int32_t minpts, int32_t *labels, uint8_t *is_core, gd_stream_t stream);

/* Finishes the context's queued call, if any, and returns its deferred
 * status: GD_OK, GD_ETIMEOUT (a bounded union-find loop ran out), GD_ERANGE
 * (d * R^2 >= 2^62, found on the device), GD_ECUDA, or the failure of an
 * earlier call finished implicitly by a later one.  If sizes reused from an
 * earlier call did not fit the data, the call is run again with exact sizes
 * before gd_sync returns (the result is the same).  Blocks the host until
 * the call's work on its stream is done.  (The paper has no counterpart:
 * this is the boundary of the GPU library.) */
gd_status gd_sync(gd_ctx *ctx, gd_stream_t stream);

/* As gd_dbscan, with X, labels and is_core in HOST memory (pinned memory
 * makes the copies asynchronous and fast).  The call copies X to the device,
 * clusters, finishes (as gd_sync) and copies the results back before
 * returning: it is synchronous. */
gd_status gd_dbscan_host(gd_ctx *ctx, const int32_t *X_host, int64_t n, int d, int64_t eps2,
                         int32_t minpts, int32_t *labels_host, uint8_t *is_core_host,
                         gd_stream_t stream);

/* As gd_dbscan_host, asynchronous (no counterpart in the paper): the copy in,
 * the run and the copies out are queued on `stream` and the call returns;
 * labels_host / is_core_host hold the results once gd_sync(ctx, stream)
 * returns GD_OK (which waits for the copies out, and queues them again after
 * a run that had to be repeated with exact sizes).  X_host must stay
 * unchanged until then.  The next call on the context finishes this one
 * first, so calls alternating between two contexts on two streams overlap
 * one call's copies with the other's kernels. */
gd_status gd_dbscan_host_async(gd_ctx *ctx, const int32_t *X_host, int64_t n, int d, int64_t eps2,
                               int32_t minpts, int32_t *labels_host, uint8_t *is_core_host,
                               gd_stream_t stream);

/* One instance of a batch: device pointers and parameters as for gd_dbscan.
 *
 * eps2_yes selects approximate FastMerging (the Remark after Alg. 5, O(1)
 * rounds whatever eps and d): 0 (what a zero-initialised record holds) is
 * exact DBSCAN; a value >= eps2, normally floor((eps + delta)^2) for a
 * constant delta > 0, lets FastMerging answer "yes" for two core grids as
 * soon as it meets a pair of their core points at squared distance <=
 * eps2_yes.  Core flags, the pruning of FastMerging, every other merge test
 * and the border rule stay exact at eps2, so the clustering lies between
 * exact DBSCAN at eps and at eps + delta: every exact cluster's core points
 * fall in one cluster of the result, and every cluster of the result lies
 * in one cluster of DBSCAN at eps2_yes.  A value in (0, eps2) is GD_EINVAL. */
typedef struct {
    const int32_t *X;  /* [n][d] row-major, device */
    int64_t n;
    int d;
    int64_t eps2;
    int32_t minpts;
    int32_t *labels;   /* [n], device */
    uint8_t *is_core;  /* [n], device, or NULL */
    int64_t eps2_yes;  /* 0: exact; else approximate FastMerging's acceptance radius^2 */
} gd_instance;

/* Exact DBSCAN of k independent instances (uneven sizes, dimensions and
 * parameters) in one batch (no counterpart in the paper, which clusters one
 * data set: Alg. 6 applied to each instance).  Every stage of the pipeline is
 * one launch per group of instances (grouped by dimension or key width)
 * covering all of them.  Asynchronous like gd_dbscan (gd_sync finishes it;
 * nothing is read back while queueing when the context has seen every
 * instance's shape, else the host waits twice per batch, whatever k is).
 * Each instance's result equals gd_dbscan's on it alone.  `inst` is a host
 * array of k records (copied by the call); k == 0 is a no-op.  On error the
 * outputs of every instance are unspecified and gd_last_error names the
 * failing instance. */
gd_status gd_dbscan_batched(gd_ctx *ctx, int k, const gd_instance *inst, gd_stream_t stream);

/* Device bytes the context currently holds (workspace kept for reuse; no
 * counterpart in the paper, like the rest of the context management). */
size_t gd_ctx_bytes(const gd_ctx *ctx);

/* Release the context's cached device and pinned host buffers (they are
 * allocated again on the next call).  Waits for the context's last work. */
gd_status gd_ctx_trim(gd_ctx *ctx);

/* Static text for a status code. */
const char *gd_status_str(gd_status s);

/* Text of the last error seen by this context ("" if none). */
const char *gd_last_error(const gd_ctx *ctx);

/* ---------------------------------------------------------------------
 * Introspection of the last gd_dbscan call on a context (tests, tuning; no
 * counterpart in the paper).  These finish a queued call first.  The
 * arrays stay valid until the next call on the context.
 * ------------------------------------------------------------------- */

typedef enum {
    GD_VIEW_PERM = 0,        /* int32 [n]: input index of the k-th point in grid order */
    GD_VIEW_CELL_START = 1,  /* int32 [C+1]: first grid-order point of each grid */
    GD_VIEW_CELL_COORD = 2,  /* int32 [C][d]: grid identifiers (Eq. 1, relative to the minimum) */
    GD_VIEW_NBR_START = 3,   /* int32 [C+1]: CSR offsets of Nei(g) */
    GD_VIEW_NBR = 4,         /* int32 [nnbr]: neighbour grid indices, g itself included */
    GD_VIEW_CORE_SORTED = 5, /* uint8 [n]: core flags in grid order */
    GD_VIEW_CELL_CID = 6     /* int32 [C]: cluster id of each grid's core points, -1 if none */
} gd_view;

/* ---------------------------------------------------------------------
 * Tuning knobs (no counterpart in the paper: launch and tile shapes of the
 * GPU kernels).  A context resolves each knob for a group of instances of
 * dimension d whose largest instance has n points: the first table entry
 * with that knob, d (or 0 = any dimension) and n <= n_max gives the value;
 * without one the built-in default applies.  Every value gives the same
 * labels; only the speed changes.
 *
 *   GD_KNOB_MERGE_BUDGET  32x32 point tiles one warp tries on a candidate
 *                         pair of core grids before it hands the pair to the
 *                         block-level FastMerging kernel (Alg. 5); 1..64,
 *                         default 2.
 *   GD_KNOB_MERGE_LANE    pairs of core grids with at most this many point
 *                         pairs are decided by one lane; 1..256, default 16.
 *   GD_KNOB_MERGE_SMALL   pairs of core grids of at most this many core
 *                         points each are decided in full by one warp;
 *                         32..1024, default 128.
 *   GD_KNOB_CORE_BANDS    a point's neighbour grids are scanned nearest band
 *                         first when the list has at most this many grids;
 *                         0..65536, default 128.
 *   GD_KNOB_FM_BLOCKS     blocks of the FastMerging kernel; 152..19456,
 *                         default 1216 (per batch: resolved for the batch's
 *                         largest dimension and instance).
 *   GD_KNOB_WALK_BLOCKS   blocks of the neighbour walk (4 warps each);
 *                         152..19456, default 4864 (per batch, likewise).
 *   GD_KNOB_MERGE_ORDER   order in which candidate pairs of core grids are
 *                         tested: 0 = touching grids first, then the rest
 *                         (two waves); 1 = low density first (the LDF
 *                         variant of Section 5.2: one queue, pairs of grids
 *                         with fewer core points first); default 1
 *                         (per instance).
 *   GD_KNOB_CORE_MODE     how points of grids with fewer than minpts points
 *                         count their neighbours: 0 = a warp per point; 1 =
 *                         a warp per grid, which reads the grid's neighbour
 *                         list once for all its points; default 1 for d <= 4,
 *                         0 above (per group).
 *
 * Groups: instances of one dimension whose sizes fall in one bucket (at most
 * 2^12, 2^15, 2^18, 2^21 points, or more) are launched together and share
 * the per-group knobs.
 * --------------------------------------------------------------------- */
typedef enum {
    GD_KNOB_MERGE_BUDGET = 1,
    GD_KNOB_MERGE_LANE = 2,
    GD_KNOB_MERGE_SMALL = 3,
    GD_KNOB_CORE_BANDS = 4,
    GD_KNOB_FM_BLOCKS = 5,
    GD_KNOB_WALK_BLOCKS = 6,
    GD_KNOB_MERGE_ORDER = 7,
    GD_KNOB_CORE_MODE = 8
} gd_knob;

typedef struct {
    int32_t knob;  /* gd_knob */
    int32_t d;     /* dimension the entry applies to, 0 = any */
    int64_t n_max; /* applies to groups whose largest instance has <= n_max points */
    int32_t value;
} gd_tuning;

/* Replace the context's tuning table with a copy of entries[0..count)
 * (count = 0 clears it).  GD_EINVAL for an unknown knob, d outside [0,8],
 * n_max < 0, a value outside the knob's range, or more than 1024 entries;
 * the table is then unchanged. */
gd_status gd_set_tuning(gd_ctx *ctx, const gd_tuning *entries, int count);

/* The value a knob resolves to for dimension d and largest instance size n. */
gd_status gd_get_knob(const gd_ctx *ctx, int knob, int d, int64_t n, int32_t *value);

/* CUDA graphs (no counterpart in the paper).  A call reads sizes back from
 * the device three times, which splits its launches into four phases.  With
 * graphs on, the launches of the last three phases, after each phase's first
 * long kernels (launched directly, so that the device works while the host
 * captures), are captured from the call's stream into a graph that the
 * context keeps (one per phase): the next call updates it
 * in place when only launch parameters differ (re-instantiating it when the
 * launch sequence differs) and launches the phase as one graph (calls of
 * fewer than 2^18 points in all run without graphs: re-capturing would cost
 * more than it saves).  Results are identical either way.  Off by default for a new context; the stream must
 * not be capturing already.  gd_graph_stats: out[0] = graph launches,
 * out[1] = in-place updates, out[2] = instantiations, since creation. */
gd_status gd_set_graphs(gd_ctx *ctx, int enable);
gd_status gd_graph_stats(const gd_ctx *ctx, int64_t out[3]);

/* Sizes of the last run: out[0]=n, out[1]=d, out[2]=C (non-empty grids),
 * out[3]=nnbr (neighbour list length), out[4]=cell side s, out[5]=key bits,
 * out[6]=kernel launches of the run, out[7]=candidate merge pairs,
 * out[8]=radix-sort passes, out[9]=bits per digit, out[10]=pairs decided by
 * FastMerging, out[11]=sort key class (0: key and point index packed in one
 * 64-bit word, 1: 64-bit key + 32-bit index, 2: 128-bit key + 32-bit index),
 * out[12]=1 if the call was queued without reading anything back (the
 * context had planned every instance's shape), else 0; a call run again with
 * exact sizes reports 0.  Returns GD_EINVAL before any run. */
gd_status gd_last_sizes(gd_ctx *ctx, int64_t out[13]);

/* Copy `bytes` bytes of an internal array of the last run into host memory
 * (synchronous).  GD_EINVAL if bytes exceeds the array's size. */
gd_status gd_copy_view(gd_ctx *ctx, gd_view which, void *host_dst, size_t bytes);

/* Per-stage device timing (CUDA events around each stage of gd_dbscan).
 * Off by default; when on, gd_stage_times fills up to max entries of
 * milliseconds and names for the last run and returns the count: the 12
 * stages in order -- bounds, quantise, sort, compact, levels, walk, lists
 * (the neighbour lists placed from the walk's pool, or a second filling
 * walk), core, core_pack, merge_order, merge, labels -- (device time from a stage's first
 * launch to its last; the host's work between the call's phases is in none
 * of them), then
 * "sort_downsweep", the summed time of the radix sort's downsweep kernels
 * (part of the "sort" stage). */
gd_status gd_set_timing(gd_ctx *ctx, int enable);
int gd_stage_times(gd_ctx *ctx, float *ms, const char **names, int max);

/* Failure paths, for tests (no counterpart in the paper).
 *
 * gd_set_retry_limit: the number of iterations each lock-free union-find
 * loop of the merge (finds and CAS links) may take before it gives up and
 * the call returns GD_ETIMEOUT; 0 restores the built-in limit (2^20, far
 * above any legitimate count).  A tiny limit makes the bounded loops run out
 * on purpose; the device stays usable and the next call with the built-in
 * limit is exact again.
 *
 * gd_inject_alloc_failure: the k-th request for a device buffer that the
 * context makes from now on (counting every request, whether or not it needs
 * a new allocation) fails as a refused cudaMalloc would, with GD_ENOMEM; the
 * injection is then spent.  0 cancels it.  GD_EINVAL for k < 0. */
gd_status gd_set_retry_limit(gd_ctx *ctx, int32_t limit);
gd_status gd_inject_alloc_failure(gd_ctx *ctx, int32_t k);

/* Run statistics (no counterpart in the paper; the quantities are the ones
 * Section 4.3.3 and Section 5.2 discuss).  Off by default; when on, each call
 * counts, summed over its instances, and gd_run_stats fills up to max values
 * and names for the last call and returns the count (0 if the last call kept
 * none).  The counters, in order:
 *   pairs                candidate pairs of neighbouring core grids
 *   pairs_skipped        ... already in one union-find set (the LDF skip)
 *   pairs_box_no         ... decided "no" by the gap of the core boxes
 *   pairs_box_yes        ... decided "yes" by the core boxes' farthest corners
 *   pairs_lane           ... decided by one lane's exact loop
 *   pairs_warp           ... decided by a warp's exact tiles
 *   pairs_fastmerging    ... handed to FastMerging (Alg. 5); each of these ends
 *                        as fm_yes, fm_no or a later skip
 *   fm_yes, fm_no        FastMerging answers
 *   fm_pruned_triangle   points removed by Alg. 4's triangle test
 *   fm_pruned_angle      points removed by Alg. 4's angle test (Def. 8)
 *   nonfull_points       points of grids with fewer than minpts points
 *   count_rows           rows of their neighbour grids, once per such grid
 *   dist_core, dist_merge, dist_fastmerging, dist_labels
 *                        exact squared distances evaluated by core
 *                        counting, the warp-level merge, FastMerging and
 *                        border labelling
 *   walk_nodes           grid-tree nodes the neighbour query (Alg. 3) tested,
 *                        summed over query grids (each pair of grids is
 *                        enumerated from one side only)
 *   walk_steps           warp steps of that query (up to 32 nodes each)
 *   kappa_1 .. kappa_15, kappa_16_or_more
 *                        FastMerging calls by number of rounds (kappa of
 *                        Section 4.3.3)
 * Counting costs atomics: do not time calls that keep statistics. */
gd_status gd_set_stats(gd_ctx *ctx, int enable);
int gd_run_stats(gd_ctx *ctx, int64_t *values, const char **names, int max);

/* Throughput ceiling of the exact squared-distance test in d dimensions on
 * CUDA device `device` (no counterpart in the paper; for measurement).  Runs
 * the instruction mix of the merge's warp tiles -- a point broadcast by
 * shuffle, d int32 differences, d 64-bit squares summed, one compare -- from
 * registers only for a few tens of milliseconds and writes the best rate in
 * distances per second to *per_s.  The dist_* statistics over a stage's time
 * give that stage's ALU utilisation against this figure.  Allocates 4 bytes
 * of device memory for the duration of the call. */
gd_status gd_distance_peak(int device, int d, double *per_s);

/* ---------------------------------------------------------------------
 * Clustering without any device allocation (no counterpart in the paper).
 *
 * Some callers cannot call cudaMalloc when they need a clustering: a plugin
 * inside an application whose memory manager owns the whole device pool, a
 * real-time loop that forbids allocation (and the device-wide synchronisation
 * cudaFree implies) on its hot path, or a process whose allocator is already
 * exhausted.  gd_dbscan_noalloc serves them for small inputs.  It needs no
 * gd_ctx and calls no cudaMalloc, cudaFree, cudaMallocHost or other
 * allocating routine: every scratch buffer is carved from one file-scope
 * device array of GD_NOALLOC_SCRATCH_BYTES bytes.  The caller still provides
 * X, labels and is_core (device pointers, as for gd_dbscan), and the result
 * is bit-identical to gd_dbscan's.
 *
 *   - The array is backed on a GPU when the library's module is loaded there
 *     and is held until the process exits.  CUDA loads modules lazily by
 *     default, so that happens inside the first call on each device (with
 *     that device current; the call looks up the array's device address with
 *     cudaGetSymbolAddress).  Make one warm-up call per device at start-up,
 *     before the device's memory is committed elsewhere and before any
 *     stream capture.  If the device cannot back the array, the call returns
 *     GD_ENOMEM.
 *   - n above GD_NOALLOC_MAX_POINTS, or data whose neighbour lists do not fit
 *     in what the array has left, returns GD_ENOMEM (nothing is written);
 *     malformed arguments return GD_EINVAL as for gd_dbscan.
 *   - All calls share the one array and it keeps the previous call's
 *     contents; the pipeline clears whatever must start at zero.  Calls that
 *     overlapped on the GPU would race on the array: this function takes a
 *     process-wide lock and returns only after its work on `stream` has
 *     finished (on success and on failure), so calls made through it do not
 *     overlap.
 * --------------------------------------------------------------------- */
#define GD_NOALLOC_MAX_POINTS 65536
#define GD_NOALLOC_SCRATCH_BYTES (64u << 20)

gd_status gd_dbscan_noalloc(const int32_t *X, int64_t n, int d, int64_t eps2, int32_t minpts,
                            int32_t *labels, uint8_t *is_core, gd_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GDBSCAN_H */
