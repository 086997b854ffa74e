// Batched host driver of the exact-DBSCAN pipeline.
//
// The K instances go through every stage together: each launch covers a flat
// space over all of them (or over the ones sharing a dimension or a key
// width, for kernels specialised on those).  Sizes that only the data
// decides stay on the device: the grid count C (flat spaces over grids and
// the scans over per-grid arrays read it there), the pair counts, the
// non-full point counts and the FastMerging pairs.  The host must know
// before it launches
//   - the sort's launch plan (key class, digit passes), which depends on the
//     coordinate bounds, and
//   - the size of the neighbour lists and the largest grid (buffers).
// A call whose instance shapes (n, d, eps2) the context has seen takes both
// from that earlier call (plus margins) and is queued at once, with nothing
// read back: the device computes the real key layout and checks that it
// fits the plan and that the lists fit their buffers; if not, finish_batch
// asks for the call to be queued again with exact sizes.  Any other call
// reads the bounds back after the first phase and the list sizes after the
// third.  The device-side fit checks keep every kernel inside its buffers
// even when the data did not fit.
//
// Launch phases: 1. bounds (+ key layout); 2. keys, sort, compaction;
// 3. point boxes, grid tree, neighbour walk, list sizes; 4. lists, core
// points, merging, labels.
#include <climits>
#include <cstring>
#include <utility>

#include "pipeline.h"

namespace gd {

const char* const kStageNames[kStages] = {"bounds", "quantise",  "sort",        "compact", "levels", "walk",
                                          "lists",  "core",      "core_pack",   "merge_order", "merge", "labels"};

namespace {

int padded_dim(int d) { return d == 1 ? 1 : d == 2 ? 2 : d <= 4 ? 4 : 8; }

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

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host view of one instance.
struct HI {
    Inst dev;            // the record uploaded to the device
    long long C, maxcell, nnbr;  // read back (synchronous path) or bounds (queued path)
    int q_tiles, c_tiles;
    size_t arena_off, arena_bytes;
};

// Appends arrays to a host staging buffer; device pointers are the same
// offsets from the device descriptor buffer.
struct Builder {
    unsigned char* host;
    size_t cap, off;
    char* dev;  // device base (known after the buffer is obtained)
    bool overflow;
    size_t take(size_t bytes) {
        off = align256(off);
        const size_t at = off;
        if (off + bytes > cap) {
            overflow = true;
        } else {
            off += bytes;
        }
        return at;
    }
    template <typename T> T* hostp(T* devp) { return reinterpret_cast<T*>(host + ((char*)devp - dev)); }
};

// Fixed-capacity bump allocator over a host work buffer (no heap use).
struct HostBump {
    unsigned char* base;
    size_t cap, off;
    template <typename T> T* take(size_t count) {
        off = (off + 15) & ~(size_t)15;
        if (off + sizeof(T) * count > cap) return nullptr;
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

// Descriptor tables of a whole call (all phases).
size_t desc_bound(int K) { return (size_t)16384 * (size_t)(K + 16); }
size_t host_work_bound(int K) { return (size_t)(sizeof(HI) + 256) * (size_t)K + (size_t)64 * K * 8 + 65536; }
constexpr int kMaxFlatSpecs = 4 * kMaxD * kSizeBuckets + 16;

// Per-instance workspace, laid out from `base` (or only sized when base is
// null).  Arrays indexed by grid are sized for n grids, the upper bound.
size_t carve(Inst& I, char* base, int n, int d, int key_words, int key_bits) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = align256(off);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t N = (size_t)n, dp = (size_t)padded_dim(d);
    I.keyA = take(N * 8 * key_words);
    I.keyB = take(N * 8 * key_words);
    I.valA = (int*)take(N * 4);
    I.valB = (int*)take(N * 4);
    I.Xs = (int*)take(N * dp * 4);
    I.pt_cell = (int*)take(N * 4);
    I.core_s = (unsigned char*)take(N);
    I.Xc = (int*)take(N * dp * 4);
    I.cell_start = (int*)take((N + 1) * 4);
    I.cell_coord = (int*)take(N * d * 4);
    I.pbox = (int*)take(N * 2 * d * 4);
    for (int j = 0; j < kMaxD; ++j) {
        I.lv_key[j] = j < d ? (int*)take((N + 1) * 4) : nullptr;
        I.lv_cb[j] = j < d - 1 ? (int*)take((N + 2) * 4) : nullptr;
    }
    I.lv_E = (int*)take((size_t)d * (N + 1) * 4);
    I.lv_L = (int*)take(N * 4);
    I.nf_pts = I.lv_E;  // the level scratch is free once the levels are written
    I.nbr_start = (int*)take((N + 1) * 4);
    I.nbr_fwd = (int*)take(N * 4);
    I.nbr_bwd = (int*)take(N * 4);
    I.nf_start = (int*)take((N + 1) * 4);
    I.core_start = (int*)take((N + 1) * 4);
    I.bbox = (int*)take(N * 2 * d * 4);
    I.ldf_grid = (int*)take(N * 4);
    I.ldf_ctr = (int*)take(kLdfBuckets * 4);
    I.parent = (int*)take(N * 4);
    I.cid_root = (int*)take(N * 4);
    I.cell_cid = (int*)take(N * 4);
    I.bcnt = (int*)take(((N + kCompactTile - 1) / kCompactTile + 1) * 4);
    int* sort_base = (int*)take(sort_tmp_ints(n, key_words, key_bits) * 4);
    if (base) sort_tmp_layout(sort_base, n, key_words, key_bits, &I.sort_tcnt, &I.sort_ctot, &I.sort_dstart);
    return align256(off) + 256;
}

// The sort plan of a key layout (host side; the device computes the layout
// itself on the queued path and checks it against this plan).
void set_plan(HI& h, int key_words, int key_class, int key_bits) {
    Params& p = h.dev.p;
    p.key_bits = key_bits;
    p.key_words = key_words;
    p.key_class = key_class;
    const int ib = p.n > 1 ? bit_length((unsigned long long)(p.n - 1)) : 1;
    p.pack_bits = key_class == 0 ? ib : 0;
    // an in-cell offset is below s: d fields of bit_length(s - 1) bits each
    const int w = bit_length((unsigned long long)(p.s - 1));
    p.xoff_w = key_class == 0 && p.d * w <= 32 ? w : -1;
    const SortPlan sp = sort_plan(p.n, key_words, key_bits);
    h.dev.passes = sp.passes;
    h.dev.digit_bits = sp.bits;
    h.dev.tiles = sp.tiles;
}

#define RUN_TRY(x)                    \
    do {                              \
        gd_status s_ = (x);           \
        if (s_ != GD_OK) return s_;   \
    } while (0)
#define RUN_CUDA(x, what) RUN_TRY(cuda((x), what))

struct Run {
    MemProvider& mem;
    int K;
    const gd_instance* in;
    cudaStream_t st;
    cudaEvent_t* ev;
    RunInfo* info;
    const Tuning* tune;
    PhaseGraphs* graphs;
    cudaEvent_t* sort_ev;  // kSortEventPairs pairs, or null
    StageSet stage;
    bool allow_async;
    long long total_points = 0;
    int knob(int kn, int d, long long n) const { return tune ? tune->value(kn, d, n) : knob_default(kn, d); }

    // Runs the launches of phase `id`: head's directly, then body's either
    // directly or captured into the phase's executable graph and launched as
    // one graph.  The head (the phase's first long kernels) keeps the device
    // busy while the host captures and updates the graph of the rest.  A
    // capture that fails is discarded and the launches are issued directly.
    template <typename H, typename F> gd_status phase(int id, H&& head, F&& body) {
        RUN_TRY(head());
        // small batches re-capture more than they save in launches
        if (!graphs || !graphs->enabled || total_points < kGraphMinPoints) return body();
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return body();
        }
        const gd_status s = body();
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (s != GD_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (s != GD_OK) return s;
            return body();
        }
        cudaGraphExec_t& ex = graphs->exec[id];
        bool ready = false;
        if (ex) {
            cudaGraphExecUpdateResultInfo ri;
            if (cudaGraphExecUpdate(ex, g, &ri) == cudaSuccess) {
                ready = true;
                graphs->updates++;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(ex);
                ex = nullptr;
            }
        }
        if (!ready) {
            if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
                cudaGetLastError();
                ex = nullptr;
                cudaGraphDestroy(g);
                return body();
            }
            graphs->instantiations++;
        }
        cudaGraphDestroy(g);
        graphs->launches++;
        return cuda(cudaGraphLaunch(ex, st), "graph launch");
    }

    HI* hi = nullptr;
    int* hsmall = nullptr;   // host mirror of the small blocks [K][kSmallInts]
    int* dsmall = nullptr;   // device small blocks
    Builder b{};
    Inst* dins = nullptr;    // device Inst array (at the start of the descriptor buffer)
    int* scan_tmp = nullptr;
    size_t scan_tmp_ints = 0;
    HostBump hw{};
    int* all_idx = nullptr;  // 0..K-1
    size_t uploaded = 0;     // descriptor bytes already uploaded
    FlatSpec* spec_dev = nullptr;
    int nspecs = 0, specs_done = 0;

    gd_status fail(gd_status s, const char* msg, int k = -1) {
        if (info) {
            info->error = msg;
            if (k >= 0) info->error += " (instance " + std::to_string(k) + ")";
        }
        return s;
    }
    gd_status cuda(cudaError_t e, const char* where) {
        if (e == cudaSuccess) return GD_OK;
        if (info) info->error = std::string(where) + ": " + cudaGetErrorString(e);
        return GD_ECUDA;
    }
    void mark(int s) {
        if (ev) record_event(ev[s], st);
    }

    gd_status begin_desc() {
        void* h = nullptr;
        void* d = nullptr;
        const size_t cap = desc_bound(K);
        gd_status s = mem.host(stage.set ? kHostDesc1 : kHostDesc0, cap, &h);
        if (s != GD_OK) return fail(s, "descriptor staging");
        s = mem.device(kMemDesc, cap, &d);
        if (s != GD_OK) return fail(s, "descriptor buffer");
        b.host = (unsigned char*)h;
        b.cap = cap;
        b.off = 0;
        b.dev = (char*)d;
        b.overflow = false;
        // the Inst array always comes first, then the table of device-filled
        // flat spaces
        dins = reinterpret_cast<Inst*>(b.dev + b.take(sizeof(Inst) * K));
        spec_dev = reinterpret_cast<FlatSpec*>(b.dev + b.take(sizeof(FlatSpec) * kMaxFlatSpecs));
        nspecs = specs_done = 0;
        uploaded = 0;
        seg_tabs = 0;
        all_idx = nullptr;
        return GD_OK;
    }
    // Uploads the instance records, the table of device-filled spaces and
    // the tables built since the last upload (earlier ones are on the
    // device already, some with offsets the device has filled since).
    gd_status upload_desc() {
        if (b.overflow) return fail(GD_ENOMEM, "descriptor tables exceed their staging buffer");
        Inst* h = b.hostp(dins);
        for (int k = 0; k < K; ++k) h[k] = hi[k].dev;
        const size_t head = (size_t)((char*)(spec_dev + kMaxFlatSpecs) - b.dev);
        RUN_CUDA(cudaMemcpyAsync(b.dev, b.host, head, cudaMemcpyHostToDevice, st), "upload descriptors");
        const size_t from = uploaded > head ? uploaded : head;
        if (b.off > from)
            RUN_CUDA(cudaMemcpyAsync(b.dev + from, b.host + from, b.off - from, cudaMemcpyHostToDevice, st),
                     "upload descriptors");
        uploaded = b.off;
        return GD_OK;
    }
    const int* idx_all() {
        if (!all_idx) {
            int* t = b.hostp(reinterpret_cast<int*>(b.dev + b.take(sizeof(int) * K)));
            all_idx = reinterpret_cast<int*>(b.dev + ((unsigned char*)t - b.host));
            if (!b.overflow)
                for (int k = 0; k < K; ++k) t[k] = k;
        }
        return all_idx;
    }
    // Host-known flat space over `m` instances (members) with sizes size(k).
    template <typename F> Flat flat(const int* members, int m, F size, long long* total) {
        const size_t at_off = b.take(sizeof(long long) * (m + 1));
        const size_t at_idx = b.take(sizeof(int) * (m > 0 ? m : 1));
        long long run = 0;
        if (!b.overflow) {
            long long* off = reinterpret_cast<long long*>(b.host + at_off);
            int* idx = reinterpret_cast<int*>(b.host + at_idx);
            for (int t = 0; t < m; ++t) {
                off[t] = run;
                idx[t] = members[t];
                run += size(members[t]);
            }
            off[m] = run;
        } else {
            for (int t = 0; t < m; ++t) run += size(members[t]);
        }
        *total = run;
        return Flat{reinterpret_cast<const long long*>(b.dev + at_off), reinterpret_cast<const int*>(b.dev + at_idx),
                    m};
    }
    // Device-filled flat space over `m` members (offsets from count_flat).
    Flat dflat(const int* members, int m, long long** off_dev) {
        const size_t at_off = b.take(sizeof(long long) * (m + 1));
        const size_t at_idx = b.take(sizeof(int) * (m > 0 ? m : 1));
        if (!b.overflow) {
            int* idx = reinterpret_cast<int*>(b.host + at_idx);
            for (int t = 0; t < m; ++t) idx[t] = members[t];
            reinterpret_cast<long long*>(b.host + at_off)[0] = 0;
        }
        *off_dev = reinterpret_cast<long long*>(b.dev + at_off);
        return Flat{*off_dev, reinterpret_cast<const int*>(b.dev + at_idx), m};
    }
    // Flat space over the grids of `m` members, filled on the device once C
    // is known (count_pending); *upper receives a bound of its size (points).
    Flat gflat(const int* members, int m, long long* upper) {
        long long* off = nullptr;
        const Flat f = dflat(members, m, &off);
        long long u = 0;
        for (int t = 0; t < m; ++t) u += in[members[t]].n;
        *upper = u;
        if (nspecs >= kMaxFlatSpecs) {
            b.overflow = true;
        } else if (!b.overflow) {
            b.hostp(spec_dev)[nspecs] = FlatSpec{f.idx, off, m, kSmCells};
        }
        ++nspecs;
        return f;
    }
    gd_status count_pending() {
        if (nspecs > specs_done)
            RUN_CUDA(count_flats(dins, spec_dev + specs_done, nspecs - specs_done, st), "grid spaces");
        specs_done = nspecs;
        return GD_OK;
    }
    // Segmented scans over one array per member instance.
    // (longest segment of each table built since the descriptors were begun,
    // so that scan() can pick the one-launch form for short segments)
    const ScanSeg* seg_tab[128] = {};
    long long seg_longest[128] = {};
    int seg_tabs = 0;
    // tot_slot >= 0: each segment's total also goes to that slot of its
    // instance's small block.  len_slot >= 0: the segment's length is that
    // slot of the small block (read on the device); arr gives its bound.
    template <typename F>
    ScanSeg* segs(const int* members, int m, F arr, long long* tiles, int tot_slot = -1, int len_slot = -1) {
        const size_t at = b.take(sizeof(ScanSeg) * (m > 0 ? m : 1));
        long long blk = 0, longest = 0;
        ScanSeg* h = reinterpret_cast<ScanSeg*>(b.host + at);
        for (int t = 0; t < m; ++t) {
            int* a = nullptr;
            long long len = 0;
            arr(members[t], &a, &len);
            int* tot = tot_slot >= 0 ? dsmall + (size_t)members[t] * kSmallInts + tot_slot : nullptr;
            const int* ld = len_slot >= 0 ? dsmall + (size_t)members[t] * kSmallInts + len_slot : nullptr;
            if (!b.overflow) h[t] = ScanSeg{a, a, len, blk, tot, ld};
            blk += (len + kScanTile - 1) / kScanTile;
            if (len > longest) longest = len;
        }
        *tiles = blk;
        ScanSeg* dev = reinterpret_cast<ScanSeg*>(b.dev + at);
        if (seg_tabs < 128) {
            seg_tab[seg_tabs] = dev;
            seg_longest[seg_tabs++] = longest;
        }
        return dev;
    }
    gd_status scan(const ScanSeg* sg, int m, long long tiles) {
        if (tiles + m > (long long)scan_tmp_ints) return fail(GD_ENOMEM, "scan scratch too small");
        long long longest = -1;  // unknown: the three-launch form
        for (int i = 0; i < seg_tabs; ++i)
            if (seg_tab[i] == sg) longest = seg_longest[i];
        return cuda(scan_segments(sg, m, tiles, scan_tmp, st, longest), "scan");
    }
    gd_status readback() {
        gd_status s = cuda(cudaMemcpyAsync(hsmall, dsmall, sizeof(int) * kSmallInts * K, cudaMemcpyDeviceToHost, st),
                           "read back");
        if (s != GD_OK) return s;
        return cuda(cudaStreamSynchronize(st), "synchronise");
    }
    int* sm(int k) { return hsmall + (size_t)k * kSmallInts; }

    gd_status go();
};

gd_status Run::go() {
    // ---------------------------------------------------------- set-up
    // this call's host staging set: its previous user's uploads must be done
    if (stage.done) RUN_CUDA(cudaEventSynchronize(stage.done), "staging");
    void* hwp = nullptr;
    RUN_TRY(mem.host(stage.set ? kHostSmall1 : kHostSmall0, sizeof(int) * kSmallInts * K + host_work_bound(K), &hwp));
    hsmall = (int*)hwp;
    hw = HostBump{(unsigned char*)hwp + sizeof(int) * kSmallInts * K, host_work_bound(K), 0};
    hi = hw.take<HI>(K);
    int* members = hw.take<int>(K);
    int* members2 = hw.take<int>(K);
    if (!hi || !members || !members2) return fail(GD_ENOMEM, "host work buffer");
    void* dsm = nullptr;
    RUN_TRY(mem.device(kMemSmall, sizeof(int) * kSmallInts * K, &dsm));
    dsmall = (int*)dsm;
    unsigned long long* dstats = nullptr;
    if (info && info->want_stats) {
        void* sp = nullptr;
        RUN_TRY(mem.device(kMemStats, sizeof(unsigned long long) * kStatCount * K, &sp));
        dstats = (unsigned long long*)sp;
        RUN_CUDA(cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * kStatCount * K, st), "statistics");
    }

    PlanCache* pc = mem.plans();
    bool queued = allow_async && pc != nullptr;  // every shape planned by an earlier call
    long long total_pts = 0;
    int dmax = 1;
    bool any_ldf = false, all_ldf = true;
    bool small_eps = true;  // every instance's eps2 < 2^31: the walk's offsets fit 32 bits
    for (int k = 0; k < K; ++k) {
        const gd_instance& g = in[k];
        HI& h = hi[k];
        memset(&h, 0, sizeof(h));
        Params& p = h.dev.p;
        p.n = (int)g.n;
        p.d = g.d;
        p.dp = padded_dim(g.d);
        // Every squared distance is below 2^62 once the range check passes, so
        // a larger eps2 changes nothing; clamping keeps the gap sums in range.
        const long long cap = (1ll << 62) - 1;
        p.eps2 = g.eps2 > cap ? cap : g.eps2;
        p.eps2_yes = g.eps2_yes <= p.eps2 ? p.eps2 : (g.eps2_yes > cap ? cap : g.eps2_yes);
        p.minpts = g.minpts;
        p.ldf = knob(GD_KNOB_MERGE_ORDER, g.d, g.n);
        p.uf_cap = info && info->uf_cap > 0 ? info->uf_cap : kMaxUfRetries;
        p.s = 1 + (long long)isqrt_u64((unsigned long long)p.eps2 / (unsigned long long)g.d);
        p.s_mul = p.s >= 2 ? ~0ull / (unsigned long long)p.s + 1 : 0;
        p.r = p.eps2 == 0 ? 0 : 1 + ((long long)isqrt_u64((unsigned long long)p.eps2) - 1) / p.s;
        if (p.r > kMaxR) return fail(GD_ERANGE, "stencil radius above its bound", k);
        h.dev.X = g.X;
        h.dev.labels = g.labels;
        h.dev.is_core = g.is_core;
        h.dev.small = dsmall + (size_t)k * kSmallInts;
        h.dev.stats = dstats ? dstats + (size_t)k * kStatCount : nullptr;
        int* s = sm(k);
        memset(s, 0, sizeof(int) * kSmallInts);
        for (int j = 0; j < kMaxD; ++j) {
            s[kSmMnmx + j] = INT_MAX;
            s[kSmMnmx + kMaxD + j] = INT_MIN;
        }
        total_pts += g.n;
        if (g.d > dmax) dmax = g.d;
        if (p.ldf) any_ldf = true;
        else all_ldf = false;
        if (p.eps2 >= (1ll << 31)) small_eps = false;
        if (queued) {
            const ShapePlan* sp = pc->find(g.n, g.d, p.eps2);
            if (!sp || sp->key_bits <= 0) {
                queued = false;
            } else {
                set_plan(h, sp->key_words, sp->key_class, sp->key_bits);
                // capacities: what the shape needed last time, plus a margin
                h.nnbr = sp->nnbr + sp->nnbr / 4 + 4096;
                h.maxcell = sp->maxcell + sp->maxcell / 4 + 32;
            }
        }
    }
    if (info) {
        info->queued_async = queued;
        info->sizes[12] = queued ? 1 : 0;
    }
    auto note_plan = [&]() {
        for (int k = 0; k < K; ++k) {
            sm(k)[kSmKeyClass] = hi[k].dev.p.key_class;
            sm(k)[kSmKeyBits] = hi[k].dev.p.key_bits;
            sm(k)[kSmKeyWords] = hi[k].dev.p.key_words;
        }
    };
    if (queued) note_plan();
    // scan scratch: enough for any segmented scan of the batch
    scan_tmp_ints = (size_t)K + 64;
    for (int k = 0; k < K; ++k) scan_tmp_ints += (size_t)(in[k].n / kScanTile + 2);
    void* stp = nullptr;
    RUN_TRY(mem.device(kMemScanTmp, scan_tmp_ints * 4, &stp));
    scan_tmp = (int*)stp;
    total_points = total_pts;
    for (int k = 0; k < K; ++k) members[k] = k;
    auto n_of = [&](int k) { return (long long)in[k].n; };
    long long tot;
    long long n_largest = 1;
    for (int k = 0; k < K; ++k) n_largest = in[k].n > n_largest ? in[k].n : n_largest;
    const int fm_blocks = knob(GD_KNOB_FM_BLOCKS, dmax, n_largest);
    const bool uf_capped = info && info->uf_cap > 0;  // a lowered union-find cap (tests)
    const int walk_blocks = knob(GD_KNOB_WALK_BLOCKS, dmax, n_largest);

    // ------------------------------------------------ phase 1: bounds
    RUN_TRY(begin_desc());
    Flat pts_d[kMaxD];
    long long tot_d[kMaxD] = {};
    for (int d = 1; d <= kMaxD; ++d) {
        int m = 0;
        for (int k = 0; k < K; ++k)
            if (in[k].d == d) members2[m++] = k;
        pts_d[d - 1] = flat(members2, m, n_of, &tot_d[d - 1]);
    }
    auto launch1 = [&]() -> gd_status {
        mark(0);
        RUN_CUDA(cudaMemcpyAsync(dsmall, hsmall, sizeof(int) * kSmallInts * K, cudaMemcpyHostToDevice, st), "init");
        for (int d = 1; d <= kMaxD; ++d)
            RUN_CUDA(launch_bounds(dins, pts_d[d - 1], tot_d[d - 1], d, st), "bounds");
        if (queued) RUN_CUDA(launch_layout(dins, K, st), "key layout");
        mark(kStages + 1);
        return GD_OK;
    };
    if (!queued) {
        RUN_TRY(upload_desc());
        RUN_TRY(launch1());
        RUN_TRY(readback());
        // the key layout and sort plan of each instance from its bounds
        for (int k = 0; k < K; ++k) {
            HI& h = hi[k];
            Params& p = h.dev.p;
            const int* s = sm(k);
            unsigned long long rmax = 0;
            int total_bits = 0;
            for (int j = 0; j < p.d; ++j) {
                const long long lo = s[kSmMnmx + j], up = s[kSmMnmx + kMaxD + j];
                const unsigned long long rj = (unsigned long long)(up - lo);
                if (rj > rmax) rmax = rj;
                p.mn[j] = (int)lo;
                p.bits[j] = bit_length(rj / (unsigned long long)p.s);
                total_bits += p.bits[j];
            }
            if ((unsigned __int128)p.d * rmax * rmax >= ((unsigned __int128)1 << 62))
                return fail(GD_ERANGE, "coordinate range too large: d * R^2 >= 2^62", k);
            if (total_bits > 128) return fail(GD_ERANGE, "packed grid key needs more than 128 bits", k);
            for (int j = p.d - 1, sh = 0; j >= 0; --j) {
                p.shift[j] = sh;
                sh += p.bits[j];
            }
            const int kw = total_bits <= 64 ? 1 : 2;
            const int ib = p.n > 1 ? bit_length((unsigned long long)(p.n - 1)) : 1;
            set_plan(h, kw, kw == 2 ? 2 : (total_bits + ib <= 64 ? 0 : 1), total_bits);
        }
        // the plans into the small blocks (read back with the results)
        note_plan();
        RUN_CUDA(cudaMemcpyAsync(dsmall, hsmall, sizeof(int) * kSmallInts * K, cudaMemcpyHostToDevice, st), "plans");
    }

    // workspaces of the plan
    int max_buckets = 1;
    size_t arena = 0;
    for (int k = 0; k < K; ++k) {
        HI& h = hi[k];
        Params& p = h.dev.p;
        h.q_tiles = (p.n + kQuantTile - 1) / kQuantTile;
        h.c_tiles = (p.n + kCompactTile - 1) / kCompactTile;
        const int R = 1 << h.dev.digit_bits;
        if (R > max_buckets) max_buckets = R;
        h.arena_off = arena;
        h.arena_bytes = carve(h.dev, nullptr, p.n, p.d, p.key_words, p.key_bits);
        arena += h.arena_bytes;
    }
    void* ap = nullptr;
    RUN_TRY(mem.device(kMemArena, arena, &ap));
    for (int k = 0; k < K; ++k) {
        HI& h = hi[k];
        carve(h.dev, (char*)ap + h.arena_off, h.dev.p.n, h.dev.p.d, h.dev.p.key_words, h.dev.p.key_bits);
    }

    // ------------------------- phase 2: keys, sort, compaction
    const Flat pts1 = flat(members, K, n_of, &tot);
    // one group per key class (packed 64-bit, 64-bit + values, 128-bit + values)
    Flat qflat[3], cflat[3];
    long long qtot[3] = {0, 0, 0}, ctot[3] = {0, 0, 0};
    Flat oflat[3][16], chflat[3][16];
    long long otot[3][16] = {}, chtot[3][16] = {};
    int gpasses[3] = {0, 0, 0};
    for (int w = 0; w < 3; ++w) {
        int m = 0;
        for (int k = 0; k < K; ++k)
            if (hi[k].dev.p.key_class == w) members2[m++] = k;
        qflat[w] = flat(members2, m, [&](int k) { return (long long)hi[k].q_tiles; }, &qtot[w]);
        cflat[w] = flat(members2, m, [&](int k) { return (long long)hi[k].c_tiles; }, &ctot[w]);
        for (int t = 0; t < m; ++t)
            if (hi[members2[t]].dev.passes > gpasses[w]) gpasses[w] = hi[members2[t]].dev.passes;
        for (int ps = 0; ps < gpasses[w]; ++ps) {
            int m2 = 0;
            for (int t = 0; t < m; ++t)
                if (hi[members2[t]].dev.passes > ps) members[m2++] = members2[t];
            oflat[w][ps] = flat(members, m2, [&](int k) { return (long long)hi[k].dev.tiles; }, &otot[w][ps]);
            chflat[w][ps] = flat(
                members, m2, [&](int k) { return (long long)(hi[k].dev.tiles + kSortChunk - 1) / kSortChunk; },
                &chtot[w][ps]);
        }
    }
    for (int k = 0; k < K; ++k) members[k] = k;
    long long cseg_tiles = 0;
    const ScanSeg* cseg = segs(
        members, K,
        [&](int k, int** a, long long* len) {
            *a = hi[k].dev.bcnt;
            *len = hi[k].c_tiles;
        },
        &cseg_tiles);
    const int* idx = idx_all();
    RUN_CUDA(prepare_sort(), "sort set-up");
    auto launch2 = [&]() -> gd_status {
        return phase(1, [&]() -> gd_status {
        mark(1);
        for (int w = 0; w < 3; ++w) RUN_CUDA(launch_quantise(dins, qflat[w], qtot[w], w, st), "quantise");
        return GD_OK;
        }, [&]() -> gd_status {
        mark(2);
        int pairs = 0;
        for (int w = 0; w < 3; ++w)
            for (int ps = 0; ps < gpasses[w]; ++ps) {
                cudaEvent_t a = nullptr, b2 = nullptr;
                if (sort_ev && otot[w][ps] > 0 && pairs < kSortEventPairs) {
                    a = sort_ev[2 * pairs];
                    b2 = sort_ev[2 * pairs + 1];
                    ++pairs;
                }
                RUN_CUDA(launch_sort_pass(dins, oflat[w][ps], otot[w][ps], chflat[w][ps], chtot[w][ps], w, ps,
                                          max_buckets, st, a, b2),
                         "sort pass");
            }
        if (info) info->sort_event_pairs = pairs;
        mark(3);
        for (int w = 0; w < 3; ++w) RUN_CUDA(launch_compact_count(dins, cflat[w], ctot[w], w, st), "compact count");
        RUN_TRY(scan(cseg, K, cseg_tiles));
        for (int w = 0; w < 3; ++w) RUN_CUDA(launch_compact_write(dins, cflat[w], ctot[w], w, st), "compact write");
        RUN_CUDA(launch_cell_max(dins, pts1, total_pts, st), "largest grid");
        mark(kStages + 2);
        return GD_OK;
        });
    };

    // --------------------------- phase 3: levels, walk, list sizes
    long long total_cells = 0;  // bound of the grids (points)
    const Flat cells = gflat(members, K, &total_cells);
    // the walk is specialised on the dimension: one launch per dimension
    // present (the grids of all instances when there is one)
    Flat wflat[kMaxD + 1];
    long long wtot[kMaxD + 1] = {};
    for (int dd = 1; dd <= kMaxD; ++dd) {
        int m = 0;
        for (int k = 0; k < K; ++k)
            if (hi[k].dev.p.d == dd) members2[m++] = k;
        if (m == 0) continue;
        if (m == K) {
            wflat[dd] = cells;
            wtot[dd] = total_cells;
        } else {
            wflat[dd] = gflat(members2, m, &wtot[dd]);
        }
    }
    Flat lflat[kMaxD];
    long long ltot[kMaxD] = {};
    const ScanSeg* lseg[kMaxD] = {};
    long long lseg_tiles[kMaxD] = {};
    int lm[kMaxD] = {};
    for (int j = 0; j + 1 < dmax; ++j) {
        int m = 0;
        for (int k = 0; k < K; ++k)
            if (hi[k].dev.p.d - 1 > j) members2[m++] = k;
        lm[j] = m;
        lflat[j] = gflat(members2, m, &ltot[j]);
        lseg[j] = segs(
            members2, m,
            [&](int k, int** a, long long* len) {
                *a = hi[k].dev.lv_E + (size_t)j * ((size_t)in[k].n + 1);
                *len = in[k].n;
            },
            &lseg_tiles[j], -1, kSmCells);
    }
    long long nseg_tiles = 0;
    const ScanSeg* nseg = segs(
        members, K,
        [&](int k, int** a, long long* len) {
            *a = hi[k].dev.nbr_start;
            *len = in[k].n;
        },
        &nseg_tiles, kSmNnbr, kSmCells);

    // Single-pass walk when a pool can be had: sized from the most pool
    // entries and runs per point this memory has seen (a first call guesses).
    WalkPool pool{};
    if (mem.pool_enabled()) {
        const double per = mem.pool_per_point() > 0 ? mem.pool_per_point() * 1.25 : 4.0;
        const double runs = mem.runs_per_point() > 0 ? mem.runs_per_point() * 1.25 : 0.25;
        const long long cap = (long long)(per * (double)total_pts) + 4096;
        const long long seg_cap = (long long)(runs * (double)total_pts) + cap / 32 + 64;
        void *pd = nullptr, *ps = nullptr;
        if (cap < (1ll << kPoolBits) && seg_cap < (1ll << (64 - kPoolBits)) &&
            mem.device(kMemPool, (size_t)cap * 4, &pd) == GD_OK &&
            mem.device(kMemPoolSeg, (size_t)seg_cap * sizeof(PoolSeg), &ps) == GD_OK) {
            pool = WalkPool{(int*)pd, (PoolSeg*)ps, (unsigned long long*)(dsmall + kSmPool), cap, seg_cap};
        }
    }
    const bool pooled = pool.data != nullptr;
    auto walk_all = [&](int mode) -> gd_status {
        for (int dd = 1; dd <= kMaxD; ++dd)
            if (wtot[dd] > 0)
                RUN_CUDA(launch_walk(dins, wflat[dd], wtot[dd], mode, pool, walk_blocks, small_eps, dd, st), "walk");
        return GD_OK;
    };
    // whether the lists need the filling walk (the pool was too small or
    // absent): known after phase 3 on the synchronous path, else always
    // launched (it returns at once when the pool held the walk)
    bool need_fill = true;
    auto launch3 = [&]() -> gd_status {
        return phase(2, [&]() -> gd_status {
        mark(4);
        RUN_TRY(count_pending());
        RUN_CUDA(launch_point_boxes(dins, cells, total_cells, st), "point boxes");
        RUN_CUDA(launch_level_diff(dins, cells, total_cells, st), "levels");
        return GD_OK;
        }, [&]() -> gd_status {
        for (int j = 0; j + 1 < dmax; ++j) {
            RUN_CUDA(launch_level_flag(dins, lflat[j], ltot[j], j, st), "level flags");
            RUN_TRY(scan(lseg[j], lm[j], lseg_tiles[j]));
        }
        RUN_CUDA(launch_level_write(dins, cells, total_cells, st), "level write");
        mark(5);
        RUN_TRY(walk_all(pooled ? kWalkPool : kWalkCount));
        RUN_CUDA(launch_nbr_total(dins, cells, total_cells, st), "list lengths");
        RUN_TRY(scan(nseg, K, nseg_tiles));
        RUN_CUDA(launch_nbr_check(dins, cells, total_cells, st), "list capacity");
        mark(kStages + 3);
        return GD_OK;
        });
    };

    // sizes of the lists and of the FastMerging bitmaps: exact (read back
    // after phase 3) or from the shape's earlier call
    void* scr = nullptr;
    int wpb = 1;
    auto size_lists = [&]() -> gd_status {
        long long total_nbr = 0, max_cell = 1;
        for (int k = 0; k < K; ++k) {
            if (hi[k].nnbr >= INT_MAX) return fail(GD_ERANGE, "neighbour lists exceed 2^31 entries", k);
            total_nbr += hi[k].nnbr;
            if (hi[k].maxcell > max_cell) max_cell = hi[k].maxcell;
        }
        wpb = (int)((max_cell + 31) / 32 + 1);
        RUN_TRY(mem.device(kMemScratch, (size_t)fm_blocks * 2 * wpb * 4, &scr));
        void *nbp = nullptr, *hp = nullptr;
        // hard pairs: each candidate pair at most once, at most one per list entry
        RUN_TRY(mem.device(kMemNbr, (size_t)total_nbr * 4 + 256 * (size_t)K + 256, &nbp));
        RUN_TRY(mem.device(kMemHard, (size_t)total_nbr * 8 + 256 * (size_t)K + 256, &hp));
        size_t o4 = 0, o8 = 0;
        for (int k = 0; k < K; ++k) {
            hi[k].dev.nbr = (int*)((char*)nbp + o4);
            hi[k].dev.hard = (int2*)((char*)hp + o8);
            hi[k].dev.nbr_cap = hi[k].nnbr;
            o4 += align256((size_t)hi[k].nnbr * 4);
            o8 += align256((size_t)hi[k].nnbr * 8);
        }
        return GD_OK;
    };

    // ------------- phase 4: lists, core, merge, labels
    // groups of instances by dimension and size bucket: the kernels that
    // take the dimension as a template argument, and the tuning knobs, go by
    // group
    constexpr int kGroups = kMaxD * kSizeBuckets;
    int dgroups[kGroups], gbucket[kGroups], ng = 0;
    long long gn[kGroups];
    for (int d = 1; d <= kMaxD; ++d)
        for (int bk = 0; bk < kSizeBuckets; ++bk) {
            long long nmax = 0;
            for (int k = 0; k < K; ++k)
                if (hi[k].dev.p.d == d && size_bucket(in[k].n) == bk && in[k].n > nmax) nmax = in[k].n;
            if (nmax > 0) {
                dgroups[ng] = d;
                gbucket[ng] = bk;
                gn[ng++] = nmax;
            }
        }
    Flat g_pts[kGroups], g_cells[kGroups], g_nf[kGroups], g_hard[2][kGroups];
    long long* g_nf_off[kGroups];
    long long* g_hard_off[2][kGroups];
    long long g_pts_tot[kGroups], g_cells_tot[kGroups];
    int g_m[kGroups];
    const int* g_idx[kGroups];
    long long coreseg_tiles = 0, nfseg_tiles = 0;
    const ScanSeg* coreseg = nullptr;
    const ScanSeg* nfseg = nullptr;
    auto build4 = [&]() {
        for (int gi = 0; gi < ng; ++gi) {
            int m = 0;
            for (int k = 0; k < K; ++k)
                if (hi[k].dev.p.d == dgroups[gi] && size_bucket(in[k].n) == gbucket[gi]) members2[m++] = k;
            g_m[gi] = m;
            g_pts[gi] = flat(members2, m, n_of, &g_pts_tot[gi]);
            g_cells[gi] = gflat(members2, m, &g_cells_tot[gi]);
            g_idx[gi] = g_pts[gi].idx;
            g_nf[gi] = dflat(members2, m, &g_nf_off[gi]);
            for (int w = 0; w < 2; ++w) g_hard[w][gi] = dflat(members2, m, &g_hard_off[w][gi]);
        }
        auto arr_seg = [&](int* Inst::*field, int tot_slot, long long* tiles) {
            return segs(
                members, K,
                [&](int k, int** a, long long* len) {
                    *a = hi[k].dev.*field;
                    *len = in[k].n;
                },
                tiles, tot_slot, kSmCells);
        };
        nfseg = arr_seg(&Inst::nf_start, kSmNonfull, &nfseg_tiles);
        coreseg = arr_seg(&Inst::core_start, -1, &coreseg_tiles);
    };
    auto launch4 = [&]() -> gd_status {
        return phase(3, [&]() -> gd_status {
        RUN_TRY(count_pending());
        mark(6);
        // the lists: from the pool's runs, or (the pool too small, or none) by
        // a second, filling walk -- the device decides
        RUN_CUDA(launch_pool_scatter(dins, pool, st), "neighbour scatter");
        if (need_fill) RUN_TRY(walk_all(kWalkFill));
        mark(7);
        RUN_CUDA(launch_core_full(dins, cells, total_cells, st), "core (full grids)");
        return GD_OK;
        }, [&]() -> gd_status {
        // a warp per point (the non-full points as a flat space, scanned on
        // the device) or a warp per grid, per group
        bool any_point_mode = false;
        for (int gi = 0; gi < ng; ++gi)
            if (!knob(GD_KNOB_CORE_MODE, dgroups[gi], gn[gi])) any_point_mode = true;
        if (any_point_mode) {
            RUN_CUDA(launch_nonfull_count(dins, cells, total_cells, st), "non-full grids");
            RUN_TRY(scan(nfseg, K, nfseg_tiles));
            for (int gi = 0; gi < ng; ++gi)
                if (!knob(GD_KNOB_CORE_MODE, dgroups[gi], gn[gi]))
                    RUN_CUDA(launch_nf_index(dins, g_cells[gi], g_cells_tot[gi], st), "non-full points");
        }
        for (int gi = 0; gi < ng; ++gi) {
            const int d = dgroups[gi], bands = knob(GD_KNOB_CORE_BANDS, d, gn[gi]);
            if (knob(GD_KNOB_CORE_MODE, d, gn[gi])) {
                RUN_CUDA(launch_core_grid(dins, g_cells[gi], g_cells_tot[gi], d, bands, st), "core (counting)");
            } else {
                RUN_CUDA(count_flat(dins, g_idx[gi], g_m[gi], kSmNonfull, g_nf_off[gi], st), "flat offsets");
                RUN_CUDA(launch_core_point(dins, g_nf[gi], d, bands, st), "core (counting)");
            }
        }
        if (info && info->want_stats) RUN_CUDA(launch_core_stats(dins, cells, total_cells, st), "core statistics");
        mark(8);
        RUN_CUDA(launch_core_count(dins, cells, total_cells, st), "core count");
        RUN_TRY(scan(coreseg, K, coreseg_tiles));
        for (int gi = 0; gi < ng; ++gi)
            RUN_CUDA(launch_core_pack(dins, g_cells[gi], g_cells_tot[gi], dgroups[gi], st), "core pack");
        mark(9);
        if (any_ldf) RUN_CUDA(launch_ldf_order(dins, idx, K, cells, total_cells, st), "low-density-first order");
        RUN_CUDA(launch_uf_init(dins, cells, total_cells, st), "union-find init");
        mark(10);
        for (int w = 0; w < 2; ++w) {
            if (w == 1 && all_ldf) break;  // one wave in the low-density-first order
            for (int gi = 0; gi < ng; ++gi) {
                const int d = dgroups[gi];
                RUN_CUDA(launch_merge_list(dins, g_cells[gi], g_cells_tot[gi], w, d,
                                           knob(GD_KNOB_MERGE_BUDGET, d, gn[gi]), knob(GD_KNOB_MERGE_LANE, d, gn[gi]),
                                           knob(GD_KNOB_MERGE_SMALL, d, gn[gi]), uf_capped, st),
                         "merge (warp)");
            }
            for (int gi = 0; gi < ng; ++gi) {
                RUN_CUDA(count_flat(dins, g_idx[gi], g_m[gi], kSmHard0 + w, g_hard_off[w][gi], st), "flat offsets");
                RUN_CUDA(launch_merge_block(dins, g_hard[w][gi], w, dgroups[gi], fm_blocks, (unsigned*)scr, wpb, uf_capped,
                                            st),
                         "merge (FastMerging)");
            }
            if (w == 0 && !all_ldf)
                RUN_CUDA(launch_uf_flatten(dins, cells, total_cells, uf_capped, st), "union-find flatten");
        }
        mark(11);
        RUN_CUDA(launch_cluster_ids(dins, cells, total_cells, uf_capped, st), "cluster ids");
        for (int gi = 0; gi < ng; ++gi)
            RUN_CUDA(launch_labels(dins, g_pts[gi], g_pts_tot[gi], dgroups[gi], st), "labels");
        mark(12);
        return GD_OK;
        });
    };

    if (queued) {
        // everything is known: one upload, then the four phases back to back
        RUN_TRY(size_lists());
        build4();
        RUN_TRY(upload_desc());
        if (stage.done) RUN_CUDA(cudaEventRecord(stage.done, st), "staging");
        RUN_TRY(launch1());
        RUN_TRY(launch2());
        RUN_TRY(launch3());
        RUN_TRY(launch4());
    } else {
        for (int k = 0; k < K; ++k) hi[k].dev.nbr_cap = LLONG_MAX;  // phase 3 writes no list
        RUN_TRY(upload_desc());
        RUN_TRY(launch2());
        RUN_TRY(launch3());
        RUN_TRY(readback());
        for (int k = 0; k < K; ++k) {
            hi[k].C = sm(k)[kSmCells];
            hi[k].maxcell = sm(k)[kSmMaxCell];
            hi[k].nnbr = (unsigned)sm(k)[kSmNnbr];
        }
        if (pooled) {
            unsigned long long ctr;
            memcpy(&ctr, sm(0) + kSmPool, sizeof(ctr));
            need_fill = (long long)(ctr & ((1ull << kPoolBits) - 1)) > pool.cap ||
                        (long long)(ctr >> kPoolBits) > pool.seg_cap;
        }
        RUN_TRY(size_lists());
        build4();
        RUN_TRY(upload_desc());
        if (stage.done) RUN_CUDA(cudaEventRecord(stage.done, st), "staging");
        RUN_TRY(launch4());
    }

    if (info) {
        // what is known now; finish_batch adds the sizes the device found
        const HI& h = hi[0];
        const int n = h.dev.p.n, d = h.dev.p.d;
        info->sizes[0] = n;
        info->sizes[1] = d;
        info->sizes[4] = h.dev.p.s;
        info->sizes[5] = h.dev.p.key_bits;
        info->sizes[8] = h.dev.passes;
        info->sizes[9] = h.dev.digit_bits;
        info->sizes[11] = h.dev.p.key_class;
        info->view_ptr[GD_VIEW_PERM] = (h.dev.passes & 1) ? h.dev.valB : h.dev.valA;
        info->view_ptr[GD_VIEW_CELL_START] = h.dev.cell_start;
        info->view_ptr[GD_VIEW_CELL_COORD] = h.dev.cell_coord;
        info->view_ptr[GD_VIEW_NBR_START] = h.dev.nbr_start;
        info->view_ptr[GD_VIEW_NBR] = h.dev.nbr;
        info->view_ptr[GD_VIEW_CORE_SORTED] = h.dev.core_s;
        info->view_ptr[GD_VIEW_CELL_CID] = h.dev.cell_cid;
    }
    return GD_OK;
}

}  // namespace

int knob_default(int knob, int d) {
    switch (knob) {
        case GD_KNOB_MERGE_BUDGET: return 2;
        case GD_KNOB_MERGE_LANE: return 16;
        case GD_KNOB_MERGE_SMALL: return 128;
        case GD_KNOB_CORE_BANDS: return 128;
        case GD_KNOB_FM_BLOCKS: return 152 * 8;
        case GD_KNOB_WALK_BLOCKS: return 152 * 32;
        case GD_KNOB_MERGE_ORDER: return 1;
        case GD_KNOB_CORE_MODE: return d <= 4 ? 1 : 0;
        default: return -1;
    }
}

bool knob_in_range(int knob, int v) {
    switch (knob) {
        case GD_KNOB_MERGE_BUDGET: return v >= 1 && v <= 64;
        case GD_KNOB_MERGE_LANE: return v >= 1 && v <= 256;
        case GD_KNOB_MERGE_SMALL: return v >= 32 && v <= 1024;
        case GD_KNOB_CORE_BANDS: return v >= 0 && v <= 65536;
        case GD_KNOB_FM_BLOCKS:
        case GD_KNOB_WALK_BLOCKS: return v >= 152 && v <= 152 * 128;
        case GD_KNOB_MERGE_ORDER: return v == 0 || v == 1;
        case GD_KNOB_CORE_MODE: return v == 0 || v == 1;
        default: return false;
    }
}

int Tuning::value(int knob, int d, long long n) const {
    for (int i = 0; i < count; ++i)
        if (e[i].knob == knob && (e[i].d == 0 || e[i].d == d) && n <= e[i].n_max) return e[i].value;
    return knob_default(knob, d);
}

gd_status run_batch(MemProvider& mem, int K, const gd_instance* inst, cudaStream_t st, cudaEvent_t* events,
                    RunInfo* info, const Tuning* tuning, PhaseGraphs* graphs, cudaEvent_t* sort_events,
                    StageSet stage, bool allow_async) {
    Run r{mem, K, inst, st, events, info, tuning, graphs, sort_events, stage, allow_async};
    const long long l0 = t_launches;
    const gd_status s = r.go();
    if (info) info->launches = t_launches - l0;
    return s;
}

gd_status finish_batch(MemProvider& mem, int K, const gd_instance* inst, cudaStream_t st, RunInfo* info) {
    auto cuda_fail = [&](cudaError_t e, const char* where) {
        if (info) info->error = std::string(where) + ": " + cudaGetErrorString(e);
        return GD_ECUDA;
    };
    const size_t small_bytes = sizeof(int) * kSmallInts * K;
    const bool stats = info && info->want_stats;
    const size_t stat_bytes = stats ? sizeof(unsigned long long) * kStatCount * K : 0;
    void* h = nullptr;
    gd_status s = mem.host(kHostFinish, small_bytes + stat_bytes + 64, &h);
    if (s != GD_OK) return s;
    // (the buffers exist and are large enough: the run asked for them)
    void* dsm = mem.current(kMemSmall);
    void* dst = mem.current(kMemStats);
    if (!dsm || (stats && !dst)) {
        if (info) info->error = "no run to finish";
        return GD_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(h, dsm, small_bytes, cudaMemcpyDeviceToHost, st);
    unsigned long long* hst = reinterpret_cast<unsigned long long*>((char*)h + ((small_bytes + 63) & ~(size_t)63));
    if (e == cudaSuccess && stats) e = cudaMemcpyAsync(hst, dst, stat_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "read back");
    const int* sm = (const int*)h;
    gd_status result = GD_OK;
    unsigned any = 0;
    for (int k = 0; k < K; ++k) {
        const unsigned bits = (unsigned)sm[(size_t)k * kSmallInts + kSmStatus];
        any |= bits;
        if ((bits & kDevRange) && result == GD_OK) {
            result = GD_ERANGE;
            if (info) info->error = "coordinate range too large: d * R^2 >= 2^62 (instance " + std::to_string(k) + ")";
        }
    }
    if (result == GD_OK && (any & (kDevReplan | kDevOverflow))) result = kGdRerun;
    if (result == GD_OK && (any & kDevTimeout)) {
        result = GD_ETIMEOUT;
        if (info) info->error = "a bounded device wait or retry loop hit its limit";
    }
    if (result == GD_OK) {
        // the shapes' plans and sizes for later calls; the pool's use
        PlanCache* pc = mem.plans();
        double entries = 0, runs = 0, pts = 0;
        for (int k = 0; k < K; ++k) {
            const int* s0 = sm + (size_t)k * kSmallInts;
            pts += (double)inst[k].n;
            if (!pc) continue;
            const long long cap = (1ll << 62) - 1;
            ShapePlan* p = pc->slot(inst[k].n, inst[k].d, inst[k].eps2 > cap ? cap : inst[k].eps2);
            p->stamp = ++pc->clock;
            p->key_class = s0[kSmKeyClass];
            p->key_words = s0[kSmKeyWords];
            p->key_bits = s0[kSmKeyBits];
            p->nnbr = (unsigned)s0[kSmNnbr];
            p->maxcell = s0[kSmMaxCell];
            entries += (double)(unsigned)s0[kSmNnbr];
        }
        const unsigned long long ctr = *reinterpret_cast<const unsigned long long*>(sm + kSmPool);
        runs = (double)(ctr >> kPoolBits);
        const double used = (double)(ctr & ((1ull << kPoolBits) - 1));
        if (pts > 0) mem.note_pool((used > 0 ? used : entries) / pts, runs / pts);
    }
    if (info) {
        const int* s0 = sm;
        const long long C = s0[kSmCells], nnbr = (unsigned)s0[kSmNnbr];
        const long long n = info->sizes[0], d = info->sizes[1];
        info->sizes[2] = C;
        info->sizes[3] = nnbr;
        info->sizes[7] = (long long)s0[kSmPairsT];
        info->sizes[10] = (long long)s0[kSmHard0] + s0[kSmHard1];
        info->view_bytes[GD_VIEW_PERM] = (size_t)n * 4;
        info->view_bytes[GD_VIEW_CELL_START] = (size_t)(C + 1) * 4;
        info->view_bytes[GD_VIEW_CELL_COORD] = (size_t)C * d * 4;
        info->view_bytes[GD_VIEW_NBR_START] = (size_t)(C + 1) * 4;
        info->view_bytes[GD_VIEW_NBR] = (size_t)nnbr * 4;
        info->view_bytes[GD_VIEW_CORE_SORTED] = (size_t)n;
        info->view_bytes[GD_VIEW_CELL_CID] = (size_t)C * 4;
        if (stats) {
            for (int i = 0; i < kStatCount; ++i) info->stats[i] = 0;
            for (int k = 0; k < K; ++k)
                for (int i = 0; i < kStatCount; ++i) info->stats[i] += hst[(size_t)k * kStatCount + i];
            info->have_stats = true;
        }
    }
    return result;
}

}  // namespace gd
