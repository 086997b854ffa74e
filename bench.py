"""Benchmark: exact DBSCAN throughput on one GB300 (or N replicas).

Default workload: seed-spreader d=3, n=10,000,000, eps=500 (eps2=250000),
MinPts=20, int32 coordinates in [0, 1e5)^3, seeded, synthetic.  One step is
one full exact-DBSCAN run (every stage of the hot path) on device-resident
points, through the C ABI.  L2 is flushed (a 256 MB device write) before every
timed step, outside the timed events.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
(the paper's grid method in plain C, all host cores) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpts/s exact DBSCAN d=3 n=10M; batched vs looped inst/s; serve p99"
WORKLOADS = {
    "ss3d_10m": "seed-spreader d=3 n=10,000,000 eps=500 MinPts=20 (+0.01% uniform noise)",
    "ss3d_2m": "seed-spreader d=3 n=2,000,000 eps=500 MinPts=20 (+0.01% uniform noise)",
    "skew5d_10m": "skewed mix d=5 n=10,000,000 eps=1000 MinPts=100 (50% in one eps-ball + 20 blobs)",
    "skew3d_10m": "skewed mix d=3 n=10,000,000 eps=500 MinPts=20 (50% in one eps-ball + 20 blobs)",
    "tiny": "blobs d=2 n=20,000 eps=800 MinPts=10 (10 blobs sigma=1500 + 5% noise)",
}
# The plain-method configurations measured beside the headline: label,
# workload, timed steps.  L3 is the headline itself (seed spreader) and its
# skewed-mix variant.
CONFIGS = [("T", "tiny", 20), ("S", "ss3d_2m", 10), ("L3", "ss3d_10m", 10), ("L3_skew", "skew3d_10m", 10),
           ("L5", "skew5d_10m", 5)]
HBM_STAGES = ("bounds", "quantise", "sort", "compact", "lists", "core")
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) per downsweep launch, from one `ncu --set full`
# capture of the kernel on the default workload, keyed by a digest of the
# kernel's source text: a changed kernel reports no traffic until it is
# captured again.
SORT_PASS_TRAFFIC = {
    "afb4db10006ca34f": {"workload": "ss3d_10m", "key_class": 0, "bytes": 113.2e6},
}


def sort_source_digest() -> str:
    """Digest of the downsweep kernel's source text (the kernel the traffic
    table describes)."""
    import hashlib
    path = os.path.join(ROOT, "paper_2210_07580_gb300", "csrc", "sort.cu")
    with open(path) as f:
        text = f.read()
    a = text.find("// Downsweep: one block per tile ranks its keys stably")
    b = text.find("template <typename K, bool PACKED> static size_t downsweep_smem")
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16] if 0 <= a < b else ""


def stage_bandwidth(stages: dict, n: int, d: int, sizes: dict, peak: float, stats: dict | None = None) -> dict:
    """Achieved bandwidth of the grid-build stages and (with run statistics)
    of the count stage: algorithmic bytes (each array the stage must read or
    write, once) over the stage's device time.  The count stage must write
    every core flag (1 B/point) and read, at least once, each non-full
    point's row and the rows of those points' neighbour grids (the statistic
    count_rows counts them once per non-full grid; no row is read from DRAM
    more than once at minimum, so the rows are capped at n)."""
    dp = 1 if d == 1 else 2 if d == 2 else 4 if d <= 4 else 8
    kc = sizes["key_class"]
    key_b = 16 if kc == 2 else 8
    val_b = 0 if kc == 0 else 4
    P = sizes["sort_passes"]
    first_hist = kc != 2  # quantisation writes the first pass's tile histograms for 64-bit keys
    # packed keys whose in-cell offsets fit one 32-bit word: quantisation
    # writes that word, and the compaction reads it instead of the input row
    xw = (int(sizes["side"]) - 1).bit_length() if kc == 0 else -1
    rebuild = kc == 0 and d * xw <= 32
    off_b = 4 if rebuild and xw > 0 else 0
    bytes_ = {
        "bounds": 4 * d * n,
        "quantise": (4 * d + key_b + val_b + off_b) * n,
        "sort": (P * 2 * (key_b + val_b) + (P - (1 if first_hist else 0)) * key_b) * n,
        "compact": (2 * key_b + val_b + 4 + 4 + (off_b if rebuild else 4 * d) + 4 * dp) * n,
    }
    # the lists: the walk's forward entries (each pair once, self included)
    # read from its pool, every entry written into the scanned lists
    nnbr, grids = sizes.get("nnbr", 0), sizes.get("grids", 0)
    if nnbr:
        bytes_["lists"] = 4 * ((nnbr + grids) // 2 + nnbr)
    if stats:
        bytes_["core"] = n + min(n, stats["nonfull_points"] + stats["count_rows"]) * 4 * dp
    out = {}
    for st, b in bytes_.items():
        ms = stages.get(st, 0.0)
        if ms > 0:
            gbs = b / (ms / 1e3) / 1e9
            out[st] = {"bytes": int(b), "ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
    return out


def reduce_over_ranks(ms: float, e2e_ms: float, points: int, ws: int, device):
    """Job-wide values from rank-local ones: the max over ranks of the step
    and end-to-end times, and the sum of the points the ranks clustered."""
    if ws == 1:
        return ms, e2e_ms, points
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([points], dtype=torch.int64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(t[1].item()), int(p[0].item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling (every 10 ms) of SM clocks and throttle reasons;
    only samples whose timestamps fall inside the marked window count."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"gdbscan_clocks_{os.getpid()}.csv")
        self.t0 = self.t1 = None

    def start(self):
        """Start sampling and wait (up to 3 s) for the first sample."""
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 3.0
        while time.time() < t_end and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def mark_start(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def mark_stop(self):
        import datetime
        self.t1 = datetime.datetime.now()

    def stop(self):
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        time.sleep(0.03)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(parts[2]), float(parts[3]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower() in ("active", "1")}))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        sm = [r[1] for r in use]
        reasons = set().union(*[r[3] for r in use]) if use else set()
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": use[-1][2] if use else None,
                "reasons": sorted(reasons), "samples": len(sm), "in_timed_region": bool(inside)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return model or os.uname().machine


def time_oracle(workload: str, seed: int, n_sample: int | None):
    """One oracle run on a bounded sample of the workload; returns (s, n, threads)."""
    import oracle
    from paper_2210_07580_gb300 import synth
    X, eps2, minpts = synth.workload(workload, seed=seed, n=n_sample)
    oracle.build()
    t0 = time.perf_counter()
    oracle.grid(X, eps2, minpts)
    return time.perf_counter() - t0, len(X), oracle.num_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    ns = args.cpu_sample
    times, n, thr = [], 0, 1
    for i in range(args.warmup + args.steps):
        t, n, thr = time_oracle(args.workload, 1, ns)
        if i >= args.warmup:
            times.append(t)
    s_per_step = sum(times) / len(times)
    value = n / s_per_step / 1e6
    sample = f"{WORKLOADS[args.workload]}" + (f", first {n} points of the walk" if ns else ", full size")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(s_per_step * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": n},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mpts/s", "cores": thr, "kind": "oracle",
                         "sample": sample, "cpu": cpu_info()},
        "e2e": {"value": round(value, 3), "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def alu_utilisation(stages: dict, stats: dict, peak_per_s: float) -> dict:
    """Exact squared distances per second of the distance-heavy stages (the
    statistics' counts over the timed stage's time) against the register-only
    ceiling of the same instruction mix (gd_distance_peak)."""
    out = {"peak_dist_per_s": round(peak_per_s / 1e9, 2), "unit": "Gdist/s"}
    for stage, keys in (("core", ("dist_core",)), ("merge", ("dist_merge", "dist_fastmerging")),
                        ("labels", ("dist_labels",))):
        ms = stages.get(stage, 0.0)
        cnt = sum(stats.get(k, 0) for k in keys)
        if ms > 0 and cnt > 0:
            rate = cnt / (ms / 1e3)
            out[stage] = {"distances": int(cnt), "ms": round(ms, 4), "gdist_per_s": round(rate / 1e9, 2),
                          "frac": round(rate / peak_per_s, 4)}
    return out


def merge_summary(stats: dict) -> dict:
    """Candidate-pair outcomes, the rate of pairs skipped because their grids
    were already joined (the LDF skip of Section 5.2), and the FastMerging
    round histogram (kappa, Section 4.3.3)."""
    pairs = stats.get("pairs", 0)
    kappa = [stats.get(f"kappa_{i}", 0) for i in range(1, 16)] + [stats.get("kappa_16_or_more", 0)]
    kmax = max((i + 1 for i, v in enumerate(kappa) if v), default=0)
    return {"pairs": pairs, "skipped_rate": round(stats.get("pairs_skipped", 0) / pairs, 4) if pairs else None,
            "outcomes": {k: stats.get(k, 0) for k in ("pairs_skipped", "pairs_box_no", "pairs_box_yes",
                                                      "pairs_lane", "pairs_warp", "pairs_fastmerging",
                                                      "fm_yes", "fm_no", "fm_pruned_triangle",
                                                      "fm_pruned_angle")},
            "kappa_hist": kappa, "kappa_max": kmax}


def measure_workload(ctx, dev, workload: str, steps: int, warmup: int, flush, stream, X=None, eps2=None,
                     minpts=None):
    """Device-timed runs of one workload (L2 flushed before each, outside the
    events), the library's stage times, and one untimed run with statistics."""
    import torch
    from paper_2210_07580_gb300 import synth
    if X is None:
        X, eps2, minpts = synth.workload(workload, seed=1)
    n = len(X)
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    core = torch.empty(n, dtype=torch.uint8, device=dev)

    def step():
        # queued asynchronously; finished (status checked) after the events
        ctx.dbscan(Xd, eps2, minpts, labels=labels, is_core=core, stream=stream, sync=False)

    for _ in range(warmup):
        flush.fill_(1)
        step()
        ctx.sync(stream)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    acc, times = {}, []
    for k in range(steps):
        flush.fill_(k + 2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ctx.sync(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        for name, ms in ctx.stage_times().items():
            acc[name] = acc.get(name, 0.0) + ms / steps
    ctx.set_timing(False)
    sizes = ctx.last_sizes()
    ctx.set_stats(True)
    step()
    ctx.sync(stream)
    torch.cuda.synchronize()
    stats = ctx.run_stats()
    ctx.set_stats(False)
    return {"X": X, "eps2": eps2, "minpts": minpts, "labels": labels.cpu().numpy(),
            "core": core.cpu().numpy().astype(bool), "ms": sum(times) / len(times),
            "stages": {k: round(v, 4) for k, v in acc.items()}, "sizes": sizes, "stats": stats}


def oracle_check(m: dict, fastmerging: bool = True) -> dict:
    """The oracle on the same input, outside the timed region: label and core
    flag parity, and its host time (plain merge, and FastMerging as the
    GriT-DBSCAN-LDF CPU baseline with its kappa)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    wl, wc = oracle.grid(m["X"], m["eps2"], m["minpts"])
    t_plain = time.perf_counter() - t0
    n = len(m["X"])
    out = {"parity": bool(np.array_equal(wl, m["labels"]) and np.array_equal(wc, m["core"])),
           "cpu_baseline": {"value": round(n / t_plain / 1e6, 3), "unit": "Mpts/s", "cores": oracle.num_threads(),
                            "kind": "oracle", "cpu": cpu_info(), "s": round(t_plain, 3),
                            "sample": "full input, merge by Def. 7"}}
    if fastmerging:
        t0 = time.perf_counter()
        _, _, st = oracle.grid(m["X"], m["eps2"], m["minpts"], merge="fastmerging", return_stats=True)
        t_fm = time.perf_counter() - t0
        out["cpu_baseline_fastmerging"] = {"value": round(n / t_fm / 1e6, 3), "unit": "Mpts/s", "s": round(t_fm, 3),
                                           "kind": "oracle (GriT-DBSCAN-LDF with FastMerging)",
                                           "kappa_max": st["max_rounds"], "kappa_hist": st["kappa_hist"],
                                           "merge_tests": st["merge_tests"]}
    return out


def stencil_offsets(d: int, eps2: int) -> int:
    """Identifier offsets delta (a stencil) whose grids can hold points
    within eps of the query grid's: sum over j of gap_j^2 <= eps2, with
    gap_j = (|delta_j| - 1) s + 1 for delta_j != 0 (the relation of Eq. 2 in
    integers, s the integer cell side).  The alternative to the tree query
    would probe each of these per grid (half of them, pairs once)."""
    import math
    s = 1 + math.isqrt(eps2 // d)
    r = 0 if eps2 == 0 else 1 + (math.isqrt(eps2) - 1) // s
    sums = {0: 1}  # partial sum of squared gaps -> number of offset prefixes
    for _ in range(d):
        nxt = {}
        for v, c in sums.items():
            for dl in range(-r, r + 1):
                g = 0 if dl == 0 else (abs(dl) - 1) * s + 1
                w = v + g * g
                if w <= eps2:
                    nxt[w] = nxt.get(w, 0) + c
        sums = nxt
    return sum(sums.values())


def walk_summary(stats: dict, grids: int, d: int, eps2: int) -> dict:
    """Work of the neighbour query (Alg. 3 on the sorted levels) per query
    grid, beside the size of the offset stencil it replaces."""
    if not grids or "walk_nodes" not in stats:
        return {}
    st = stencil_offsets(d, eps2)
    return {"nodes_tested_per_grid": round(stats["walk_nodes"] / grids, 1),
            "warp_steps_per_grid": round(stats["walk_steps"] / grids, 2),
            "stencil_offsets": st, "stencil_probes_per_grid": (st + 1) // 2}


def config_line(label: str, workload: str, m: dict, peak: float, dist_peak: float, check: dict | None) -> dict:
    n, d = m["X"].shape
    stages = m["stages"]
    sb = stage_bandwidth(stages, n, d, m["sizes"], peak, m["stats"])
    main = {k: v for k, v in stages.items() if k != "sort_downsweep"}
    dom = max(main, key=main.get)
    total = sum(main.values())
    line = {"label": label, "workload": WORKLOADS[workload], "n": n, "d": d, "eps2": m["eps2"],
            "minpts": m["minpts"], "ms_per_step": round(m["ms"], 4), "value": round(n / (m["ms"] / 1e3) / 1e6, 3),
            "unit": "Mpts/s", "grids": m["sizes"]["grids"], "neighbour_entries": m["sizes"]["nnbr"],
            "stages_ms": stages,
            "dominant_stage": {"name": dom, "ms": round(main[dom], 4), "share": round(main[dom] / total, 3)},
            "stage_bandwidth": sb,
            "alu": alu_utilisation(stages, m["stats"], dist_peak),
            "merge": merge_summary(m["stats"]),
            "walk": walk_summary(m["stats"], m["sizes"]["grids"], d, m["eps2"])}
    # roofline of the config's dominant HBM-bound stage (grid build or count)
    hb = {k: v for k, v in sb.items() if k in HBM_STAGES}
    if hb:
        k = max(hb, key=lambda s: hb[s]["ms"])
        line["roofline"] = {"bound": "hbm", "stage": k, "achieved": hb[k]["gbs"], "peak": peak, "unit": "GB/s",
                            "frac": hb[k]["frac"], "bytes": hb[k]["bytes"]}
    if check:
        line.update(check)
    return line


def bench_batched(ctx, dev, args):
    """Batched vs looped throughput (inst/s) on the 256-instance workload,
    same GPU, same context; the labels of both paths must be identical."""
    import torch
    from paper_2210_07580_gb300 import synth
    jobs = synth.batch_instances(args.batch_k, seed=7)
    djobs = [(torch.from_numpy(X).to(dev), e, m) for X, e, m in jobs]
    outs_b = [(torch.empty(len(X), dtype=torch.int32, device=dev), torch.empty(len(X), dtype=torch.uint8, device=dev))
              for X, _, _ in jobs]
    outs_l = [(torch.empty(len(X), dtype=torch.int32, device=dev), torch.empty(len(X), dtype=torch.uint8, device=dev))
              for X, _, _ in jobs]
    stream = torch.cuda.current_stream()

    def batched():
        ctx.dbscan_batched(djobs, outputs=outs_b, stream=stream)

    def looped():
        for (Xd, e, m), (lab, core) in zip(djobs, outs_l):
            ctx.dbscan(Xd, e, m, labels=lab, is_core=core, stream=stream, sync=False)
        ctx.sync(stream)

    res = {}
    for name, fn in (("batched", batched), ("looped", looped)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        res[name] = min(ts)
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs_b, outs_l))
    k = len(jobs)
    return {"workload": f"{k} instances: n log-uniform in [1e3, 5e5], d in {{2,3,5,7}}, eps in [200, 2000], "
                        f"MinPts in {{5,10,50,100}}, blobs + 5% noise",
            "points": int(sum(len(X) for X, _, _ in jobs)),
            "batched_inst_per_s": round(k / (res["batched"] / 1e3), 1),
            "looped_inst_per_s": round(k / (res["looped"] / 1e3), 1),
            "batched_ms": round(res["batched"], 3), "looped_ms": round(res["looped"], 3),
            "speedup": round(res["looped"] / res["batched"], 2), "labels_identical": bool(same)}


def _replay(srv, jobs, arrivals):
    """Submit jobs at their arrival times (seconds from now; None = all at
    once); wait for every result.  Returns (results, stats)."""
    srv.reset_stats()
    t0 = time.perf_counter()
    futs = []
    for i, (X, e, m) in enumerate(jobs):
        if arrivals is not None:
            wait = t0 + arrivals[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        futs.append(srv.submit(X, e, m))
    res = [f.result(timeout=900) for f in futs]
    return res, srv.stats()


def _stream(srv, pool, picks, arrivals):
    """A request stream: request i is pool job picks[i], submitted at
    arrivals[i] seconds from now.  Results are checked for errors and then
    dropped (a long stream would not fit in host memory).  Returns the
    latencies in submission order (seconds) and the server's stats."""
    srv.reset_stats()
    t0 = time.perf_counter()
    futs = []
    for i, k in enumerate(picks):
        wait = t0 + arrivals[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        X, e, m = pool[k]
        futs.append(srv.submit(X, e, m))
    for f in futs:
        f.result(timeout=900)
    st = srv.stats()
    return srv.latencies(), st


def _pcts(lat) -> dict:
    lat = np.asarray(lat) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2)}


def bench_serve(dev, args):
    """Serving: the same jobs through (a) the sequential plain path -- one
    slot, one job per gd_dbscan call, host arrays in and out -- and (b) the
    continuous-batching server (several slots, small jobs coalesced into
    gd_dbscan_batched).
    - Capacity: the job pool queued all at once, three times per path after
      an untimed pass (resident workspaces); jobs/s of each repeat.
    - Latency: a Poisson stream of `serve_requests` requests drawn from the
      pool (seeded) after `serve_warmup` untimed ones, at `load` times the
      sequential path's measured capacity; p50/p99 over all requests and per
      third of the stream (their spread), and the mean batch size.
    - Results: every pool job's labels and core flags from the two paths
      must be identical."""
    from paper_2210_07580_gb300 import synth
    from paper_2210_07580_gb300.serve import Server
    pool = synth.serve_jobs(args.serve_jobs, seed=11)
    npts = int(sum(len(X) for X, _, _ in pool))
    rng = np.random.default_rng(13)
    nreq, nwarm = args.serve_requests, args.serve_warmup
    picks = rng.integers(0, len(pool), size=nreq + nwarm)
    out = {"workload": f"pool of {len(pool)} jobs: n log-uniform in [1e3, 1e7], d in 2..7, eps in [200, 2000], "
                       f"MinPts in {{5,10,50,100}}, blobs + 5% noise; host int32 arrays in, labels + core flags out",
           "jobs": len(pool), "points": npts, "load": args.serve_load,
           "stream": f"{nreq} Poisson requests drawn from the pool after {nwarm} warm-up requests"}
    configs = (("sequential", dict(slots=1, small_job_points=0)),
               ("served", dict(slots=args.serve_slots, small_job_points=200_000)))
    results = {}
    rate = None
    for name, kw in configs:
        with Server(device=dev.index or 0, **kw) as srv:
            # warm-up: every pool job on every slot (workspaces grow to the mix,
            # once), then one pass through the queue
            srv.warm(pool)
            res, _ = _replay(srv, pool, None)
            results[name] = res
            caps, batch = [], []
            for _ in range(3):
                _, st = _replay(srv, pool, None)
                caps.append(round(st["jobs_per_s"], 2))
                batch.append(st["mean_batch"])
            o = {"slots": kw["slots"], "jobs_per_s": round(float(np.mean(caps)), 2), "jobs_per_s_repeats": caps,
                 "mean_batch": round(float(np.mean(batch)), 2)}
            if rate is None:
                rate = args.serve_load * float(np.mean(caps))
                arrivals = synth.poisson_arrivals(nreq + nwarm, rate, seed=12)
                out["rate_per_s"] = round(rate, 2)
            if nwarm:
                _stream(srv, pool, picks[:nwarm], arrivals[:nwarm])
            lat, st = _stream(srv, pool, picks[nwarm:], arrivals[nwarm:] - (arrivals[nwarm - 1] if nwarm else 0.0))
            thirds = [_pcts(part) for part in np.array_split(lat, 3)]
            o.update({"poisson_" + k: v for k, v in _pcts(lat).items()})
            o.update({"poisson_requests": int(len(lat)), "poisson_mean_batch": round(st["mean_batch"], 2),
                      "poisson_jobs_per_s": round(st["jobs_per_s"], 2),
                      "poisson_p99_ms_thirds": [t["p99_ms"] for t in thirds],
                      "poisson_p50_ms_thirds": [t["p50_ms"] for t in thirds]})
            out[name] = o
            del res
    seq, srv_ = out["sequential"]["jobs_per_s_repeats"], out["served"]["jobs_per_s_repeats"]
    out["speedup_jobs_per_s"] = round(out["served"]["jobs_per_s"] / out["sequential"]["jobs_per_s"], 3)
    out["speedup_range"] = [round(min(srv_) / max(seq), 3), round(max(srv_) / min(seq), 3)]
    out["labels_identical"] = bool(all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
                                       for a, b in zip(results["sequential"], results["served"])))
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2210_07580_gb300 import Context, synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # each rank clusters its own independent instance (replicas, weak scaling)
    X, eps2, minpts = synth.workload(args.workload, seed=1 + rank, n=args.n)
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    core = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = Context(local)
    stream = torch.cuda.current_stream()

    def step():
        # queued asynchronously (gd_dbscan); its status is read after the
        # step's end event (gd_sync), outside the timed span
        ctx.dbscan(Xd, eps2, minpts, labels=labels, is_core=core, stream=stream, sync=False)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
        ctx.sync(stream)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    sampler = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_acc = {}
    launches = 0
    sampler.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark_start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k + 2)  # L2 flush, outside the timed events
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        ctx.sync(stream)
        for name, ms in ctx.stage_times().items():
            stage_acc[name] = stage_acc.get(name, 0.0) + ms
        launches += ctx.last_sizes()["launches"]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    sampler.mark_stop()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    sizes = ctx.last_sizes()
    stages = {k: round(v / args.steps, 4) for k, v in stage_acc.items()}
    ctx.set_timing(False)

    # end to end through the host-buffer entry point: pinned X in, labels and
    # core flags out, every step.  The calls alternate between two contexts
    # on two streams (gd_dbscan_host_async; each call first finishes its
    # context's previous one), so that one step's copies overlap the other
    # context's kernels; the time is the wall clock from the first call to
    # the last sync, over the steps.  Every step copies its 120 MB input in
    # afresh (no L2 flush between them).
    Xh = torch.from_numpy(X).pin_memory()
    ctx2 = Context(local)
    ctxs = [ctx, ctx2]
    streams = [stream, torch.cuda.Stream(device=dev)]
    outs = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory())
            for _ in ctxs]
    for c in (0, 1):  # the second context learns the shape's plan
        ctxs[c].dbscan_host(Xh, eps2, minpts, labels=outs[c][0], is_core=outs[c][1], stream=streams[c])
    torch.cuda.synchronize()
    # a fixed number of calls, so the pipeline's fill and drain weigh the
    # same whatever the timed step count
    e2e_steps = 20
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        c = k % 2
        ctxs[c].dbscan_host(Xh, eps2, minpts, labels=outs[c][0], is_core=outs[c][1], stream=streams[c], sync=False)
    for c in (0, 1):
        ctxs[c].sync(streams[c])
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    ctx2.close()
    ms_max, e2e_ms, total_pts = reduce_over_ranks(ms, e2e_ms, n, ws, dev)

    if rank == 0:
        value = total_pts / (ms_max / 1e3) / 1e6
        peak, peak_kind = peaks()
        # dominant kernel: the radix sort's downsweep (one per pass), timed
        # by the library's events around each launch.  Algorithmic bytes of
        # one launch: every key (and value) of the pass read once and
        # written once.
        passes = max(1, sizes["sort_passes"])
        # bytes one pass reads and writes per point: the packed key word, or
        # the key plus the 32-bit index
        unit_bytes = {0: 8, 1: 12, 2: 20}[sizes["key_class"]]
        launch_bytes = 2 * unit_bytes * n
        launch_ms = stages.get("sort_downsweep", 0.0) / passes
        achieved = launch_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
        tr = SORT_PASS_TRAFFIC.get(sort_source_digest())
        traffic = (int(tr["bytes"]) if tr and tr["workload"] == args.workload and tr["key_class"] == sizes["key_class"]
                   else None)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Mpts/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": n, "d": d, "eps2": eps2, "minpts": minpts,
                       "grids": sizes["grids"], "neighbour_entries": sizes["nnbr"], "key_bits": sizes["key_bits"],
                       "l2": "flushed before every timed step (256 MB write, outside the timed events)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "clocks": clocks,
            "e2e": {"value": round(total_pts / (e2e_ms / 1e3) / 1e6, 3), "unit": "Mpts/s",
                    "ms_per_step": round(e2e_ms, 3), "h2d_bytes_per_step": int(X.nbytes),
                    "d2h_bytes_per_step": int(n * 4 + n), "steps": e2e_steps,
                    "how": "gd_dbscan_host_async on two contexts and streams in turn, pinned host buffers"},
            "gpu_launches": int(launches),
            "stages_ms": stages,
            "roofline": {"bound": "hbm", "kernel": "downsweep_kernel (radix-sort pass: rank and scatter)",
                         "achieved": round(achieved, 1) if achieved else None, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": round(achieved / peak, 4) if achieved else None, "traffic": traffic,
                         "bytes_per_launch": int(launch_bytes), "launch_ms": round(launch_ms, 4),
                         "launches_per_step": passes},
            "wall_s_timed": round(t_wall, 3),
            "stage_bandwidth": stage_bandwidth(stages, n, d, sizes, peak),
        }
        headline_check = None
        if not args.no_configs and ws == 1:
            # every plain-method configuration: device time, stages, HBM and
            # ALU fractions, merge statistics, and (outside the timed region)
            # the oracle's labels and host time on the same input
            from paper_2210_07580_gb300 import binding
            dist_peak = {}
            configs = {}
            for label, wl, steps in CONFIGS:
                m = measure_workload(ctx, dev, wl, steps, args.warmup, flush, stream)
                dd = m["X"].shape[1]
                if dd not in dist_peak:
                    dist_peak[dd] = binding.distance_peak(dd, local)
                check = None if args.no_cpu_baseline else oracle_check(m, fastmerging=not args.no_oracle_fm)
                configs[label] = config_line(label, wl, m, peak, dist_peak[dd], check)
                if wl == args.workload:
                    headline_check = check
                del m
            line["configs"] = configs
            line["parity_all_configs"] = all(c.get("parity", False) for c in configs.values()) \
                if not args.no_cpu_baseline else None
        if not args.no_batch:
            line["batched"] = bench_batched(ctx, dev, args)
        if not args.no_serve:
            line["serve"] = bench_serve(dev, args)
        if not args.no_cpu_baseline and ws == 1:
            if headline_check and not args.cpu_sample:
                cb = dict(headline_check["cpu_baseline"])
                cb["sample"] = f"{WORKLOADS[args.workload]}, full size, one run, {cb.pop('s'):.1f} s"
                line["cpu_baseline"] = cb
                if "cpu_baseline_fastmerging" in headline_check:
                    line["cpu_baseline_fastmerging"] = headline_check["cpu_baseline_fastmerging"]
            else:
                t, ns, thr = time_oracle(args.workload, 1, args.cpu_sample)
                line["cpu_baseline"] = {"value": round(ns / t / 1e6, 3), "unit": "Mpts/s", "cores": thr,
                                        "kind": "oracle", "cpu": cpu_info(),
                                        "sample": f"{WORKLOADS[args.workload]}, "
                                                  + (f"first {ns} points of the walk" if args.cpu_sample
                                                     else "full size")
                                                  + f", one run, {t:.1f} s"}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gdbscan", "reference"], default="gdbscan")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ss3d_10m")
    ap.add_argument("--n", type=int, default=None,
                    help="points of the headline workload (default: its full size; for profiling captures)")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="points of the workload the CPU oracle times (default: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-configuration measurements (T, S, L3, L3_skew, L5)")
    ap.add_argument("--no-oracle-fm", action="store_true",
                    help="skip timing the oracle's FastMerging variant beside its plain merge")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched vs looped measurement")
    ap.add_argument("--batch-k", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-jobs", type=int, default=48)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="Poisson arrival rate as a fraction of the sequential path's jobs/s")
    ap.add_argument("--serve-requests", type=int, default=2000, help="timed requests of the Poisson stream")
    ap.add_argument("--serve-warmup", type=int, default=100, help="untimed requests before them")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
