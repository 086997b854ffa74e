"""Autotuner for the library's launch and tile knobs (gd_knob in gdbscan.h).

Instances are grouped by dimension and size bucket, as the library groups
them.  For every group the per-group knobs are tuned by coordinate descent:
each candidate value is set in the context's table for that group only, the
group's instances are clustered with gd_dbscan_batched, and the time of the
stages the knob affects (the library's own CUDA-event stage timers, median of
`reps` runs) decides.  The per-batch knobs are then tuned on all instances
together.  Every candidate run must give the labels of the default run; the
tuner stops with an error otherwise.

    python -m paper_2210_07580_gb300.autotune --out tuning.json

writes a table that `Context(tuning=...)` / `load_tuning` read; the package
ships one made this way on a GB300 (`tuning_gb300.json`), loaded by default.
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

# upper end of each size bucket (points), as in the library
BUCKET_MAX = [1 << 12, 1 << 15, 1 << 18, 1 << 21, 1 << 62]

PER_GROUP = {
    "merge_budget": ([1, 2, 4, 8], ["merge"]),
    "merge_lane": ([1, 4, 16, 64], ["merge"]),
    "merge_small": ([64, 128, 256], ["merge"]),
    "core_bands": ([0, 128, 4096], ["core"]),
    "merge_order": ([0, 1], ["merge_order", "merge"]),
    "core_mode": ([0, 1], ["core"]),
}
PER_BATCH = {
    "fm_blocks": ([152 * 2, 152 * 8, 152 * 32], ["merge"]),
    "walk_blocks": ([152 * 8, 152 * 32, 152 * 64], ["walk"]),
}
DEFAULTS = {"merge_budget": 2, "merge_lane": 16, "merge_small": 128, "core_bands": 128, "fm_blocks": 152 * 8,
            "walk_blocks": 152 * 32, "merge_order": 1}


def default_value(knob: str, d: int) -> int:
    """The library's built-in value of a knob for dimension d (the core
    counting form depends on the dimension: a warp per grid up to d = 4)."""
    if knob == "core_mode":
        return 1 if 1 <= d <= 4 else 0
    return DEFAULTS[knob]


def bucket_of(n: int) -> int:
    for b, top in enumerate(BUCKET_MAX):
        if n <= top:
            return b
    return len(BUCKET_MAX) - 1


def ordered(table: dict) -> list:
    """Table entries {(knob, d, n_max): value} as a list the library reads
    first-match: per knob and dimension, smaller buckets first, dimension-
    specific entries before d = 0 ones."""
    keys = sorted(table, key=lambda k: (k[0], k[1] == 0, k[1], k[2]))
    return [(k[0], k[1], k[2], table[k]) for k in keys]


class _Runner:
    def __init__(self, ctx, jobs):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.jobs = [(torch.from_numpy(X).to(f"cuda:{ctx.device}"), e, m) for X, e, m in jobs]
        self.out = [(torch.empty(len(X), dtype=torch.int32, device=X.device),
                     torch.empty(len(X), dtype=torch.uint8, device=X.device)) for X, _, _ in self.jobs]

    def run(self, table: dict, stages, reps: int):
        self.ctx.set_tuning(ordered(table))
        times = []
        for _ in range(reps):
            self.ctx.dbscan_batched(self.jobs, outputs=self.out)
            self.torch.cuda.synchronize()
            st = self.ctx.stage_times()
            times.append(sum(st.get(s, 0.0) for s in stages))
        labels = [lab.clone() for lab, _ in self.out]
        return statistics.median(times), labels


def tune(instances, device: int = 0, reps: int = 3, log=print) -> dict:
    """Returns {"entries": [...], "log": [...]} for a list of (X, eps2, minpts)."""
    import torch

    from .binding import Context
    ctx = Context(device, tuning=None)
    ctx.set_timing(True)
    table: dict = {}
    records = []
    groups: dict = {}
    for X, e, m in instances:
        groups.setdefault((X.shape[1], bucket_of(len(X))), []).append((X, e, m))

    def descend(runner, scope_d, n_max, knobs):
        _, want = runner.run(table, [], 1)
        for knob, (cands, stages) in knobs.items():
            key = (knob, scope_d, n_max)
            best_v, best_t = None, None
            for v in cands:
                table[key] = v
                t, labels = runner.run(table, stages, reps)
                if not all(torch.equal(a, b) for a, b in zip(labels, want)):
                    raise RuntimeError(f"knob {knob}={v} changed the labels (d={scope_d}, n_max={n_max})")
                records.append({"knob": knob, "d": scope_d, "n_max": n_max, "value": v, "ms": round(t, 4)})
                if best_t is None or t < best_t:
                    best_v, best_t = v, t
            table[key] = best_v
            log(f"d={scope_d} n<={n_max}: {knob} = {best_v} ({best_t:.3f} ms)")

    for (d, b), jobs in sorted(groups.items()):
        descend(_Runner(ctx, jobs), d, BUCKET_MAX[b], PER_GROUP)
    descend(_Runner(ctx, instances), 0, BUCKET_MAX[-1], PER_BATCH)
    ctx.close()
    # drop entries equal to the built-in default
    entries = [e for e in ordered(table) if e[3] != default_value(e[0], e[1]) or e[0] in PER_BATCH]
    return {"entries": [{"knob": k, "d": d, "n_max": n, "value": v} for k, d, n, v in entries], "log": records}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--k", type=int, default=256, help="instances of the batched workload to tune on")
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true",
                    help="tune on the batched instances only (by default the single-instance workloads "
                         "tiny, ss3d_2m, ss3d_10m, skew3d_10m and skew5d_10m join them, each in its own group)")
    args = ap.parse_args()
    import torch

    from . import synth
    jobs = synth.batch_instances(args.k, seed=args.seed)
    what = f"{args.k} batched instances (synth.batch_instances seed {args.seed})"
    if not args.no_plain:
        plain = ["tiny", "ss3d_2m", "ss3d_10m", "skew3d_10m", "skew5d_10m"]
        jobs = jobs + [synth.workload(w, seed=1) for w in plain]
        what += " + " + ", ".join(plain)
    t0 = time.time()
    res = tune(jobs, args.device, args.reps)
    doc = {"device": torch.cuda.get_device_name(args.device), "workload": what,
           "seconds": round(time.time() - t0, 1), **res}
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {args.out}: {len(res['entries'])} entries")


if __name__ == "__main__":
    main()
