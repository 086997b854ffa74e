"""Continuous-batching server for exact DBSCAN jobs on one GPU.

Clients submit clustering jobs (points, eps2, MinPts) at any time and get a
future.  A fixed set of slots serves them; each slot owns a gd_ctx (its
device workspace stays resident and is reused from job to job) and its own
CUDA stream, and runs on its own host thread, so the work of several slots
overlaps on the device.  Scheduling:

- admission by HBM footprint: a job is started only when a slot is free and
  its estimated device footprint fits in what the budget has left; jobs that
  do not fit wait (small jobs behind them may go first -- backfill);
- a large job (more than `large_job_points` points) keeps the whole GPU busy
  by itself, so at most `max_large` of them compute at a time (running two
  only makes them compete for L2); their host staging (copies in and out)
  overlaps the other's compute, and batches of small jobs may run beside
  them;
- continuous batching: a slot that takes a small job also takes the other
  small jobs queued at that moment (up to a point and job budget) and runs
  them as one gd_dbscan_batched call; large jobs run alone;
- requests that arrive while others are on the GPU join the queue and are
  admitted as slots and memory free up.

The scheduler is plain Python over a backend object; GpuBackend calls the C
ABI through the binding (every step of the clustering runs in the CUDA
library).  Results equal those of the same job run alone (gd_dbscan and
gd_dbscan_batched give bit-identical labels).
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


@dataclass(eq=False)  # jobs compare by identity (queue removal)
class Job:
    X: np.ndarray
    eps2: int
    minpts: int
    footprint: int
    t_submit: float
    future: Future = field(default_factory=Future)
    t_start: float = 0.0
    t_done: float = 0.0
    batch_size: int = 1

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def estimate_footprint(n: int, d: int, workspace_bytes) -> int:
    """Device bytes a job may need: the library's workspace bound, the input
    and output copies, and room for neighbour lists and pairs (64 entries of
    4 + 8 + 8 bytes per grid, grids <= points)."""
    return int(workspace_bytes(n, d)) + n * (4 * d + 5) + n * 64 * 20 // 4


def stage_in(hin, jobs, offsets) -> None:
    """Copy the jobs' points (int32 rows) into the byte tensor `hin` at the
    given byte offsets.  torch copies release the GIL, so the staging of
    several slots' threads overlaps."""
    import torch
    for j, o in zip(jobs, offsets):
        src = torch.from_numpy(np.ascontiguousarray(j.X, dtype=np.int32).reshape(-1).view(np.uint8))
        hin[o:o + src.numel()].copy_(src)


def stage_out(hout, jobs, offsets, align: int) -> list:
    """Each job's (labels int32 [n], core flags bool [n]) from the byte tensor
    `hout`: labels at the job's offset, flags at the next multiple of `align`
    after them.  Copies out of `hout` (torch, GIL released)."""
    import torch
    res = []
    for j, oo in zip(jobs, offsets):
        n = j.n
        fo = oo + (4 * n + align - 1) // align * align
        lab = hout[oo:oo + 4 * n].view(torch.int32).clone().numpy()
        core = hout[fo:fo + n].to(torch.bool).numpy()
        res.append((lab, core))
    return res


class GpuBackend:
    """Runs jobs through the C ABI: one Context and one CUDA stream per slot.
    Each slot keeps grow-only staging buffers: pinned host memory for the
    inputs and results of a batch, and device memory they are copied to and
    from (one host-to-device and one device-to-host copy per batch)."""

    ALIGN = 256

    def __init__(self, device: int = 0, slots: int = 4):
        import torch

        from .binding import Context, workspace_bytes
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.ctxs = [Context(device) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.bufs = [{} for _ in range(slots)]
        self.workspace_bytes = workspace_bytes

    def footprint(self, n: int, d: int) -> int:
        return estimate_footprint(n, d, self.workspace_bytes)

    def _buf(self, slot: int, name: str, nbytes: int, pinned: bool):
        torch = self.torch
        b = self.bufs[slot].get(name)
        if b is None or b.numel() < nbytes:
            size = max(nbytes + nbytes // 4, 1 << 20)
            if pinned:
                b = torch.empty(size, dtype=torch.uint8, pin_memory=True)
            else:
                b = torch.empty(size, dtype=torch.uint8, device=self.device)
            self.bufs[slot][name] = b
        return b

    def run(self, slot: int, jobs, gate=None):
        """Stage the jobs in, cluster them (holding `gate`, if given, only
        around the library call) and stage the results out."""
        torch = self.torch
        ctx, stream = self.ctxs[slot], self.streams[slot]
        al = self.ALIGN
        up = lambda v: (v + al - 1) // al * al  # noqa: E731
        in_off, out_off, tin, tout = [], [], 0, 0
        for j in jobs:
            in_off.append(tin)
            tin += up(j.X.nbytes)
            out_off.append(tout)
            tout += up(4 * j.n) + up(j.n)
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            hin = self._buf(slot, "hin", tin, True)
            hout = self._buf(slot, "hout", tout, True)
            din = self._buf(slot, "din", tin, False)
            dout = self._buf(slot, "dout", tout, False)
            stage_in(hin, jobs, in_off)
            din[:tin].copy_(hin[:tin], non_blocking=True)
            dev, outs = [], []
            for j, oi, oo in zip(jobs, in_off, out_off):
                n, d = j.X.shape
                Xd = din[oi:oi + 4 * n * d].view(torch.int32).view(n, d)
                lab = dout[oo:oo + 4 * n].view(torch.int32)
                core = dout[oo + up(4 * n):oo + up(4 * n) + n]
                dev.append((Xd, j.eps2, j.minpts))
                outs.append((lab, core))
            if gate is not None:
                stream.synchronize()  # inputs on the device before taking the GPU
                gate.acquire()
            try:
                if len(dev) == 1:
                    Xd, e, m = dev[0]
                    ctx.dbscan(Xd, e, m, labels=outs[0][0], is_core=outs[0][1], stream=stream)
                else:
                    ctx.dbscan_batched(dev, outputs=outs, stream=stream)
            finally:
                if gate is not None:
                    gate.release()
            hout[:tout].copy_(dout[:tout], non_blocking=True)
            stream.synchronize()
        return stage_out(hout, jobs, out_off, al)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.bufs = [{} for _ in self.bufs]


class Server:
    """See the module docstring.  `backend` defaults to GpuBackend(device,
    slots); tests pass a fake one."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int | None = None,
                 small_job_points: int = 200_000, batch_max_jobs: int = 64, batch_max_points: int = 4_000_000,
                 large_job_points: int = 1_000_000, max_large: int = 1, backend=None):
        self.backend = backend if backend is not None else GpuBackend(device, slots)
        if hbm_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(free * 0.6)
        self.budget = int(hbm_budget)
        self.in_use = 0
        self.small = small_job_points
        self.batch_max_jobs = batch_max_jobs
        self.batch_max_points = batch_max_points
        self.large = large_job_points
        self.max_large = max_large
        self.large_gate = threading.Semaphore(max_large)
        self.queue: collections.deque[Job] = collections.deque()
        self.cv = threading.Condition()
        self.closed = False
        self.done: list[Job] = []
        self.workers = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(slots)]
        for w in self.workers:
            w.start()

    # ------------------------------------------------------------ client
    def submit(self, X, eps2: int, minpts: int) -> Future:
        X = np.ascontiguousarray(X, dtype=np.int32)
        if X.ndim != 2 or X.shape[0] < 1:
            raise ValueError("X must be a non-empty int32 array of shape [n, d]")
        fp = self.backend.footprint(X.shape[0], X.shape[1])
        if fp > self.budget:
            raise ValueError(f"job needs about {fp} device bytes, more than the server budget {self.budget}")
        job = Job(X, int(eps2), int(minpts), fp, time.perf_counter())
        with self.cv:
            if self.closed:
                raise RuntimeError("server is closed")
            self.queue.append(job)
            self.cv.notify_all()
        return job.future

    def close(self, wait: bool = True):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        if wait:
            for w in self.workers:
                w.join()
        close = getattr(self.backend, "close", None)
        if close:
            close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------- scheduling
    def _take(self):
        """Called with the lock held: the next unit of work that fits the
        budget, or None.  A large job at the head runs alone; small jobs are
        coalesced (FIFO) into one batch; when the head does not fit, the first
        queued job that does is taken (backfill)."""
        if not self.queue:
            return None
        room = self.budget - self.in_use
        head = self.queue[0]
        if head.footprint <= room:
            if head.n > self.small:
                self.queue.popleft()
                return [head]
            batch, pts, fp = [], 0, 0
            for j in list(self.queue):
                if j.n > self.small:
                    continue
                if len(batch) >= self.batch_max_jobs or pts + j.n > self.batch_max_points or fp + j.footprint > room:
                    break
                batch.append(j)
                pts += j.n
                fp += j.footprint
            for j in batch:
                self.queue.remove(j)
            return batch
        for j in self.queue:
            if j.footprint <= room:
                self.queue.remove(j)
                return [j]
        return None

    def _worker(self, slot: int):
        while True:
            with self.cv:
                work = None
                while not self.closed or self.queue:
                    work = self._take()
                    if work is not None:
                        break
                    if self.closed and not self.queue:
                        break
                    self.cv.wait(timeout=0.05)
                if work is None:
                    return
                fp = sum(j.footprint for j in work)
                self.in_use += fp
            t0 = time.perf_counter()
            for j in work:
                j.t_start = t0
                j.batch_size = len(work)
            try:
                large = any(j.n > self.large for j in work)
                results = self.backend.run(slot, work, self.large_gate if large else None)
                err = None
            except Exception as e:  # the jobs fail, the server goes on
                results, err = None, e
            t1 = time.perf_counter()
            with self.cv:
                self.in_use -= fp
                for k, j in enumerate(work):
                    j.t_done = t1
                    self.done.append(j)
                self.cv.notify_all()
            for k, j in enumerate(work):
                if err is not None:
                    j.future.set_exception(err)
                else:
                    j.future.set_result(results[k])

    def warm(self, jobs):
        """Run every given job once on every slot, outside the queue (call it
        before submitting), so that each slot's device workspace and staging
        buffers have grown to the job mix: workspaces only grow, and growing
        one reallocates it, which a timed run should not include.  The
        results are dropped."""
        ests = [Job(np.ascontiguousarray(X, dtype=np.int32), int(e), int(m), 0, 0.0) for X, e, m in jobs]
        ests.sort(key=lambda j: -j.X.size)
        for slot in range(len(self.workers)):
            for j in ests:
                self.backend.run(slot, [j])

    # --------------------------------------------------------------- stats
    def reset_stats(self):
        """Forget the finished jobs (e.g. after a warm-up pass)."""
        with self.cv:
            self.done = []

    def latencies(self):
        """Latencies (seconds) of the finished jobs, in submission order."""
        with self.cv:
            jobs = sorted(self.done, key=lambda j: j.t_submit)
        return np.array([j.t_done - j.t_submit for j in jobs])

    def stats(self) -> dict:
        lat = self.latencies()
        with self.cv:
            jobs = list(self.done)
        if not jobs:
            return {"jobs": 0}
        t0 = min(j.t_submit for j in jobs)
        t1 = max(j.t_done for j in jobs)
        return {"jobs": len(jobs), "wall_s": t1 - t0, "jobs_per_s": len(jobs) / max(t1 - t0, 1e-9),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_batch": float(np.mean([j.batch_size for j in jobs]))}
