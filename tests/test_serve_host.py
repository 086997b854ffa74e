"""Host-side logic of the continuous-batching server, with a fake backend
(no GPU): admission by footprint, batching, backfill, routing of results,
failure propagation and draining on close."""
import threading
import time

import numpy as np
import pytest

from paper_2210_07580_gb300.serve import Server


class FakeBackend:
    """Footprint n * 10 bytes; a run sleeps briefly and returns labels equal
    to the first coordinate, so each result identifies its job."""

    def __init__(self, fail_on=None):
        self.lock = threading.Lock()
        self.calls = []
        self.in_use = 0
        self.max_in_use = 0
        self.fail_on = fail_on

    def footprint(self, n, d):
        return n * 10

    large_at = 2000  # jobs above this many points count as large here

    def run(self, slot, jobs, gate=None):
        if gate is not None:
            with gate:
                return self._run(jobs)
        return self._run(jobs)

    def _run(self, jobs):
        fp = sum(j.footprint for j in jobs)
        nl = sum(1 for j in jobs if j.n > self.large_at)
        with self.lock:
            self.in_use += fp
            self.max_in_use = max(self.max_in_use, self.in_use)
            self.calls.append([j.n for j in jobs])
            self.large_now = getattr(self, "large_now", 0) + nl
            self.max_large_now = max(getattr(self, "max_large_now", 0), self.large_now)
        time.sleep(0.002 + 1e-7 * sum(j.n for j in jobs))
        with self.lock:
            self.in_use -= fp
            self.large_now -= nl
        if self.fail_on is not None and any(j.n == self.fail_on for j in jobs):
            raise RuntimeError("planted failure")
        return [(j.X[:, 0].copy(), j.X[:, 0] % 2 == 0) for j in jobs]


def job(n, tag, d=2):
    X = np.zeros((n, d), np.int32)
    X[:, 0] = tag
    return X


def test_results_route_to_their_jobs_and_budget_holds():
    fb = FakeBackend()
    with Server(slots=3, hbm_budget=200_000, small_job_points=1000, backend=fb) as srv:
        futs = [(t, srv.submit(job(50 + (t * 37) % 900, t), 100, 3)) for t in range(120)]
        for t, f in futs:
            lab, core = f.result(timeout=30)
            assert (lab == t).all()
    assert fb.max_in_use <= 200_000
    assert any(len(c) > 1 for c in fb.calls), "small jobs were never batched"


def test_large_jobs_run_alone_and_small_ones_backfill():
    fb = FakeBackend()
    srv = Server(slots=2, hbm_budget=60_000, small_job_points=1000, backend=fb)
    big = [srv.submit(job(5000, 1000 + t), 1, 1) for t in range(3)]
    small = [srv.submit(job(100, t), 1, 1) for t in range(20)]
    for f in big + small:
        f.result(timeout=30)
    srv.close()
    for c in fb.calls:
        if any(n > 1000 for n in c):
            assert c == [5000], "a large job shared a batch"
    assert fb.max_in_use <= 60_000


def test_oversized_job_is_refused():
    srv = Server(slots=1, hbm_budget=1000, backend=FakeBackend())
    with pytest.raises(ValueError):
        srv.submit(job(500, 1), 1, 1)
    srv.close()


def test_failures_reach_the_jobs_and_the_server_goes_on():
    fb = FakeBackend(fail_on=777)
    with Server(slots=2, hbm_budget=10**9, small_job_points=10, backend=fb) as srv:
        bad = srv.submit(job(777, 1), 1, 1)
        good = srv.submit(job(500, 2), 1, 1)
        with pytest.raises(RuntimeError, match="planted"):
            bad.result(timeout=30)
        assert (good.result(timeout=30)[0] == 2).all()


def test_close_drains_the_queue_and_stats():
    fb = FakeBackend()
    srv = Server(slots=2, hbm_budget=10**9, small_job_points=100, backend=fb)
    futs = [srv.submit(job(10 + t, t), 1, 1) for t in range(40)]
    srv.close(wait=True)
    assert all(f.done() for f in futs)
    st = srv.stats()
    assert st["jobs"] == 40 and st["p99_ms"] >= st["p50_ms"] >= 0
    with pytest.raises(RuntimeError):
        srv.submit(job(10, 1), 1, 1)


def test_large_jobs_never_overlap_and_small_ones_keep_flowing():
    fb = FakeBackend()
    with Server(slots=3, hbm_budget=10**9, small_job_points=1000, large_job_points=FakeBackend.large_at,
                max_large=1, backend=fb) as srv:
        big = [srv.submit(job(200_000, 5000 + t), 1, 1) for t in range(4)]
        small = [srv.submit(job(100, t), 1, 1) for t in range(30)]
        for t, f in enumerate(small):
            assert (f.result(timeout=30)[0] == t).all()
        small_done_at = time.perf_counter()
        for f in big:
            f.result(timeout=30)
        big_done_at = time.perf_counter()
    assert fb.max_large_now == 1
    assert small_done_at < big_done_at, "small jobs waited behind the large ones"


def test_staging_round_trip():
    """GpuBackend's host staging: rows in at aligned byte offsets, labels and
    core flags out of the result buffer."""
    torch = pytest.importorskip("torch")
    from paper_2210_07580_gb300.serve import Job, stage_in, stage_out
    rng = np.random.default_rng(3)
    jobs = [Job(rng.integers(-10**6, 10**6, size=(n, d)).astype(np.int32), 1, 1, 0, 0.0)
            for n, d in ((1, 3), (257, 5), (1000, 2))]
    al = 256
    up = lambda v: (v + al - 1) // al * al  # noqa: E731
    in_off, out_off, tin, tout = [], [], 0, 0
    for j in jobs:
        in_off.append(tin)
        tin += up(j.X.nbytes)
        out_off.append(tout)
        tout += up(4 * j.n) + up(j.n)
    hin = torch.zeros(tin, dtype=torch.uint8)
    stage_in(hin, jobs, in_off)
    for j, o in zip(jobs, in_off):
        got = hin[o:o + j.X.nbytes].numpy().view(np.int32).reshape(j.X.shape)
        np.testing.assert_array_equal(got, j.X)
    hout = torch.zeros(tout, dtype=torch.uint8)
    want = []
    for j, o in zip(jobs, out_off):
        lab = rng.integers(-1, j.n, size=j.n).astype(np.int32)
        core = rng.integers(0, 2, size=j.n).astype(np.uint8)
        hout[o:o + 4 * j.n] = torch.from_numpy(lab.view(np.uint8))
        hout[o + up(4 * j.n):o + up(4 * j.n) + j.n] = torch.from_numpy(core)
        want.append((lab, core.astype(bool)))
    got = stage_out(hout, jobs, out_off, al)
    hout.fill_(0)  # the results are copies
    for (gl, gc), (wl, wc) in zip(got, want):
        assert gl.dtype == np.int32 and gc.dtype == bool
        np.testing.assert_array_equal(gl, wl)
        np.testing.assert_array_equal(gc, wc)


def test_warm_runs_every_job_on_every_slot_before_the_queue():
    class SlotBackend(FakeBackend):
        def run(self, slot, jobs, gate=None):
            with self.lock:
                self.slots = getattr(self, "slots", []) + [(slot, jobs[0].n)]
            return super().run(slot, jobs, gate)

    fb = SlotBackend()
    jobs = [(job(n, n), 100, 3) for n in (5, 700, 40)]
    srv = Server(slots=3, hbm_budget=10 ** 9, backend=fb)
    srv.warm(jobs)
    # largest first, on each slot in turn; nothing reached the statistics
    assert fb.slots == [(s, n) for s in range(3) for n in (700, 40, 5)]
    assert srv.stats() == {"jobs": 0}
    res = [srv.submit(X, e, m).result(timeout=10) for X, e, m in jobs]
    assert [int(r[0][0]) for r in res] == [5, 700, 40]
    srv.close()
