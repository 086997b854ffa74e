"""The server on the GPU: every job's result in the mix equals the same job
run alone through gd_dbscan (and the oracle for the smaller ones)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, synth  # noqa: E402
from paper_2210_07580_gb300.serve import Server  # noqa: E402

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(77)
    jobs = []
    for t in range(40):
        n = int(np.exp(rng.uniform(np.log(300), np.log(300_000))))
        d = int(rng.integers(2, 8))
        eps = int(rng.uniform(200, 2000))
        m = int(rng.choice([5, 10, 50, 100]))
        X = synth.blobs(n, d, k=int(rng.integers(2, 6)), sigma=float(rng.uniform(300, 3000)), noise=0.05,
                        seed=int(rng.integers(1 << 30)))
        jobs.append((X, eps * eps, m))
    with Server(device=0, slots=4, small_job_points=50_000) as srv:
        futs = [srv.submit(X, e, m) for X, e, m in jobs]
        got = [f.result(timeout=600) for f in futs]
        st = srv.stats()
    assert st["jobs"] == len(jobs) and st["mean_batch"] > 1.0
    ctx = Context(0)
    for i, ((X, e, m), (lab, core)) in enumerate(zip(jobs, got)):
        Xd = torch.from_numpy(X).cuda()
        want_l, want_c = ctx.dbscan(Xd, e, m)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(core, want_c.cpu().numpy(), err_msg=f"job {i} core flags")
        np.testing.assert_array_equal(lab, want_l.cpu().numpy(), err_msg=f"job {i} labels")
        if len(X) <= 20000:
            wl, wc = oracle.grid(X, e, m)
            np.testing.assert_array_equal(lab, wl, err_msg=f"job {i} vs oracle")
    ctx.close()
