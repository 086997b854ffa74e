"""Merge heuristics of the paper on the GPU, through the C ABI.

- FastMerging (Alg. 5) with both pruning tests of Alg. 4 (triangle and
  angle, Def. 8 / Thm. 1) on adversarial pairs of dense core grids whose
  closest points are exactly eps apart (one witness: merge) or just beyond
  (no witness): the labels equal the oracle's, and the run statistics show
  that FastMerging ran, proved "no" and pruned by angle.
- The low-density-first pair order of GriT-DBSCAN-LDF (Section 5.2) gives
  the labels of the touching-first order and of the oracle.
- The run statistics are consistent: every candidate pair ends in exactly
  one outcome.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, synth  # noqa: E402

pytestmark = pytest.mark.gpu

# every pair of core grids with more than 32 core points on a side gets one
# 32 x 32 tile from the warp before it is handed to FastMerging
FORCE_FM = [("merge_budget", 0, 1 << 62, 1), ("merge_lane", 0, 1 << 62, 1), ("merge_small", 0, 1 << 62, 32)]
OUTCOMES = ("pairs_skipped", "pairs_box_no", "pairs_box_yes", "pairs_lane", "pairs_warp", "fm_yes", "fm_no")


def run(ctx, X, eps2, minpts):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy()


def same(got, want, what):
    assert np.array_equal(got[1], want[1]), f"{what}: core flags differ"
    assert np.array_equal(got[0], want[0]), f"{what}: labels differ at {int((got[0] != want[0]).sum())}"


def near_eps_pairs(d, eps, k, m, seed):
    """k pairs of dense clusters.  In pair t the clusters face each other
    across a gap along dimension 0; their closest points are one planted pair
    at squared distance eps^2 (t even: a witness) or eps^2 + 1 (t odd: none),
    every other cross pair being more than eps apart."""
    rng = np.random.default_rng(seed)
    spread = 1.5 * eps if d <= 3 else 0.5 * eps
    pts = []
    for t in range(k):
        o = np.full(d, 20000.0)
        o[0] += 12 * eps * t
        A = np.empty((m, d))
        B = np.empty((m, d))
        A[:, 0] = rng.uniform(o[0] - 3 * eps, o[0] - 10, m)
        B[:, 0] = rng.uniform(o[0] + eps + 11, o[0] + 4 * eps, m)
        for j in range(1, d):
            A[:, j] = rng.uniform(o[j] - spread, o[j] + spread, m)
            B[:, j] = rng.uniform(o[j] - spread, o[j] + spread, m)
        pa = o.copy()
        pb = o.copy()
        pb[0] += eps
        if t % 2 == 1:
            pb[1] += 1  # squared distance eps^2 + 1
        pts += [np.floor(A), np.floor(B), pa[None], pb[None]]
    X = np.vstack(pts).astype(np.int32)
    return np.ascontiguousarray(X[rng.permutation(len(X))])


@pytest.mark.parametrize("d,m", [(2, 3000), (3, 10000), (5, 10000)])
def test_fastmerging_on_near_eps_pairs(d, m):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps = 400
    X = near_eps_pairs(d, eps, 6, m, seed=40 + d)
    eps2, minpts = eps * eps, 4
    want = oracle.grid(X, eps2, minpts)
    ctx = Context(0, tuning=FORCE_FM)
    ctx.set_stats(True)
    got = run(ctx, X, eps2, minpts)
    st = ctx.run_stats()
    ctx.close()
    same(got, want, f"near-eps pairs d={d}")
    # three pairs merged across the gap, three not: 6 + 3 clusters in all
    assert len(np.unique(want[0][want[0] >= 0])) == 9
    assert st["pairs_fastmerging"] > 0 and st["fm_no"] > 0
    assert sum(st[f"kappa_{i}"] for i in range(1, 16)) + st["kappa_16_or_more"] == st["fm_yes"] + st["fm_no"]
    if d == 2:
        assert st["fm_pruned_angle"] > 0, st


@pytest.mark.parametrize("name,n", [("tiny", 20000), ("skew3d_10m", 300000), ("skew5d_10m", 200000),
                                    ("ss3d_2m", 400000)])
def test_low_density_first_order_gives_the_same_labels(name, n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload(name, n=n, seed=3)
    want = oracle.grid(X, eps2, minpts)
    stats = {}
    for order in (0, 1):
        ctx = Context(0, tuning=[("merge_order", 0, 1 << 62, order)])
        ctx.set_stats(True)
        same(run(ctx, X, eps2, minpts), want, f"{name} merge_order={order}")
        stats[order] = ctx.run_stats()
        ctx.close()
    # the same candidate pairs, each decided once
    assert stats[0]["pairs"] == stats[1]["pairs"]
    for order in (0, 1):
        st = stats[order]
        assert sum(st[k] for k in OUTCOMES) == st["pairs"], (order, st)


def test_statistics_off_by_default_and_per_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload("tiny", n=5000, seed=1)
    ctx = Context(0)
    run(ctx, X, eps2, minpts)
    assert ctx.run_stats() == {}
    ctx.set_stats(True)
    run(ctx, X, eps2, minpts)
    st = ctx.run_stats()
    assert st["pairs"] > 0 and st["nonfull_points"] > 0 and st["count_rows"] >= st["nonfull_points"]
    ctx.set_stats(False)
    run(ctx, X, eps2, minpts)
    assert ctx.run_stats() == {}
    ctx.close()
