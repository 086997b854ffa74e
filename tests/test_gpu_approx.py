"""Approximate FastMerging (the Remark after Alg. 5) on the GPU, through the
C ABI (gd_instance.eps2_yes): the results lie in the sandwich between exact
DBSCAN at eps and at eps + delta (tests/sandwich.py, both sides from the
oracle), the mode does join grids whose closest core points are beyond eps,
eps2_yes = eps2 is exact DBSCAN, and a run repeats bit for bit (the answer
of approximate FastMerging for a pair does not depend on the order in which
pairs are tested, so neither does the partition)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, GdError, synth  # noqa: E402
from sandwich import check_sandwich  # noqa: E402

pytestmark = pytest.mark.gpu

# pairs of core grids with more than 32 core points on a side get one 32 x 32
# tile before FastMerging decides them
FORCE_FM = [("merge_budget", 0, 1 << 62, 1), ("merge_lane", 0, 1 << 62, 1), ("merge_small", 0, 1 << 62, 32)]


def run(ctx, X, eps2, minpts, eps2_yes):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts, eps2_yes=eps2_yes)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy()


def beyond_eps_pairs(d, eps, gap, k, m, seed):
    """k pairs of dense clusters facing each other across a gap along
    dimension 0.  Only the grids of one planted pair (squared distance
    eps^2 + gap^2) have point boxes within eps of the other side; every cross
    pair is more than eps apart, so exact DBSCAN keeps all 2k clusters."""
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
        pb[1] += gap
        pts += [np.floor(A), np.floor(B), pa[None], pb[None]]
    X = np.vstack(pts).astype(np.int32)
    return np.ascontiguousarray(X[rng.permutation(len(X))])


def nclusters(lab):
    return len(np.unique(lab[lab >= 0]))


@pytest.mark.parametrize("d,m", [(2, 3000), (3, 10000)])
def test_approximate_fastmerging_joins_within_delta(d, m):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps, delta = 400, 100
    X = beyond_eps_pairs(d, eps, 60, 6, m, seed=70 + d)
    eps2, yes2, minpts = eps * eps, (eps + delta) ** 2, 4
    E = oracle.grid(X, eps2, minpts)
    H = oracle.grid(X, yes2, minpts)
    assert nclusters(E[0]) == 12 and nclusters(H[0]) == 6
    ctx = Context(0, tuning=FORCE_FM)
    ctx.set_stats(True)
    got = run(ctx, X, eps2, minpts, yes2)
    st = ctx.run_stats()
    check_sandwich(X, eps2, got[0], got[1], E, H)
    # FastMerging met a cross pair within eps + delta on some planted pair
    assert st["fm_yes"] > 0 and nclusters(got[0]) < 12, (nclusters(got[0]), st)
    again = run(ctx, X, eps2, minpts, yes2)
    assert np.array_equal(again[0], got[0]) and np.array_equal(again[1], got[1])
    # eps2_yes = eps2 is exact DBSCAN
    exact = run(ctx, X, eps2, minpts, eps2)
    assert np.array_equal(exact[0], E[0]) and np.array_equal(exact[1].astype(bool), E[1].astype(bool))
    ctx.close()


@pytest.mark.parametrize("name,n,tuning", [("tiny", 20000, FORCE_FM), ("skew3d_10m", 20000, FORCE_FM),
                                           ("skew5d_10m", 20000, FORCE_FM), ("tiny", 20000, None)])
def test_approximate_results_lie_in_the_sandwich(name, n, tuning):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload(name, n=n, seed=9)
    eps = int(np.sqrt(eps2))
    yes2 = (eps + eps // 10) ** 2
    E = oracle.grid(X, eps2, minpts)
    H = oracle.grid(X, yes2, minpts)
    ctx = Context(0, tuning=tuning)
    got = run(ctx, X, eps2, minpts, yes2)
    ctx.close()
    check_sandwich(X, eps2, got[0], got[1], E, H)


def test_eps2_yes_below_eps2_is_rejected():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload("tiny", n=2000, seed=1)
    ctx = Context(0)
    with pytest.raises(GdError) as e:
        run(ctx, X, eps2, minpts, eps2 - 1)
    assert e.value.status == 1  # GD_EINVAL
    # the context still works
    got = run(ctx, X, eps2, minpts, 0)
    ctx.close()
    want = oracle.grid(X, eps2, minpts)
    assert np.array_equal(got[0], want[0])
