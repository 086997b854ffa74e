"""Pins for the CPU oracle (no GPU).

The oracle must be right before anything is compared against it, so every
check here ties it to something other than itself: hand-derived fixtures from
the paper's definitions, the worked example's printed facts, closed forms and
special cases that reduce to library routines (scipy connected components,
scikit-learn's DBSCAN, exact float64 distance matrices), brute force on tiny
inputs and invariants of the clustering.
"""
import numpy as np
import pytest

import oracle
from golden_io import load_grid_case, load_labels_case


def rand_points(rng, n, d, lo=0, hi=1000, lattice=1):
    """Integer points; with lattice > 1 they sit on a coarse lattice so that
    many pairwise distances tie exactly with the eps boundary."""
    X = rng.integers(lo // lattice, hi // lattice, size=(n, d)) * lattice
    return np.ascontiguousarray(X.astype(np.int32))


def core_partition(labels, core):
    """Set of frozensets of core-point indices, one per cluster."""
    groups = {}
    for i in np.flatnonzero(core):
        groups.setdefault(int(labels[i]), []).append(int(i))
    return {frozenset(g) for g in groups.values()}


def float_dist2(X):
    """Exact all-pairs squared distances (integers < 2^53 in float64)."""
    Xf = X.astype(np.float64)
    return ((Xf[:, None, :] - Xf[None, :, :]) ** 2).sum(-1)


# ---------------------------------------------------------------- fixtures

@pytest.mark.parametrize("name", ["border_tie_2d.txt", "chain_dup_1d.txt"])
@pytest.mark.parametrize("impl", ["brute", "grid", "grid_fm"])
def test_golden_labels(name, impl):
    X, eps2, minpts, want_label, want_core = load_labels_case(name)
    if impl == "brute":
        lab, core = oracle.bruteforce(X, eps2, minpts)
    else:
        lab, core = oracle.grid(X, eps2, minpts, merge="plain" if impl == "grid" else "fastmerging")
    np.testing.assert_array_equal(core, want_core)
    np.testing.assert_array_equal(lab, want_label)


def test_worked_example_neighbour_query():
    """Section 4.2.2's query of g6 on the constructed Fig. 1 layout."""
    case = load_grid_case("fig2_neighbors_2d.txt")
    X, eps2 = case["X"], case["eps2"]
    assert X.shape == (19, 2)
    assert oracle.cell_side(eps2, case["d"]) == 11
    gs = oracle.grid_structure(X, eps2)
    coords = [tuple(int(v) for v in c) for c in gs["cell_coord"]]
    # nine non-empty grids, in the lexicographic order of Alg. 1, eta = 5
    assert coords == [case["grids"][k] for k in range(1, 10)]
    assert max(max(c) for c in coords) == 5
    q, want = case["query"]
    got = gs["nei"][gs["nei_start"][q - 1]: gs["nei_start"][q]]
    assert sorted(int(v) + 1 for v in got) == want


# ---------------------------------------------------------- special cases

@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_minpts1_is_connected_components(d):
    """MinPts = 1: every point is core and the clusters are the connected
    components of the eps-graph (scipy.sparse.csgraph)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(10 + d)
    X = rand_points(rng, 400, d, hi=400, lattice=5)
    eps2 = 25 * 4
    lab, core = oracle.grid(X, eps2, 1)
    assert core.all()
    A = csr_matrix(float_dist2(X) <= eps2)
    ncomp, comp = connected_components(A, directed=False)
    assert len(np.unique(lab)) == ncomp
    # canonical id = smallest index in the component
    first = {}
    for i, c in enumerate(comp):
        first.setdefault(c, i)
    np.testing.assert_array_equal(lab, np.array([first[c] for c in comp], np.int32))
    lab_b, core_b = oracle.bruteforce(X, eps2, 1)
    np.testing.assert_array_equal(lab_b, lab)


@pytest.mark.parametrize("impl", ["brute", "grid"])
def test_huge_eps_is_one_cluster(impl):
    rng = np.random.default_rng(3)
    X = rand_points(rng, 300, 3, hi=10_000)
    eps2 = 3 * 10_000 ** 2
    f = oracle.bruteforce if impl == "brute" else oracle.grid
    lab, core = f(X, eps2, 50)
    assert core.all()
    assert (lab == 0).all()


@pytest.mark.parametrize("impl", ["brute", "grid"])
def test_eps_below_min_spacing_is_all_noise(impl):
    rng = np.random.default_rng(4)
    X = rand_points(rng, 500, 2, hi=100_000, lattice=10)
    X = np.unique(X, axis=0)
    D = float_dist2(X)
    np.fill_diagonal(D, np.inf)
    eps2 = int(D.min()) - 1
    f = oracle.bruteforce if impl == "brute" else oracle.grid
    lab, core = f(X, eps2, 2)
    assert not core.any()
    assert (lab == -1).all()


def test_fewer_points_than_minpts_is_noise():
    X = np.array([[0, 0], [1, 0], [0, 1]], np.int32)
    for f in (oracle.bruteforce, oracle.grid):
        lab, core = f(X, 10, 4)
        assert not core.any() and (lab == -1).all()
        lab, core = f(X, 10, 3)
        assert core.all() and (lab == 0).all()


def test_empty_input():
    X = np.zeros((0, 3), np.int32)
    for f in (oracle.bruteforce, oracle.grid):
        lab, core = f(X, 10, 3)
        assert lab.shape == (0,) and core.shape == (0,)


def test_range_and_argument_errors():
    X = np.array([[0], [2**31 - 1], [-2**31]], np.int32)
    with pytest.raises(ValueError, match="range"):
        oracle.grid(X, 10, 2)
    Y = np.zeros((4, 2), np.int32)
    with pytest.raises(ValueError):
        oracle.grid(Y, -1, 2)
    with pytest.raises(ValueError):
        oracle.bruteforce(Y, 1, 0)


def test_sklearn_agreement():
    """scikit-learn's DBSCAN uses the same inclusive eps and a min_samples that
    counts the point itself: core sets and the partition of core points must
    match.  (Its border tie-break differs, so only border-ness is compared.)"""
    sk = pytest.importorskip("sklearn.cluster")
    from paper_2210_07580_gb300 import synth
    X, eps2, minpts = synth.workload("tiny", n=6000)
    lab, core = oracle.grid(X, eps2, minpts)
    # integer dist2 <= eps2  <=>  dist < sqrt(eps2 + 0.5): no float tie risk
    res = sk.DBSCAN(eps=float(np.sqrt(eps2 + 0.5)), min_samples=minpts).fit(X.astype(np.float64))
    sk_core = np.zeros(len(X), bool)
    sk_core[res.core_sample_indices_] = True
    np.testing.assert_array_equal(core, sk_core)
    assert core_partition(lab, core) == core_partition(res.labels_, sk_core)
    np.testing.assert_array_equal(lab == -1, res.labels_ == -1)


# -------------------------------------------------- brute force vs grid

CASES = [
    # d, n, hi, lattice, eps2, minpts
    (1, 600, 3000, 1, 25, 3),
    (2, 800, 2000, 10, 900, 4),
    (2, 1500, 5000, 1, 40_000, 8),
    (3, 1200, 600, 20, 1600, 5),
    (3, 1000, 2000, 1, 40_000, 6),
    (4, 900, 300, 10, 2500, 4),
    (5, 800, 200, 10, 1500, 3),
    (6, 700, 100, 10, 600, 3),
    (7, 600, 80, 10, 500, 3),
    (8, 500, 60, 10, 400, 3),
    (2, 400, 50, 1, 0, 2),       # eps = 0: duplicates only
]


@pytest.mark.parametrize("d,n,hi,lattice,eps2,minpts", CASES)
def test_brute_equals_grid(d, n, hi, lattice, eps2, minpts):
    rng = np.random.default_rng(1000 * d + n)
    X = rand_points(rng, n, d, hi=hi, lattice=lattice)
    # a few exact duplicates and a dense clump
    X[: n // 20] = X[n // 20: 2 * (n // 20)]
    lb, cb = oracle.bruteforce(X, eps2, minpts)
    for merge in ("plain", "fastmerging"):
        lg, cg = oracle.grid(X, eps2, minpts, merge=merge)
        np.testing.assert_array_equal(cg, cb)
        np.testing.assert_array_equal(lg, lb)
    # the cases must exercise all three kinds of points
    assert cb.any() and (~cb).any()


def test_tiny_workload_brute_equals_grid():
    from paper_2210_07580_gb300 import synth
    X, eps2, minpts = synth.workload("tiny")
    lb, cb = oracle.bruteforce(X, eps2, minpts)
    lg, cg = oracle.grid(X, eps2, minpts)
    np.testing.assert_array_equal(cg, cb)
    np.testing.assert_array_equal(lg, lb)
    assert 5 <= len(np.unique(lb[lb >= 0])) <= 20 and (lb == -1).any()


def test_neighbor_counts_match_core_flags():
    rng = np.random.default_rng(7)
    X = rand_points(rng, 700, 3, hi=500, lattice=5)
    eps2, minpts = 2500, 6
    cnt = oracle.neighbor_counts(X, eps2, np.arange(len(X)))
    want = (float_dist2(X) <= eps2).sum(1)
    np.testing.assert_array_equal(cnt, want)
    _, core = oracle.grid(X, eps2, minpts)
    np.testing.assert_array_equal(core, cnt >= minpts)


# ------------------------------------------------------------ invariants

def _case(seed=11, n=900, d=3):
    rng = np.random.default_rng(seed)
    return rand_points(rng, n, d, hi=800, lattice=4), 3600, 5


def test_permutation_invariance():
    X, eps2, minpts = _case()
    lab, core = oracle.grid(X, eps2, minpts)
    perm = np.random.default_rng(5).permutation(len(X))
    lab_p, core_p = oracle.grid(np.ascontiguousarray(X[perm]), eps2, minpts)
    inv = np.argsort(perm)
    lab_b, core_b = lab_p[inv], core_p[inv]
    np.testing.assert_array_equal(core_b, core)
    # cluster ids are input indices: map them back before comparing
    mapped = np.where(lab_b >= 0, perm[np.maximum(lab_b, 0)], -1)
    assert core_partition(mapped, core) == core_partition(lab, core)
    np.testing.assert_array_equal(lab_b == -1, lab == -1)


def test_translation_scaling_padding_invariance():
    X, eps2, minpts = _case(seed=12)
    lab, core = oracle.grid(X, eps2, minpts)
    l2, c2 = oracle.grid(X + np.int32(12345), eps2, minpts)
    np.testing.assert_array_equal(l2, lab)
    l3, c3 = oracle.grid(X * np.int32(7), eps2 * 49, minpts)
    np.testing.assert_array_equal(l3, lab)
    Xp = np.ascontiguousarray(np.concatenate([X, np.zeros((len(X), 1), np.int32)], axis=1))
    l4, c4 = oracle.grid(Xp, eps2, minpts)
    np.testing.assert_array_equal(l4, lab)
    np.testing.assert_array_equal(c4, core)


# --------------------------------------------- grids and neighbour query

@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_cell_side_is_largest_valid(d):
    rng = np.random.default_rng(d)
    for eps2 in list(rng.integers(0, 10**12, 200)) + [0, 1, d - 1, d, 4 * d, 2**61]:
        s = oracle.cell_side(int(eps2), d)
        assert d * (s - 1) ** 2 <= eps2 < d * s ** 2


@pytest.mark.parametrize("d,eps2,hi", [(2, 13, 40), (3, 30, 25), (2, 0, 10), (2, 1, 20), (4, 50, 9)])
def test_neighbour_lists_are_exact(d, eps2, hi):
    """Nei(g) against brute force over boxes: two grids are neighbours iff some
    pair of integer points, one in each grid's box, is within eps.  The boxes
    are enumerated point by point (small sides only)."""
    import itertools
    rng = np.random.default_rng(d * 100 + eps2)
    X = rand_points(rng, 300, d, hi=hi)
    X[0] = 0  # pins the per-dimension minimum to 0
    s = oracle.cell_side(eps2, d)
    gs = oracle.grid_structure(X, eps2)
    coords = gs["cell_coord"]
    C = len(coords)
    offs = np.array(list(itertools.product(range(s), repeat=d)))

    def box_points(c):
        return c * s + offs

    for a in range(C):
        got = set(int(v) for v in gs["nei"][gs["nei_start"][a]: gs["nei_start"][a + 1]])
        Pa = box_points(coords[a]).astype(np.float64)
        want = set()
        for b in range(C):
            if np.abs(coords[a] - coords[b]).max() > 3 * (1 + int(np.sqrt(eps2 + 1)) // s + 1):
                continue
            Pb = box_points(coords[b]).astype(np.float64)
            dmin = ((Pa[:, None, :] - Pb[None, :, :]) ** 2).sum(-1).min()
            if dmin <= eps2:
                want.add(b)
        assert got == want, a


def test_grid_diameter_and_completeness():
    """Any two points of one grid are within eps (the point of Eq. 1), and every
    pair of points within eps lies in grids that are neighbours (Alg. 3 misses
    nothing)."""
    rng = np.random.default_rng(21)
    for d, eps2 in [(2, 400), (3, 700), (5, 900), (7, 1500)]:
        X = rand_points(rng, 500, d, hi=120)
        gs = oracle.grid_structure(X, eps2)
        cell_of = np.empty(len(X), np.int64)
        for c in range(len(gs["cell_start"]) - 1):
            members = gs["order"][gs["cell_start"][c]: gs["cell_start"][c + 1]]
            cell_of[members] = c
            P = X[members]
            assert float_dist2(P).max() <= eps2
        D = float_dist2(X)
        nei = [set(gs["nei"][gs["nei_start"][c]: gs["nei_start"][c + 1]].tolist())
               for c in range(len(gs["cell_start"]) - 1)]
        I, J = np.nonzero(D <= eps2)
        for i, j in zip(I, J):
            assert cell_of[j] in nei[cell_of[i]]
        # grid order: lexicographic by identifier, input order inside a grid
        keys = [tuple(v) for v in gs["cell_coord"]]
        assert keys == sorted(keys)
        for c in range(len(keys)):
            m = gs["order"][gs["cell_start"][c]: gs["cell_start"][c + 1]]
            assert (np.diff(m) > 0).all()


# ---------------------------------------------- set minimum distance / FM

def test_mindist_plain_and_fastmerging_match_exact():
    """MinDist(A,B) <= eps by Def. 7 and by FastMerging (Alg. 5) against the
    exact float64 distance matrix, on separated sets like two grids' core
    points, including sets whose minimum distance equals eps exactly."""
    rng = np.random.default_rng(99)
    rounds = []
    for t in range(400):
        d = int(rng.integers(1, 8))
        na, nb = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        A = rng.integers(0, 50, size=(na, d))
        shift = np.zeros(d, np.int64)
        shift[0] = int(rng.integers(40, 90))
        B = rng.integers(0, 50, size=(nb, d)) + shift
        A = A.astype(np.int32)
        B = B.astype(np.int32)
        Dm = ((A[:, None, :].astype(np.float64) - B[None, :, :]) ** 2).sum(-1).min()
        for eps2 in (int(Dm) - 1, int(Dm), int(Dm) + 1, int(rng.integers(0, 3 * int(Dm) + 1))):
            if eps2 < 0:
                continue
            want = Dm <= eps2
            got_p, _ = oracle.mindist_le(A, B, eps2, "plain")
            got_f, r = oracle.mindist_le(A, B, eps2, "fastmerging")
            assert got_p == want and got_f == want, (t, eps2)
            rounds.append(r)
    assert max(rounds) >= 2  # pruning iterations were exercised


def test_fastmerging_rounds_small_on_grid_pairs():
    """kappa stays small on neighbouring grids: the paper observed at most 11
    rounds in all its experiments (Section 4.3.3, remark after Thm. 3)."""
    from paper_2210_07580_gb300 import synth
    for name, n in (("ss3d_2m", 200_000), ("tiny", 20_000), ("skew3d_10m", 200_000)):
        X, eps2, minpts = synth.workload(name, n=n)
        _, _, st = oracle.grid(X, eps2, minpts, merge="fastmerging", return_stats=True)
        assert 1 <= st["max_rounds"] <= 11, name
        assert sum(st["kappa_hist"]) == st["merge_tests"], name
