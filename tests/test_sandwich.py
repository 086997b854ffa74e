"""The sandwich checker of approximate results (tests/sandwich.py), pinned on
the oracle: exact DBSCAN itself lies in the sandwich, and so does a result
that joins two exact clusters whose core points are within eps + delta;
every planted mistake (a join beyond eps + delta, a split, a flipped core
flag, a wrong id, a wrong border label) is caught."""
import numpy as np
import pytest

import oracle
from sandwich import border_labels, check_sandwich

EPS, DELTA, MINPTS = 100, 20, 4


def three_blocks():
    """Lattice blocks A, B and C (spacing 10, 21 x 21 points).  B starts
    eps + 5 to the right of A (joined at eps + delta, apart at eps); C is far.
    Plus a border point of A and a noise point."""
    g = np.arange(0, 201, 10)
    blk = np.array([(x, y) for x in g for y in g], dtype=np.int64)
    A = blk
    B = blk + [200 + EPS + 5, 0]
    C = blk + [5000, 5000]
    extra = np.array([[-99, 0], [-3000, -3000]], dtype=np.int64)
    X = np.vstack([A, B, C, extra])
    perm = np.random.default_rng(5).permutation(len(X))
    return np.ascontiguousarray(X[perm].astype(np.int32))


@pytest.fixture(scope="module")
def case():
    X = three_blocks()
    eps2, hi2 = EPS * EPS, (EPS + DELTA) ** 2
    E = oracle.grid(X, eps2, MINPTS)
    H = oracle.grid(X, hi2, MINPTS)
    return X, eps2, E, H


def relabel(core, labels):
    """Ids as the smallest core index of each cluster (core points only)."""
    out = labels.astype(np.int64).copy()
    ci = np.flatnonzero(core)
    first = {}
    for i in ci:
        first.setdefault(int(labels[i]), int(i))
    out[ci] = [first[int(labels[i])] for i in ci]
    return out


def test_reference_clusterings(case):
    X, eps2, E, H = case
    ncl = lambda r: len(np.unique(r[0][r[0] >= 0]))  # noqa: E731
    assert ncl(E) == 3 and ncl(H) == 2
    # the border point joins A, the noise point stays noise
    assert (E[0] == -1).sum() == 1


def test_exact_result_is_in_the_sandwich(case):
    X, eps2, E, H = case
    check_sandwich(X, eps2, E[0], E[1], E, H)


def test_joining_within_eps_plus_delta_is_allowed(case):
    X, eps2, E, H = case
    lab, core = E[0].astype(np.int64), E[1].astype(bool)
    # the two exact clusters H joins
    ci = np.flatnonzero(core)
    hi_of = {int(lab[i]): int(H[0][i]) for i in ci}
    joined = [c for c in hi_of if list(hi_of.values()).count(hi_of[c]) == 2]
    assert len(joined) == 2
    merged = lab.copy()
    merged[np.isin(merged, joined)] = min(joined)
    merged = relabel(core, merged)
    merged = border_labels(X, eps2, core, merged)
    check_sandwich(X, eps2, merged, core, E, H)


def test_planted_mistakes_are_caught(case):
    X, eps2, E, H = case
    lab, core = E[0].astype(np.int64), E[1].astype(bool)
    ci = np.flatnonzero(core)
    ids = sorted({int(v) for v in lab[ci]})
    hi_of = {int(lab[i]): int(H[0][i]) for i in ci}
    far = [c for c in ids if list(hi_of.values()).count(hi_of[c]) == 1][0]
    near = [c for c in ids if c != far][0]
    # 1. a join beyond eps + delta
    bad = lab.copy()
    bad[bad == far] = near
    bad = border_labels(X, eps2, core, relabel(core, bad))
    with pytest.raises(AssertionError, match="eps \\+ delta"):
        check_sandwich(X, eps2, bad, core, E, H)
    # 2. an exact cluster split in two
    bad = lab.copy()
    members = ci[lab[ci] == near]
    bad[members[len(members) // 2:]] = 10 ** 6
    bad = border_labels(X, eps2, core, relabel(core, bad))
    with pytest.raises(AssertionError, match="exact clusters"):
        check_sandwich(X, eps2, bad, core, E, H)
    # 3. a core flag flipped
    flip = core.copy()
    flip[ci[0]] = False
    with pytest.raises(AssertionError, match="core flags"):
        check_sandwich(X, eps2, lab, flip, E, H)
    # 4. an id that is not the cluster's smallest core index
    bad = lab.copy()
    bad[lab == near] = int(members[-1])
    with pytest.raises(AssertionError, match="smallest core index"):
        check_sandwich(X, eps2, bad, core, E, H)
    # 5. a border point labelled noise
    border = np.flatnonzero(~core & (lab >= 0))
    assert len(border) == 1
    bad = lab.copy()
    bad[border[0]] = -1
    with pytest.raises(AssertionError, match="border rule"):
        check_sandwich(X, eps2, bad, core, E, H)
