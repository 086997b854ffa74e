"""Checker of approximate DBSCAN results against the sandwich definition.

Approximate FastMerging (the Remark after Alg. 5) answers "yes" for two core
grids when it meets a pair of their core points within eps + delta, and
"no" only when its pruning (exact at eps) has emptied a set.  Core points
and the border rule stay those of eps.  So a result R of it lies between two
exact clusterings, both computed by the oracle:

- exact DBSCAN at eps (E): R has E's core points, and the core points of
  every cluster of E lie in one cluster of R;
- exact DBSCAN at eps + delta (H, squared radius eps2_yes): the core points
  of every cluster of R lie in one cluster of H (core points at eps are core
  points at eps + delta).

R's ids follow the library's rule (smallest input index among a cluster's
core points) and its border points follow Section 4.4 on R's clusters: a
non-core point takes the smallest id among the clusters of the core points
within eps, or -1 when there is none.
"""
import numpy as np


def _refines(fine, coarse, what):
    """Every class of `fine` lies inside one class of `coarse` (arrays of
    labels over the same points)."""
    order = np.lexsort((coarse, fine))
    f, c = fine[order], coarse[order]
    same = f[1:] == f[:-1]
    bad = same & (c[1:] != c[:-1])
    if bad.any():
        k = int(np.argmax(bad))
        raise AssertionError(f"{what}: points {int(order[k])} and {int(order[k + 1])} are together "
                             f"in the finer clustering but apart in the coarser one")


def border_labels(X, eps2, core, labels):
    """Labels of the non-core points by the border rule on the clustering
    that `labels` gives the core points (exact integer distances)."""
    X = np.asarray(X, dtype=np.int64)
    core = np.asarray(core, dtype=bool)
    ci = np.flatnonzero(core)
    out = np.full(len(X), -1, dtype=np.int64)
    out[ci] = labels[ci]
    if len(ci) == 0:
        return out
    C = X[ci]
    cl = labels[ci].astype(np.int64)
    for i in np.flatnonzero(~core):
        d2 = ((C - X[i]) ** 2).sum(axis=1)
        hit = d2 <= eps2
        if hit.any():
            out[i] = cl[hit].min()
    return out


def check_sandwich(X, eps2, labels, core, exact, hi):
    """Raise AssertionError unless (labels, core) is a valid approximate
    result: `exact` = (labels, core) of DBSCAN at eps2 and `hi` = (labels,
    core) of DBSCAN at eps2_yes, both from the oracle."""
    labels = np.asarray(labels, dtype=np.int64)
    core = np.asarray(core).astype(bool)
    el, ec = np.asarray(exact[0], dtype=np.int64), np.asarray(exact[1]).astype(bool)
    hl, hc = np.asarray(hi[0], dtype=np.int64), np.asarray(hi[1]).astype(bool)
    if not np.array_equal(core, ec):
        raise AssertionError("core flags differ from exact DBSCAN at eps")
    ci = np.flatnonzero(core)
    if (labels[ci] < 0).any():
        raise AssertionError("a core point is labelled noise")
    if not hc[ci].all():
        raise AssertionError("a core point at eps is not core at eps + delta (the reference is wrong)")
    _refines(el[ci], labels[ci], "exact clusters inside the result's")
    _refines(labels[ci], hl[ci], "the result's clusters inside those at eps + delta")
    # ids: smallest input index among each cluster's core points
    ids = labels[ci]
    first = {}
    for i, c in zip(ci.tolist(), ids.tolist()):
        first.setdefault(c, i)
    for c, i in first.items():
        if c != i:
            raise AssertionError(f"cluster id {c} is not its smallest core index {i}")
    want = border_labels(X, eps2, core, labels)
    bad = np.flatnonzero(want != labels)
    if len(bad):
        raise AssertionError(f"border rule broken at {len(bad)} points, first {int(bad[0])}: "
                             f"{int(labels[bad[0]])} instead of {int(want[bad[0]])}")
