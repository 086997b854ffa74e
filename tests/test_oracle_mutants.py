"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a copy of the oracle's C source (on the
CPU), builds it, points the oracle module at it and runs a fast subset of the
pins from test_oracle.py: at least one of them must fail.  A pin suite that
passes a mutant is too weak to trust.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gd_oracle.c")

# (name, text to find, replacement)
MUTANTS = [
    ("def1_strict_boundary",
     "if (sqdist(X + p * d, X + q * d, d) <= eps2)\n                cnt++;",
     "if (sqdist(X + p * d, X + q * d, d) < eps2)\n                cnt++;"),
    # (">= minpts" -> "> minpts" would be an equivalent mutant: a grid with
    # exactly MinPts points is all core either way, its diameter being <= eps)
    ("full_grid_rule_off_by_one", "if (e - b >= minpts) {", "if (e - b >= minpts - 1) {"),
    ("gap_term_off_by_one", "i64 gap = delta == 0 ? 0 : (delta - 1) * g->s + 1;",
     "i64 gap = delta == 0 ? 0 : (delta - 1) * g->s;"),
    ("neighbour_window_short", "g->r = (eps2 == 0) ? 0 : 1 + (re - 1) / g->s;",
     "g->r = (eps2 == 0) ? 0 : (re - 1) / g->s;"),
    ("cell_side_too_big", "return 1 + (long long)isqrt_u64((u64)eps2 / (u64)d);",
     "return 2 + (long long)isqrt_u64((u64)eps2 / (u64)d);"),
    ("sqdist_drops_last_dim", "for (int j = 0; j < d; ++j) {\n        i64 t = (i64)a[j] - (i64)b[j];",
     "for (int j = 0; j < d - 1 + (d == 1); ++j) {\n        i64 t = (i64)a[j] - (i64)b[j];"),
    ("root_is_largest", "if (a < b)\n        parent[b] = a;\n    else\n        parent[a] = b;",
     "if (a > b)\n        parent[b] = a;\n    else\n        parent[a] = b;"),
    ("border_takes_largest_id", "if (best < 0 || c < best) best = c;", "if (best < 0 || c > best) best = c;"),
    ("triangle_missing_factor4", "(unsigned __int128)4 * (u64)A * (u64)eps2;",
     "(unsigned __int128)1 * (u64)A * (u64)eps2;"),
    ("fastmerging_prunes_sj_around_p",
     "cb = prune_set(B, ib, cb, q, p, dpq, angle_lambda(A, ia, ca, q, p, d, eps2), d, eps2);",
     "cb = prune_set(B, ib, cb, p, q, dpq, angle_lambda(A, ia, ca, q, p, d, eps2), d, eps2);"),
    ("angle_lambda_drops_arcsin",
     "const double ly = asin(clamp1(eps / b)) + acos(",
     "const double ly = 0.0 * asin(clamp1(eps / b)) + acos("),
    ("angle_test_without_margin_sign", "if (lambda + ANGLE_MARGIN < theta)",
     "if (lambda - 0.5 < theta)"),
    ("merge_skips_union", "if (yes) uf_union(parent, ci, cj);", "if (yes && ci < 0) uf_union(parent, ci, cj);"),
    ("border_strict_boundary", "if (sqdist(g.Xs + k * d, S + w * d, d) <= eps2) {",
     "if (sqdist(g.Xs + k * d, S + w * d, d) < eps2) {"),
]

FAST_PINS = [
    lambda: [pins.test_golden_labels(n, i) for n in ("border_tie_2d.txt", "chain_dup_1d.txt")
             for i in ("brute", "grid", "grid_fm")],
    pins.test_worked_example_neighbour_query,
    lambda: [pins.test_brute_equals_grid(*c) for c in pins.CASES],
    pins.test_grid_diameter_and_completeness,
    lambda: pins.test_neighbour_lists_are_exact(2, 1, 20),
    pins.test_mindist_plain_and_fastmerging_match_exact,
    lambda: pins.test_minpts1_is_connected_components(2),
    lambda: pins.test_cell_side_is_largest_valid(3),
]


def test_unmutated_source_passes_fast_pins():
    for pin in FAST_PINS:
        pin()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    oracle.compile_source(str(mpath), str(lib))
    prev = oracle.use_library(str(lib))
    caught = []
    try:
        for k, pin in enumerate(FAST_PINS):
            try:
                pin()
            except (AssertionError, ValueError):
                caught.append(k)
                break
    finally:
        oracle.restore_library(prev)
    assert caught, f"no pin caught the planted mistake {name}"
