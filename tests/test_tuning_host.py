"""Tuning tables on the host: ordering (the library takes the first matching
entry) and size buckets (the same boundaries as the library's groups)."""
import json

from paper_2210_07580_gb300 import autotune
from paper_2210_07580_gb300.binding import KNOBS, load_tuning


def test_buckets_match_library_boundaries():
    # the library groups instances at <= 2^12, 2^15, 2^18, 2^21 points
    assert [autotune.bucket_of(n) for n in (1, 4096, 4097, 32768, 32769, 262144, 262145, 2097152, 2097153)] == \
        [0, 0, 1, 1, 2, 2, 3, 3, 4]


def test_ordered_puts_small_buckets_and_specific_dims_first():
    table = {("merge_budget", 0, 1 << 62): 4, ("merge_budget", 5, 1 << 18): 1, ("merge_budget", 5, 1 << 12): 8,
             ("core_bands", 3, 1 << 15): 0}
    got = autotune.ordered(table)
    mb = [e for e in got if e[0] == "merge_budget"]
    assert mb == [("merge_budget", 5, 1 << 12, 8), ("merge_budget", 5, 1 << 18, 1), ("merge_budget", 0, 1 << 62, 4)]

    def first_match(knob, d, n):  # the library's rule
        for k, dd, n_max, v in got:
            if k == knob and dd in (0, d) and n <= n_max:
                return v
    assert first_match("merge_budget", 5, 1000) == 8
    assert first_match("merge_budget", 5, 100000) == 1
    assert first_match("merge_budget", 5, 10 ** 7) == 4
    assert first_match("merge_budget", 2, 10) == 4


def test_every_knob_has_candidates_defaults_and_a_number(tmp_path):
    for name, (cands, stages) in {**autotune.PER_GROUP, **autotune.PER_BATCH}.items():
        assert name in KNOBS and stages
        assert all(autotune.default_value(name, d) in cands for d in range(1, 9))
    doc = {"entries": [{"knob": "merge_lane", "d": 7, "n_max": 4096, "value": 4}]}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(doc))
    assert load_tuning(str(p)) == [("merge_lane", 7, 4096, 4)]
