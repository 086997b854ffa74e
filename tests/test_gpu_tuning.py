"""Tuning knobs change speed, never labels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_07580_gb300 import Context, GdError, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LOW = [("merge_budget", 0, 1 << 62, 1), ("merge_lane", 0, 1 << 62, 1), ("merge_small", 0, 1 << 62, 32),
       ("core_bands", 0, 1 << 62, 0), ("fm_blocks", 0, 1 << 62, 152), ("walk_blocks", 0, 1 << 62, 152),
       ("merge_order", 0, 1 << 62, 0), ("core_mode", 0, 1 << 62, 0)]
HIGH = [("merge_budget", 0, 1 << 62, 64), ("merge_lane", 0, 1 << 62, 256), ("merge_small", 0, 1 << 62, 1024),
        ("core_bands", 0, 1 << 62, 65536), ("fm_blocks", 0, 1 << 62, 152 * 128),
        ("walk_blocks", 0, 1 << 62, 152 * 128), ("core_mode", 0, 1 << 62, 1)]
# the per-point core count with and without bands, the per-grid one with bands
POINT_BANDS = [("core_mode", 0, 1 << 62, 0), ("core_bands", 0, 1 << 62, 65536)]
GRID_BANDS = [("core_mode", 0, 1 << 62, 1), ("core_bands", 0, 1 << 62, 65536)]


def test_knob_extremes_give_identical_labels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    jobs = synth.batch_instances(24, seed=5, n_lo=300, n_hi=60000)
    dj = [(torch.from_numpy(X).cuda(), e, m) for X, e, m in jobs]
    res = {}
    for name, table in (("none", None), ("low", LOW), ("high", HIGH), ("default", "default"),
                        ("point_bands", POINT_BANDS), ("grid_bands", GRID_BANDS)):
        ctx = Context(0, tuning=table)
        out = ctx.dbscan_batched(dj)
        torch.cuda.synchronize()
        res[name] = [(lab.cpu().numpy(), core.cpu().numpy()) for lab, core in out]
        ctx.close()
    for name in ("low", "high", "default", "point_bands", "grid_bands"):
        for i, ((a, ac), (b, bc)) in enumerate(zip(res["none"], res[name])):
            np.testing.assert_array_equal(ac, bc, err_msg=f"{name} core {i}")
            np.testing.assert_array_equal(a, b, err_msg=f"{name} labels {i}")


def test_knob_resolution_and_validation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = Context(0, tuning=None)
    assert ctx.get_knob("merge_budget", 3, 1000) == 2
    ctx.set_tuning([("merge_budget", 5, 4096, 8), ("merge_budget", 0, 1 << 62, 4)])
    assert ctx.get_knob("merge_budget", 5, 4096) == 8
    assert ctx.get_knob("merge_budget", 5, 4097) == 4
    assert ctx.get_knob("merge_budget", 3, 10) == 4
    assert ctx.get_knob("core_bands", 5, 10) == 128
    for bad in ([("merge_budget", 0, 10, 0)], [("merge_small", 0, 10, 2048)], [("merge_budget", 9, 10, 2)],
                [(99, 0, 10, 1)], [("walk_blocks", 0, -1, 304)]):
        with pytest.raises(GdError):
            ctx.set_tuning(bad)
    assert ctx.get_knob("merge_budget", 5, 4096) == 8  # unchanged by the rejected tables
    ctx.set_tuning([])
    assert ctx.get_knob("merge_budget", 5, 4096) == 2
    ctx.close()
