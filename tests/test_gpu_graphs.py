"""Phases launched as CUDA graphs give the results of direct launches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _np(res):
    return [(lab.cpu().numpy(), core.cpu().numpy()) for lab, core in res]


def test_graph_phases_match_direct_launches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # every case above the library's graph threshold (2^18 points)
    cases = [synth.workload("tiny", n=300_000, seed=s) for s in (1, 2)] + [synth.workload("ss3d_2m", n=300_000, seed=3)]
    direct = Context(0)
    graphed = Context(0)
    graphed.set_graphs(True)
    for rep in range(3):
        for X, e, m in cases:  # alternating inputs: updates and re-instantiations
            Xd = torch.from_numpy(X).cuda()
            a = _np([direct.dbscan(Xd, e, m)])[0]
            b = _np([graphed.dbscan(Xd, e, m)])[0]
            np.testing.assert_array_equal(a[0], b[0])
            np.testing.assert_array_equal(a[1], b[1])
    st = graphed.graph_stats()
    assert st["launches"] == 3 * 9 and st["instantiations"] >= 3 and st["updates"] > 0
    # the same input again: every phase updates in place
    X, e, m = cases[0]
    Xd = torch.from_numpy(X).cuda()
    graphed.dbscan(Xd, e, m)  # after a different input some phases re-instantiate
    before = graphed.graph_stats()
    for _ in range(3):
        lab, core = graphed.dbscan(Xd, e, m)
    after = graphed.graph_stats()
    assert after["updates"] - before["updates"] == 9 and after["instantiations"] == before["instantiations"]
    want = oracle.grid(X, e, m)
    np.testing.assert_array_equal(lab.cpu().numpy(), want[0])
    # stage timing still works inside graphs
    graphed.set_timing(True)
    graphed.dbscan(Xd, e, m)
    times = graphed.stage_times()
    assert len(times) == 13 and all(v >= 0 for v in times.values()) and sum(times.values()) > 0
    assert 0 < times["sort_downsweep"] <= times["sort"]
    # a small call runs without graphs
    X, e, m = synth.workload("tiny", n=8000, seed=4)
    before = graphed.graph_stats()
    lab, core = graphed.dbscan(torch.from_numpy(X).cuda(), e, m)
    assert graphed.graph_stats() == before
    np.testing.assert_array_equal(lab.cpu().numpy(), oracle.grid(X, e, m)[0])
    direct.close()
    graphed.close()


def test_graph_phases_batched():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    jobs = synth.batch_instances(16, seed=3, n_lo=20_000, n_hi=60_000)  # above the graph threshold in all
    dj = [(torch.from_numpy(X).cuda(), e, m) for X, e, m in jobs]
    ref = _np(Context(0).dbscan_batched(dj))
    ctx = Context(0)
    ctx.set_graphs(True)
    for _ in range(2):
        got = _np(ctx.dbscan_batched(dj))
        for (a, ac), (b, bc) in zip(ref, got):
            np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(ac, bc)
    assert ctx.graph_stats()["launches"] == 6
    ctx.close()
