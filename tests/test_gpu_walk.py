"""Neighbour lists on sparse data in 2 to 7 dimensions, where most grids hold
one or two points and the query (Alg. 3) descends every level: the lists
equal the oracle's Nei(g) narrowed by point boxes (as in the parity tests,
whose structure test is 2-d) and the labels equal the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, binding, synth  # noqa: E402
from test_gpu_parity import refined_neighbours  # noqa: E402

pytestmark = pytest.mark.gpu


# scale 1000 puts eps2 above 2^31, where the query's offsets take 64 bits
@pytest.mark.parametrize("d,eps,scale", [(2, 700, 1), (4, 900, 1), (6, 1500, 1), (7, 1800, 1), (4, 900, 1000),
                                         (6, 1500, 1000)])
def test_sparse_lists_and_labels(d, eps, scale):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = synth.blobs(12000, d, k=4, sigma=2500.0, noise=0.05, seed=100 + d) * np.int32(scale)
    eps2, minpts = (eps * scale) ** 2, 5
    ctx = Context(0)
    Xd = torch.from_numpy(X).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts)
    torch.cuda.synchronize()
    want = oracle.grid(X, eps2, minpts)
    np.testing.assert_array_equal(core.cpu().numpy(), want[1].astype(bool))
    np.testing.assert_array_equal(lab.cpu().numpy(), want[0])
    C = ctx.last_sizes()["grids"]
    ns = ctx.copy_view(binding.VIEW_NBR_START, np.int32, C + 1)
    nb = ctx.copy_view(binding.VIEW_NBR, np.int32, int(ns[-1]))
    ctx.close()
    gs = oracle.grid_structure(X, eps2)
    assert C == len(gs["cell_start"]) - 1
    ref = refined_neighbours(X, eps2, gs)
    for c in range(C):
        assert sorted(nb[ns[c]:ns[c + 1]].tolist()) == ref[c], c
