"""gd_dbscan_noalloc: clustering for callers that cannot allocate device memory.

Such callers (code under a memory manager that owns the device pool, or a
hot loop where allocation is forbidden) get an entry point that takes all of
its scratch from a fixed static device array.  Through the C ABI, its labels
and core flags must equal those of gd_dbscan (bit for bit: both are exact
integer results) on two calls in a row, the second on different data, so that
nothing left in the shared array by one call leaks into the next.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_07580_gb300 import Context, GdError, binding, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs():
    X1, e1, m1 = synth.workload("tiny", n=20000, seed=11)
    X2 = synth.blobs(30000, 3, k=6, sigma=900.0, noise=0.08, seed=12)
    return [(X1, e1, m1), (X2, 600 ** 2, 8), (X1, e1, m1)]


def test_noalloc_matches_gd_dbscan_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = Context(0)
    for k, (X, eps2, minpts) in enumerate(_inputs()):
        Xd = torch.from_numpy(X).cuda()
        want_l, want_c = ctx.dbscan(Xd, eps2, minpts)
        got_l, got_c = binding.dbscan_noalloc(Xd, eps2, minpts)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got_c.cpu().numpy().astype(bool), want_c.cpu().numpy(),
                                      err_msg=f"call {k}: core flags")
        np.testing.assert_array_equal(got_l.cpu().numpy(), want_l.cpu().numpy(), err_msg=f"call {k}: labels")
    ctx.close()


def test_noalloc_rejects_inputs_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = torch.zeros((binding.NOALLOC_MAX_POINTS + 1, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(GdError) as e:
        binding.dbscan_noalloc(X, 100, 3)
    assert e.value.status == binding.GD_ENOMEM


def test_noalloc_allocates_no_device_memory():
    """After a warm-up call (which may load the library's module and back the
    static array), further calls leave the device's free memory unchanged."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload("tiny", n=20000, seed=13)
    Xd = torch.from_numpy(X).cuda()
    lab = torch.empty(len(X), dtype=torch.int32, device="cuda")
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    binding.dbscan_noalloc(Xd, eps2, minpts, labels=lab, is_core=core)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        binding.dbscan_noalloc(Xd, eps2, minpts, labels=lab, is_core=core)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_lists_beyond_the_array_give_enomem_then_recover():
    """Data whose neighbour lists need more than the static array has left
    (65,536 points in 8 dimensions with a large eps: hundreds of neighbour
    grids per grid) are refused with GD_ENOMEM; the next call still matches
    gd_dbscan."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(14)
    X = rng.integers(0, 100000, size=(binding.NOALLOC_MAX_POINTS, 8)).astype(np.int32)
    with pytest.raises(GdError) as e:
        binding.dbscan_noalloc(torch.from_numpy(X).cuda(), 50000 ** 2, 5)
    assert e.value.status == binding.GD_ENOMEM
    X1, e1, m1 = synth.workload("tiny", n=20000, seed=15)
    Xd = torch.from_numpy(X1).cuda()
    ctx = Context(0)
    want_l, want_c = ctx.dbscan(Xd, e1, m1)
    got_l, got_c = binding.dbscan_noalloc(Xd, e1, m1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got_l.cpu().numpy(), want_l.cpu().numpy())
    np.testing.assert_array_equal(got_c.cpu().numpy().astype(bool), want_c.cpu().numpy())
    ctx.close()
