"""The asynchronous boundary: gd_dbscan queues, gd_sync finishes.

- A call followed by gd_sync gives the oracle's labels; the second call of
  the same shape is queued without reading anything back.
- Sizes reused from an earlier call that do not fit the new data (longer
  neighbour lists, a wider key layout) make gd_sync run the call again with
  exact sizes: the labels are still the oracle's.
- A coordinate range too large for exact int64 distances is reported by
  gd_sync (GD_ERANGE) when the call was queued without reading the bounds.
- Several calls queued back to back on one stream, then one gd_sync: the
  last call's labels are final (each call finishes its predecessor).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, GdError, binding, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(ctx, X, eps2, minpts, sync=True):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts, sync=False)
    if sync:
        ctx.sync()
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy(), Xd


def same(got, want, what):
    assert np.array_equal(got[1], want[1]), f"{what}: core flags differ"
    assert np.array_equal(got[0], want[0]), f"{what}: labels differ at {int((got[0] != want[0]).sum())}"


@pytest.mark.parametrize("name,n", [("tiny", 20000), ("ss3d_2m", 300000), ("skew5d_10m", 100000)])
def test_queued_call_then_sync(gpu, name, n):
    X, eps2, minpts = synth.workload(name, n=n, seed=21)
    want = oracle.grid(X, eps2, minpts)
    ctx = Context(0)
    same(run(ctx, X, eps2, minpts)[:2], want, "first call")
    assert ctx.last_sizes()["queued"] == 0
    X2, _, _ = synth.workload(name, n=n, seed=22)
    same(run(ctx, X2, eps2, minpts)[:2], oracle.grid(X2, eps2, minpts), "second call")
    assert ctx.last_sizes()["queued"] == 1
    ctx.close()


def test_lists_longer_than_last_time_run_again(gpu):
    rng = np.random.default_rng(23)
    n, eps2, minpts = 40000, 900 ** 2, 5
    sparse = rng.integers(0, 100000, size=(n, 3)).astype(np.int32)
    dense = rng.integers(0, 8000, size=(n, 3)).astype(np.int32)  # same shape, many more neighbours
    ctx = Context(0)
    same(run(ctx, sparse, eps2, minpts)[:2], oracle.grid(sparse, eps2, minpts), "sparse")
    nn_sparse = ctx.last_sizes()["nnbr"]
    same(run(ctx, dense, eps2, minpts)[:2], oracle.grid(dense, eps2, minpts), "dense after sparse")
    assert ctx.last_sizes()["nnbr"] > 2 * nn_sparse
    assert ctx.last_sizes()["queued"] == 0  # the queued attempt did not fit: run again
    ctx.close()


def test_wider_key_layout_than_last_time_runs_again(gpu):
    rng = np.random.default_rng(24)
    n, eps2, minpts = 30000, 200 ** 2, 4
    narrow = rng.integers(0, 2000, size=(n, 3)).astype(np.int32)
    wide = rng.integers(0, 1 << 30, size=(n, 3)).astype(np.int32)  # many more key bits
    ctx = Context(0)
    same(run(ctx, narrow, eps2, minpts)[:2], oracle.grid(narrow, eps2, minpts), "narrow")
    bits = ctx.last_sizes()["key_bits"]
    same(run(ctx, wide, eps2, minpts)[:2], oracle.grid(wide, eps2, minpts), "wide after narrow")
    assert ctx.last_sizes()["key_bits"] > bits
    ctx.close()


def test_range_error_is_deferred_when_queued(gpu):
    rng = np.random.default_rng(25)
    n, eps2, minpts = 5000, 1000 ** 2, 4
    ok = rng.integers(0, 100000, size=(n, 8)).astype(np.int32)
    bad = ok.copy()
    bad[0, 0], bad[1, 0] = -2**31, 2**31 - 1  # d * R^2 >= 2^62
    ctx = Context(0)
    run(ctx, ok, eps2, minpts)
    Xd = torch.from_numpy(bad).cuda()
    ctx.dbscan(Xd, eps2, minpts, sync=False)  # queued: nothing read back
    with pytest.raises(GdError) as e:
        ctx.sync()
    assert e.value.status == binding.GD_ERANGE
    # a fresh context reads the bounds back and refuses while queueing
    ctx2 = Context(0)
    with pytest.raises(GdError) as e2:
        ctx2.dbscan(Xd, eps2, minpts, sync=False)
    assert e2.value.status == binding.GD_ERANGE
    # the first context is usable again
    same(run(ctx, ok, eps2, minpts)[:2], oracle.grid(ok, eps2, minpts), "after the range error")
    ctx.close()
    ctx2.close()


def test_calls_back_to_back_then_one_sync(gpu):
    X, eps2, minpts = synth.workload("tiny", n=20000, seed=26)
    Xd = torch.from_numpy(X).cuda()
    ctx = Context(0)
    outs = []
    for _ in range(4):
        outs.append(ctx.dbscan(Xd, eps2, minpts, sync=False))
    ctx.sync()
    torch.cuda.synchronize()
    want = oracle.grid(X, eps2, minpts)
    for lab, core in outs:
        same((lab.cpu().numpy(), core.cpu().numpy()), want, "back to back")
    ctx.close()


def test_host_buffers_async_on_two_contexts(gpu):
    """gd_dbscan_host_async alternating between two contexts and streams:
    every call's host outputs equal the oracle's after its context's sync,
    including a call whose neighbour lists outgrew the plan (its copies out
    are queued again after the run with exact sizes)."""
    rng = np.random.default_rng(31)
    n, eps2, minpts = 60000, 900 ** 2, 5
    sparse = rng.integers(0, 100000, size=(n, 3)).astype(np.int32)
    dense = rng.integers(0, 8000, size=(n, 3)).astype(np.int32)
    seq = [sparse, sparse, dense, sparse, dense, dense]
    want = {id(sparse): oracle.grid(sparse, eps2, minpts), id(dense): oracle.grid(dense, eps2, minpts)}
    pinned = {k: torch.from_numpy(X).pin_memory() for k, X in ((id(sparse), sparse), (id(dense), dense))}
    ctxs = [Context(0), Context(0)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory())
            for _ in seq]
    for i, X in enumerate(seq):
        c = i % 2
        if i >= 2:  # this context's previous call is finished by the next one; check it now
            ctxs[c].sync(streams[c])
            j = i - 2
            same((outs[j][0].numpy(), outs[j][1].numpy().astype(bool)), want[id(seq[j])], f"call {j}")
        ctxs[c].dbscan_host(pinned[id(X)], eps2, minpts, labels=outs[i][0], is_core=outs[i][1],
                            stream=streams[c], sync=False)
    for c in (0, 1):
        ctxs[c].sync(streams[c])
    for j in (len(seq) - 2, len(seq) - 1):
        same((outs[j][0].numpy(), outs[j][1].numpy().astype(bool)), want[id(seq[j])], f"call {j}")
    for c in ctxs:
        c.close()
