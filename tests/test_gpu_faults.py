"""Failure paths of the library, made on the host or through bounded device
loops -- never by faulting, trapping or hanging the GPU.

- The union-find loops of the merge are bounded: with a tiny retry limit
  they run out, the call returns GD_ETIMEOUT, and the next call with the
  built-in limit equals the oracle on the same context.
- A refused device allocation at any request of a call returns GD_ENOMEM and
  leaves the context usable: the next call equals the oracle.
- A context whose memory cap is too small for an input refuses it with
  GD_ENOMEM and still clusters inputs that fit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, GdError, binding, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def run(ctx, X, eps2, minpts):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy()


def same(got, want, what):
    assert np.array_equal(got[1], want[1]), f"{what}: core flags differ"
    assert np.array_equal(got[0], want[0]), f"{what}: labels differ"


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, eps2, minpts = synth.workload("tiny", n=20000, seed=8)
    return X, eps2, minpts, oracle.grid(X, eps2, minpts)


@pytest.mark.parametrize("order", [0, 1])
def test_union_find_retry_limit_gives_timeout_then_recovers(case, order):
    X, eps2, minpts, want = case
    ctx = Context(0, tuning=[("merge_order", 0, 1 << 62, order)])
    ctx.set_retry_limit(1)
    with pytest.raises(GdError) as e:
        run(ctx, X, eps2, minpts)
    assert e.value.status == binding.GD_ETIMEOUT
    ctx.set_retry_limit(0)
    same(run(ctx, X, eps2, minpts), want, "after the timeout")
    ctx.close()


def test_refused_allocation_at_every_request(case):
    """Refuse the k-th device request of a first call, for every k up to past
    the call's last request: each refusal is GD_ENOMEM (or, for a buffer the
    driver can do without -- the single-pass walk's pool -- a correct result
    without it), and the context then gives the oracle's labels."""
    X, eps2, minpts, want = case
    refused = 0
    for k in range(1, 24):
        ctx = Context(0)
        ctx.inject_alloc_failure(k)
        try:
            got = run(ctx, X, eps2, minpts)
        except GdError as err:
            assert err.status == binding.GD_ENOMEM, (k, str(err))
            refused += 1
            same(run(ctx, X, eps2, minpts), want, f"after a refused request {k}")
        else:
            same(got, want, f"request {k} refused without failing the call, or past the last one")
        ctx.inject_alloc_failure(0)
        ctx.close()
    assert refused >= 5  # the call made several requests that cannot be done without


def test_refused_allocation_on_a_warm_context(case):
    X, eps2, minpts, want = case
    ctx = Context(0)
    run(ctx, X, eps2, minpts)
    X2, e2, m2 = synth.workload("tiny", n=60000, seed=9)  # larger: buffers must grow
    ctx.inject_alloc_failure(3)
    with pytest.raises(GdError) as e:
        run(ctx, X2, e2, m2)
    assert e.value.status == binding.GD_ENOMEM
    same(run(ctx, X2, e2, m2), oracle.grid(X2, e2, m2), "the larger input after the refusal")
    same(run(ctx, X, eps2, minpts), want, "the first input again")
    ctx.close()


def test_memory_cap(case):
    X, eps2, minpts, want = case
    cap = 64 << 20
    ctx = Context(0, arena_bytes=cap)
    same(run(ctx, X, eps2, minpts), want, "within the cap")
    big, eb, mb = synth.workload("ss3d_2m", n=1_000_000, seed=2)
    with pytest.raises(GdError) as e:
        run(ctx, big, eb, mb)
    assert e.value.status == binding.GD_ENOMEM
    assert ctx.bytes_held() <= cap
    same(run(ctx, X, eps2, minpts), want, "within the cap, after the refusal")
    ctx.close()
