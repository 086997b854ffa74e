"""CUDA path against the CPU oracle, through the C ABI (needs a GB300).

Labels and core flags are integers decided by exact int64 comparisons, so the
bar is bit-exactness: every label, every core flag, and the intermediate grid
structure (sorted permutation, non-empty grids, neighbour lists) equal the
oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2210_07580_gb300 import Context, GdError, binding, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Context(0)
    yield c
    c.close()


def run_gpu(ctx, X, eps2, minpts):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    lab, core = ctx.dbscan(Xd, eps2, minpts)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy()


def assert_same(got, want, what=""):
    gl, gc = got
    wl, wc = want
    if not np.array_equal(gc, wc):
        raise AssertionError(f"{what}: core flags differ at {int((gc != wc).sum())} points")
    if not np.array_equal(gl, wl):
        idx = np.flatnonzero(gl != wl)
        raise AssertionError(f"{what}: labels differ at {len(idx)} points, first {idx[:5]}: "
                             f"got {gl[idx[:5]]} want {wl[idx[:5]]}")


def rand_points(rng, n, d, hi, lattice=1):
    return np.ascontiguousarray((rng.integers(0, hi // lattice, size=(n, d)) * lattice).astype(np.int32))


# ------------------------------------------------------------ small cases

def test_tiny_workload_vs_bruteforce(ctx):
    X, eps2, minpts = synth.workload("tiny")
    assert_same(run_gpu(ctx, X, eps2, minpts), oracle.bruteforce(X, eps2, minpts), "tiny")


@pytest.mark.parametrize("name", ["border_tie_2d.txt", "chain_dup_1d.txt"])
def test_golden_fixtures(ctx, name):
    from golden_io import load_labels_case
    X, eps2, minpts, want_l, want_c = load_labels_case(name)
    gl, gc = run_gpu(ctx, X, eps2, minpts)
    np.testing.assert_array_equal(gc, want_c)
    np.testing.assert_array_equal(gl, want_l)


RANDOM_CASES = [
    # d, n, hi, lattice, eps2, minpts
    (1, 3000, 20000, 1, 400, 4),
    (2, 5000, 4000, 10, 900, 5),
    (2, 7000, 30000, 1, 250000, 12),
    (3, 6000, 3000, 20, 6400, 6),
    (3, 9000, 100000, 1, 250000, 20),
    (4, 5000, 1000, 10, 4000, 5),
    (5, 5000, 500, 10, 3000, 4),
    (6, 4000, 200, 10, 900, 3),
    (7, 4000, 120, 10, 700, 3),
    (8, 3000, 90, 10, 500, 3),
    (2, 2000, 60, 1, 0, 2),          # eps = 0: duplicates only
    (3, 3000, 500, 1, 10**7, 50),    # huge eps: one cluster
    (3, 3000, 100000, 1, 1, 2),      # eps below the spacing: all noise
    (2, 4000, 2000, 1, 2500, 1),     # MinPts = 1: every point core
    (3, 5000, 50000, 1, 90000, 200), # MinPts above most grid sizes
]


@pytest.mark.parametrize("d,n,hi,lattice,eps2,minpts", RANDOM_CASES)
def test_random_cases_vs_oracle(ctx, d, n, hi, lattice, eps2, minpts):
    rng = np.random.default_rng(7919 * d + n + minpts)
    X = rand_points(rng, n, d, hi, lattice)
    X[: n // 25] = X[n // 25: 2 * (n // 25)]  # exact duplicates
    want = oracle.grid(X, eps2, minpts)
    assert_same(run_gpu(ctx, X, eps2, minpts), want, f"d={d} n={n} eps2={eps2} M={minpts}")


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 4095, 4096, 4097, 70001])
def test_ragged_sizes(ctx, n):
    """Sizes around the warp, sort-tile and scan-tile boundaries."""
    rng = np.random.default_rng(n)
    X = rand_points(rng, n, 3, 3000, 1)
    want = oracle.grid(X, 40000, 4)
    assert_same(run_gpu(ctx, X, 40000, 4), want, f"n={n}")


def test_two_word_keys(ctx):
    """d=7 with eps=200: identifiers need 77 bits, the 128-bit key path."""
    rng = np.random.default_rng(5)
    centres = rng.integers(0, 100000, size=(20, 7))
    X = (centres[rng.integers(0, 20, 6000)] + rng.normal(0, 120, size=(6000, 7))).clip(0, 99999)
    X = np.ascontiguousarray(np.vstack([X, rng.integers(0, 100000, size=(1, 7)) * 0 + 99999,
                                        np.zeros((1, 7))]).astype(np.int32))
    want = oracle.grid(X, 200 ** 2, 5)
    assert_same(run_gpu(ctx, X, 200 ** 2, 5), want, "two-word keys")
    assert ctx.last_sizes()["key_bits"] > 64


def test_negative_and_offset_coordinates(ctx):
    rng = np.random.default_rng(17)
    X = rand_points(rng, 5000, 3, 20000, 1) - 10000 - 2**30
    want = oracle.grid(X, 250000, 6)
    assert_same(run_gpu(ctx, X, 250000, 6), want, "offset")


# ------------------------------------------------- intermediate structure

def refined_neighbours(X, eps2, gs):
    """The GPU's neighbour lists from the oracle's grid-level Nei(g): the grids
    of Nei(g) whose boxes are within eps of g's box, where a grid's box is the
    box of its points, or its whole identifier range when it holds more than
    1024 points (a symmetric relation)."""
    cs, ns, nei, order = gs["cell_start"], gs["nei_start"], gs["nei"], gs["order"]
    Xs = X[order].astype(np.int64)
    lo = np.minimum.reduceat(Xs, cs[:-1], axis=0)
    hi = np.maximum.reduceat(Xs, cs[:-1], axis=0)
    big = np.diff(cs) > 1024
    if big.any():
        s = oracle.cell_side(eps2, X.shape[1])
        base = X.min(0).astype(np.int64) + gs["cell_coord"][big] * s
        lo[big], hi[big] = base, base + s - 1
    out = []
    for c in range(len(cs) - 1):
        nb = nei[ns[c]:ns[c + 1]]
        gap = np.maximum(0, np.maximum(lo[nb] - hi[c], lo[c] - hi[nb]))
        out.append(sorted(int(v) for v in nb[(gap ** 2).sum(1) <= eps2]))
    return out


def test_grid_structure_matches_oracle(ctx):
    """Sorted permutation (stable), non-empty grids, and neighbour lists: the
    oracle's Nei(g) (Alg. 3) narrowed to grids whose point boxes are within
    eps, which must still hold every grid with a point within eps."""
    X, eps2, minpts = synth.workload("tiny", n=8000, seed=2)
    run_gpu(ctx, X, eps2, minpts)
    sz = ctx.last_sizes()
    gs = oracle.grid_structure(X, eps2)
    C = sz["grids"]
    assert C == len(gs["cell_start"]) - 1
    assert sz["side"] == oracle.cell_side(eps2, 2)
    perm = ctx.copy_view(binding.VIEW_PERM, np.int32, len(X))
    np.testing.assert_array_equal(perm, gs["order"])
    np.testing.assert_array_equal(ctx.copy_view(binding.VIEW_CELL_START, np.int32, C + 1), gs["cell_start"])
    np.testing.assert_array_equal(ctx.copy_view(binding.VIEW_CELL_COORD, np.int32, C * 2).reshape(C, 2),
                                  gs["cell_coord"])
    ns = ctx.copy_view(binding.VIEW_NBR_START, np.int32, C + 1)
    nb = ctx.copy_view(binding.VIEW_NBR, np.int32, int(ns[-1]))
    want = refined_neighbours(X, eps2, gs)
    for c in range(C):
        assert sorted(nb[ns[c]:ns[c + 1]]) == want[c], c
    # completeness: every pair of points within eps lies in neighbouring grids
    cell_of = np.empty(len(X), np.int64)
    for c in range(C):
        cell_of[gs["order"][gs["cell_start"][c]:gs["cell_start"][c + 1]]] = c
    sub = np.random.default_rng(0).choice(len(X), 1500, replace=False)
    D = ((X[sub, None, :].astype(np.int64) - X[None, :, :]) ** 2).sum(-1)
    nsets = [set(nb[ns[c]:ns[c + 1]].tolist()) for c in range(C)]
    I, J = np.nonzero(D <= eps2)
    for a, b2 in zip(sub[I], J):
        assert cell_of[b2] in nsets[cell_of[a]]


def test_worked_example_neighbours(ctx):
    """The constructed Fig. 1 layout: the GPU's grids and their order are the
    paper's; its list for g6 is the oracle's Nei(g6) (pinned to the worked
    example) narrowed by point boxes."""
    from golden_io import load_grid_case
    case = load_grid_case("fig2_neighbors_2d.txt")
    X, eps2 = case["X"], case["eps2"]
    run_gpu(ctx, X, eps2, case["minpts"])
    sz = ctx.last_sizes()
    assert sz["grids"] == 9 and sz["side"] == 11
    coord = ctx.copy_view(binding.VIEW_CELL_COORD, np.int32, 18).reshape(9, 2)
    assert [tuple(c) for c in coord] == [case["grids"][k] for k in range(1, 10)]
    ns = ctx.copy_view(binding.VIEW_NBR_START, np.int32, 10)
    nb = ctx.copy_view(binding.VIEW_NBR, np.int32, int(ns[-1]))
    gs = oracle.grid_structure(X, eps2)
    q, paper = case["query"]
    got = sorted(int(v) + 1 for v in nb[ns[q - 1]:ns[q]])
    assert got == [v + 1 for v in refined_neighbours(X, eps2, gs)[q - 1]]
    assert set(got) <= set(paper)


# ------------------------------------------------------------ ABI paths

def test_host_entry_point_matches_device(ctx):
    X, eps2, minpts = synth.workload("tiny", n=12000, seed=4)
    dev = run_gpu(ctx, X, eps2, minpts)
    hl, hc = ctx.dbscan_host(torch.from_numpy(X).pin_memory(), eps2, minpts)
    np.testing.assert_array_equal(hl.numpy(), dev[0])
    np.testing.assert_array_equal(hc.numpy().astype(bool), dev[1])


def test_errors_and_empty(ctx):
    Xd = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    lab, core = ctx.dbscan(Xd, 10, 3)
    assert lab.numel() == 0
    with pytest.raises(GdError) as e:
        ctx.dbscan(torch.zeros((5, 9), dtype=torch.int32, device="cuda"), 10, 3)
    assert e.value.status == binding.GD_EINVAL
    with pytest.raises(GdError) as e:
        ctx.dbscan(torch.zeros((5, 2), dtype=torch.int32, device="cuda"), -1, 3)
    assert e.value.status == binding.GD_EINVAL
    big = torch.tensor([[-2**31], [2**31 - 1]], dtype=torch.int32, device="cuda")
    with pytest.raises(GdError) as e:
        ctx.dbscan(big, 10, 1)
    assert e.value.status == binding.GD_ERANGE
    wide = torch.from_numpy(np.array([[0] * 8, [99999] * 8], np.int32)).cuda()
    with pytest.raises(GdError) as e:  # 8 x 17 identifier bits > 128
        ctx.dbscan(wide, 0, 1)
    assert e.value.status == binding.GD_ERANGE
    # the context stays usable after errors
    X, eps2, minpts = synth.workload("tiny", n=3000)
    assert_same(run_gpu(ctx, X, eps2, minpts), oracle.grid(X, eps2, minpts), "after errors")


def test_context_reuse_across_sizes(ctx):
    for n, seed in [(50000, 1), (2000, 2), (120000, 3), (7000, 4)]:
        X, eps2, minpts = synth.workload("tiny", n=n, seed=seed)
        assert_same(run_gpu(ctx, X, eps2, minpts), oracle.grid(X, eps2, minpts), f"n={n}")


# ------------------------------------------------ full-size workloads

@pytest.mark.parametrize("name", ["ss3d_2m", "ss3d_10m", "skew5d_10m"])
def test_full_size_workloads(ctx, name):
    """The benchmark's workloads at full size, every label against the grid
    oracle (which is itself pinned to brute force on small inputs)."""
    X, eps2, minpts = synth.workload(name)
    got = run_gpu(ctx, X, eps2, minpts)
    want = oracle.grid(X, eps2, minpts)
    assert_same(got, want, name)


@pytest.mark.parametrize("gap_extra,d", [(0, 2), (1, 2), (0, 3), (1, 3)])
def test_dense_slabs_rare_or_no_witness(ctx, gap_extra, d):
    """Two dense slabs whose facing grids are neighbours: with the gap equal to
    eps exactly one planted pair of points is a witness (merge), with eps + 1
    there is none.  Large core sets on both sides drive the pairs past the
    warp's tile budget into FastMerging, which must prove 'no' exactly or find
    the one witness."""
    rng = np.random.default_rng(100 + 10 * d + gap_extra)
    eps = 300
    n_side = 60000
    A = rng.integers(0, 3000, size=(n_side, d))
    A[:, 0] = rng.integers(0, 2001, size=n_side)
    B = rng.integers(0, 3000, size=(n_side, d))
    B[:, 0] = rng.integers(0, 2001, size=n_side) + 2000 + eps + gap_extra + 1
    # keep the facing faces sparse except for the planted pair
    A = A[A[:, 0] < 1990]
    B = B[B[:, 0] > 2000 + eps + gap_extra + 11]
    pa = np.zeros((1, d), np.int64)
    pa[0, 0] = 2000
    pa[0, 1:] = 1500
    pb = pa.copy()
    pb[0, 0] = 2000 + eps + gap_extra
    X = np.ascontiguousarray(np.vstack([A, B, pa, pb, A[:5] + 1]).astype(np.int32))
    X = np.ascontiguousarray(X[rng.permutation(len(X))])
    eps2 = eps * eps
    want = oracle.grid(X, eps2, 5, merge="fastmerging")
    got = run_gpu(ctx, X, eps2, 5)
    assert_same(got, want, f"slabs d={d} gap_extra={gap_extra}")
    # the planted points must be core for the test to mean anything
    assert want[1].sum() > 0.9 * len(X)


# ------------------------------------------------------------ batches

def batch_jobs(seed, k, n_lo=200, n_hi=20000):
    """Uneven instances: sizes log-uniform, d in {2,3,5,7}, eps and MinPts
    swept, blobs plus noise."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(k):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(rng.choice([2, 3, 5, 7]))
        eps = int(rng.uniform(200, 2000))
        minpts = int(rng.choice([5, 10, 50, 100]))
        X = synth.blobs(n, d, k=int(rng.integers(2, 8)), sigma=float(rng.uniform(300, 3000)), noise=0.05,
                        seed=int(rng.integers(1 << 30)))
        jobs.append((X, eps * eps, minpts))
    return jobs


def test_batched_equals_single_and_oracle(ctx):
    jobs = batch_jobs(2024, 24)
    dev_jobs = [(torch.from_numpy(X).cuda(), e, m) for X, e, m in jobs]
    res = ctx.dbscan_batched(dev_jobs)
    torch.cuda.synchronize()
    for i, ((X, e, m), (lab, core)) in enumerate(zip(jobs, res)):
        want = oracle.grid(X, e, m)
        assert_same((lab.cpu().numpy(), core.cpu().numpy()), want, f"batch instance {i} (n={len(X)}, d={X.shape[1]})")
    # each instance alone gives the same result
    for i in (0, 7, 23):
        X, e, m = jobs[i]
        single = run_gpu(ctx, X, e, m)
        np.testing.assert_array_equal(single[0], res[i][0].cpu().numpy())


def clustered(rng, n, d, hi, sigma, k=6):
    c = rng.integers(0, hi, size=(k, d))
    X = c[np.arange(n) % k] + rng.normal(0, sigma, size=(n, d))
    return np.ascontiguousarray(X.clip(0, hi - 1).astype(np.int32))


@pytest.mark.parametrize("d,eps2,width", [
    (4, 260400, 8),             # s = 256: four 8-bit offsets fill the 32-bit word
    (2, 2 * 40000 ** 2, 16),    # s = 40001: two 16-bit offsets
    (3, 3 * 1000 ** 2, 10),     # s = 1001: 30 bits
    (3, 3 * 1500 ** 2, 11),     # s = 1501: 33 bits, past the word: the input rows are gathered
])
def test_grid_order_rows_from_in_cell_offsets(ctx, d, eps2, width):
    """The compaction rebuilds each grid-order row from its identifiers and
    the point's in-cell offsets (Eq. 1: x_j = mn_j + id_j * s + offset_j)
    when the d offsets fit one 32-bit word, and gathers the input row
    otherwise; the labels equal the oracle's either way, on coordinates far
    below zero."""
    s = oracle.cell_side(eps2, d)
    assert (s - 1).bit_length() == width
    rng = np.random.default_rng(100 + d + width)
    X = np.vstack([clustered(rng, 24000, d, 60 * s, sigma=3 * s), rand_points(rng, 6000, d, 60 * s)])
    X = np.ascontiguousarray((X.astype(np.int64) - (1 << 30) - 12345).astype(np.int32))
    got = run_gpu(ctx, X, eps2, 20)
    assert ctx.last_sizes()["key_class"] == 0
    want = oracle.grid(X, eps2, 20)
    assert_same(got, want, f"d={d} offset width {width}")
    # clusters, border points and noise all present
    assert len(np.unique(want[0][want[0] >= 0])) > 1 and (want[0] < 0).any() and (want[1] == 0).any()


@pytest.mark.parametrize("key_class,n,d,hi,eps2,kind", [
    (0, 600_000, 3, 1 << 20, 5000 ** 2, "uniform"),    # packed keys, 147 sort tiles, most grids distinct
    (0, 600_000, 3, 1 << 20, 5000 ** 2, "clustered"),  # long runs of equal digits in every tile
    (1, 300_000, 6, 1 << 24, 6 << 28, "clustered"),    # 64-bit key + index values, 74 sort tiles
])
def test_sort_order_over_many_tiles(ctx, key_class, n, d, hi, eps2, kind):
    """Over many sort tiles (each tile takes its digit offsets from the tiles
    before it), the sort gives the oracle's stable grid order (Alg. 1: ties
    in input order) and its grids."""
    rng = np.random.default_rng(n + d)
    if kind == "uniform":
        X = rng.integers(0, hi, size=(n, d)).astype(np.int32)
    else:
        X = clustered(rng, n, d, hi, sigma=float(np.sqrt(eps2)) * 0.5)
    run_gpu(ctx, X, eps2, 4)
    sz = ctx.last_sizes()
    assert sz["key_class"] == key_class
    gs = oracle.grid_structure(X, eps2)
    np.testing.assert_array_equal(ctx.copy_view(binding.VIEW_PERM, np.int32, n), gs["order"])
    C = sz["grids"]
    assert C == len(gs["cell_start"]) - 1
    np.testing.assert_array_equal(ctx.copy_view(binding.VIEW_CELL_START, np.int32, C + 1), gs["cell_start"])


@pytest.mark.parametrize("key_class,n,d,hi,eps2", [
    (0, 5000, 2, 100_000, 800 ** 2),         # 16 key bits + 13 index bits: packed
    (1, 5000, 6, 1 << 24, 6 << 28),          # 60 key bits + 13 index bits: 64-bit key + index
    (2, 3000, 8, 1 << 24, 8 << 20),          # 112 key bits: 128-bit key + index
])
def test_every_sort_key_class(ctx, key_class, n, d, hi, eps2):
    """Each sort key layout gives the oracle's labels and its stable grid
    order (ties in input order)."""
    rng = np.random.default_rng(key_class + 40)
    X = clustered(rng, n, d, hi, sigma=float(np.sqrt(eps2)) * 0.2)
    got = run_gpu(ctx, X, eps2, 4)
    assert ctx.last_sizes()["key_class"] == key_class
    assert_same(got, oracle.grid(X, eps2, 4), f"key class {key_class}")
    assert len(np.unique(got[0][got[0] >= 0])) > 1
    gs = oracle.grid_structure(X, eps2)
    np.testing.assert_array_equal(ctx.copy_view(binding.VIEW_PERM, np.int32, n), gs["order"])


def test_cluster_ids_identical_over_repeated_runs(ctx):
    """A sparse 7-d instance (124,710 points, one-point grids) on which a race
    in resolving cluster ids once left a grid with a private id in about one
    run of 60: every run, in a reused or a fresh context, equals the oracle."""
    (X, e, m), = synth.batch_instances(256, seed=21, only={66})
    want = oracle.grid(X, e, m)
    Xd = torch.from_numpy(X).cuda()
    for rep in range(60):
        c = ctx if rep % 2 else Context(0)
        lab, core = c.dbscan(Xd, e, m)
        torch.cuda.synchronize()
        assert_same((lab.cpu().numpy(), core.cpu().numpy()), want, f"run {rep}")
        if c is not ctx:
            c.close()


def test_batched_mixed_key_widths_and_tiny(ctx):
    """One batch mixing 64- and 128-bit keys, a one-point instance and d=1."""
    rng = np.random.default_rng(9)
    jobs = [
        (rand_points(rng, 1, 3, 1000), 100, 1),
        (rand_points(rng, 500, 1, 5000), 400, 3),
        (np.ascontiguousarray(np.vstack([rng.normal(50000, 300, size=(3000, 7)), np.zeros((1, 7)),
                                         np.full((1, 7), 99999)]).clip(0, 99999).astype(np.int32)), 200 ** 2, 5),
        (rand_points(rng, 4000, 2, 3000), 2500, 4),
    ]
    res = ctx.dbscan_batched([(torch.from_numpy(X).cuda(), e, m) for X, e, m in jobs])
    torch.cuda.synchronize()
    for i, ((X, e, m), (lab, core)) in enumerate(zip(jobs, res)):
        assert_same((lab.cpu().numpy(), core.cpu().numpy()), oracle.grid(X, e, m), f"mixed instance {i}")


def test_labels_without_core_flags(ctx):
    """is_core may be NULL: labels only, alone and in a batch that mixes
    instances with and without core flags (labels are then written directly,
    with flags as one packed word split afterwards)."""
    rng = np.random.default_rng(12)
    jobs = [
        (rand_points(rng, 6000, 3, 4000), 90 ** 2, 6),
        (rand_points(rng, 3000, 2, 2000), 60 ** 2, 4),
        (rand_points(rng, 5000, 5, 3000), 400 ** 2, 5),
    ]
    want = [oracle.grid(X, e, m) for X, e, m in jobs]
    # single instance through the raw entry point
    X, e, m = jobs[0]
    Xd = torch.from_numpy(X).cuda()
    lab = torch.full((len(X),), -7, dtype=torch.int32, device="cuda")
    ctx._check(ctx._lib.gd_dbscan(ctx._h, Xd.data_ptr(), len(X), X.shape[1], e, m, lab.data_ptr(), None,
                                  binding._stream_handle(None)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lab.cpu().numpy(), want[0][0])
    # batch: core flags for the middle instance only
    arr = (binding.GdInstance * len(jobs))()
    keep, outs = [], []
    for i, (X, e, m) in enumerate(jobs):
        Xd = torch.from_numpy(X).cuda()
        lab = torch.full((len(X),), -7, dtype=torch.int32, device="cuda")
        core = torch.full((len(X),), 7, dtype=torch.uint8, device="cuda") if i == 1 else None
        keep.append(Xd)
        outs.append((lab, core))
        arr[i] = binding.GdInstance(Xd.data_ptr(), len(X), X.shape[1], e, m, lab.data_ptr(),
                                    core.data_ptr() if core is not None else None)
    ctx._check(ctx._lib.gd_dbscan_batched(ctx._h, len(jobs), binding.ctypes.cast(arr, binding.ctypes.c_void_p),
                                          binding._stream_handle(None)))
    torch.cuda.synchronize()
    for i, ((lab, core), (wl, wc)) in enumerate(zip(outs, want)):
        np.testing.assert_array_equal(lab.cpu().numpy(), wl, err_msg=f"instance {i}")
        if core is not None:
            np.testing.assert_array_equal(core.cpu().numpy().astype(bool), wc.astype(bool),
                                          err_msg=f"instance {i} core")


def test_batched_workload_at_full_size_vs_oracle(ctx):
    """The bench's batched workload itself (256 instances, n up to 5e5,
    d in {2,3,5,7}) in one call; the largest instance of each dimension and
    a spread of others are checked against the oracle element by element,
    and every instance against its own single call."""
    jobs = synth.batch_instances(256, seed=7)
    dev_jobs = [(torch.from_numpy(X).cuda(), e, m) for X, e, m in jobs]
    res = ctx.dbscan_batched(dev_jobs)
    torch.cuda.synchronize()
    pick = set(range(0, 256, 23))
    for dd in (2, 3, 5, 7):
        ids = [i for i, (X, _, _) in enumerate(jobs) if X.shape[1] == dd]
        pick.add(max(ids, key=lambda i: len(jobs[i][0])))
    for i in sorted(pick):
        X, e, m = jobs[i]
        want = oracle.grid(X, e, m)
        assert_same((res[i][0].cpu().numpy(), res[i][1].cpu().numpy()), want,
                    f"batched instance {i} (n={len(X)}, d={X.shape[1]})")
    for i, (X, e, m) in enumerate(jobs):
        single = run_gpu(ctx, X, e, m)
        np.testing.assert_array_equal(single[0], res[i][0].cpu().numpy(), err_msg=f"instance {i}")
