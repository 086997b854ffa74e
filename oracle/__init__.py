"""CPU oracle for exact DBSCAN -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and
the two share no code.  The arithmetic lives in ``gd_oracle.c`` (plain C,
OpenMP over grids); this module compiles it with gcc on first use and wraps
it with ctypes.

Functions (all inputs are numpy arrays; coordinates int32 [n, d], row-major):

``bruteforce``       the DBSCAN definitions (Section 3.1, Defs. 1-5) as O(n^2)
                     loops; canonical labels.
``grid``             the paper's grid method (Section 4: Eq. 1, Alg. 1, Alg. 3,
                     G13 core rule, LDF union-find merging, border step).
``grid_structure``   non-empty grids and Nei(g) of every grid (Alg. 1, Alg. 3).
``neighbor_counts``  |N_eps(p)| for a list of query points, by brute force.
``mindist_le``       MinDist(A, B) <= eps by Def. 7 or by FastMerging (Alg. 5, with
                     both pruning tests of Alg. 4).
``cell_side``        the integer cell side of Eq. 1 (largest s, d(s-1)^2 <= eps2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgd_oracle.so")

_lib = None
_lock = threading.Lock()

_ERRORS = {1: "invalid argument", 2: "coordinate range too large (d*R^2 >= 2^62)", 3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile gd_oracle.c into a shared library (gcc, OpenMP); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wextra",
           "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_longlong)
    ll = ctypes.c_longlong
    lib.oracle_bruteforce.argtypes = [i32p, ll, ctypes.c_int, ll, ctypes.c_int, i32p, u8p]
    lib.oracle_bruteforce.restype = ctypes.c_int
    lib.oracle_grid.argtypes = [i32p, ll, ctypes.c_int, ll, ctypes.c_int, i32p, u8p, ctypes.c_int, i64p]
    lib.oracle_grid.restype = ctypes.c_int
    lib.oracle_grid_structure.argtypes = [i32p, ll, ctypes.c_int, ll, i64p, i64p, i64p, i64p, i64p, i64p]
    lib.oracle_grid_structure.restype = ll
    lib.oracle_neighbor_counts.argtypes = [i32p, ll, ctypes.c_int, ll, i64p, ll, i64p]
    lib.oracle_neighbor_counts.restype = ctypes.c_int
    lib.oracle_mindist_le.argtypes = [i32p, ll, i32p, ll, ctypes.c_int, ll, ctypes.c_int, i64p]
    lib.oracle_mindist_le.restype = ctypes.c_int
    lib.oracle_cell_side.argtypes = [ll, ctypes.c_int]
    lib.oracle_cell_side.restype = ll
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def use_library(path: str):
    """Point this module at another build of the oracle (the tests use it to
    load copies with planted mistakes).  Returns the previous library."""
    global _lib
    with _lock:
        prev = _lib
        _lib = _bind(ctypes.CDLL(path))
        return prev


def restore_library(lib):
    global _lib
    with _lock:
        _lib = lib


def compile_source(src_path: str, out_path: str):
    """Compile a gd_oracle.c variant with the same flags as build()."""
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", src_path, "-o",
                    out_path, "-lm"], check=True)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _points(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.int32)
    if X.ndim != 2:
        raise ValueError("points must be a 2-D [n, d] array")
    return X


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle: {_ERRORS.get(rc, rc)}")


def bruteforce(X, eps2: int, minpts: int):
    """Labels (int32 [n]) and core flags (bool [n]) by the definitions."""
    X = _points(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    core = np.empty(n, np.uint8)
    _check(_load().oracle_bruteforce(_ptr(X, ctypes.c_int32), n, d, int(eps2), int(minpts),
                                     _ptr(labels, ctypes.c_int32), _ptr(core, ctypes.c_uint8)))
    return labels, core.astype(bool)


def grid(X, eps2: int, minpts: int, merge: str = "plain", return_stats: bool = False):
    """Labels and core flags by the grid method; merge is 'plain' (Def. 7) or
    'fastmerging' (Alg. 5).  With return_stats, also a dict of counters."""
    X = _points(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    core = np.empty(n, np.uint8)
    stats = np.zeros(20, np.int64)
    mode = {"plain": 0, "fastmerging": 1}[merge]
    _check(_load().oracle_grid(_ptr(X, ctypes.c_int32), n, d, int(eps2), int(minpts),
                               _ptr(labels, ctypes.c_int32), _ptr(core, ctypes.c_uint8), mode,
                               _ptr(stats, ctypes.c_longlong)))
    if return_stats:
        return labels, core.astype(bool), dict(grids=int(stats[0]), merge_tests=int(stats[1]),
                                               max_rounds=int(stats[2]), core_grids=int(stats[3]),
                                               kappa_hist=[int(v) for v in stats[4:20]])
    return labels, core.astype(bool)


def grid_structure(X, eps2: int):
    """Non-empty grids and neighbour lists: dict with order [n], cell_start
    [C+1], cell_coord [C, d] (grid identifiers), nei_start [C+1], nei [...]."""
    X = _points(X)
    n, d = X.shape
    lib = _load()
    nn = ctypes.c_longlong(0)
    C = lib.oracle_grid_structure(_ptr(X, ctypes.c_int32), n, d, int(eps2), None, None, None, None,
                                  None, ctypes.byref(nn))
    if C < 0:
        _check(-C)
    order = np.empty(n, np.int64)
    cell_start = np.empty(C + 1, np.int64)
    cell_coord = np.empty((C, d), np.int64)
    nei_start = np.empty(C + 1, np.int64)
    nei = np.empty(max(nn.value, 1), np.int64)
    i64 = ctypes.c_longlong
    C2 = lib.oracle_grid_structure(_ptr(X, ctypes.c_int32), n, d, int(eps2), _ptr(order, i64),
                                   _ptr(cell_start, i64), _ptr(cell_coord, i64), _ptr(nei_start, i64),
                                   _ptr(nei, i64), ctypes.byref(nn))
    assert C2 == C
    return dict(order=order, cell_start=cell_start, cell_coord=cell_coord, nei_start=nei_start,
                nei=nei[: nn.value])


def neighbor_counts(X, eps2: int, query) -> np.ndarray:
    """|N_eps(X[q])| (self included) for each q in query, by brute force."""
    X = _points(X)
    n, d = X.shape
    q = np.ascontiguousarray(query, dtype=np.int64)
    out = np.empty(q.shape[0], np.int64)
    _check(_load().oracle_neighbor_counts(_ptr(X, ctypes.c_int32), n, d, int(eps2),
                                          _ptr(q, ctypes.c_longlong), q.shape[0],
                                          _ptr(out, ctypes.c_longlong)))
    return out


def mindist_le(A, B, eps2: int, method: str = "plain"):
    """(MinDist(A, B) <= eps, rounds): by Def. 7 ('plain') or Alg. 5 ('fastmerging')."""
    A = _points(A)
    B = _points(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("dimension mismatch")
    it = ctypes.c_longlong(0)
    r = _load().oracle_mindist_le(_ptr(A, ctypes.c_int32), A.shape[0], _ptr(B, ctypes.c_int32),
                                  B.shape[0], A.shape[1], int(eps2),
                                  {"plain": 0, "fastmerging": 1}[method], ctypes.byref(it))
    if r < 0:
        raise ValueError("oracle: invalid argument")
    return bool(r), int(it.value)


def cell_side(eps2: int, d: int) -> int:
    return int(_load().oracle_cell_side(int(eps2), int(d)))


def num_threads() -> int:
    return int(_load().oracle_num_threads())
