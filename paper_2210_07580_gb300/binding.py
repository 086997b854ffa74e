"""ctypes binding of libgdbscan (include/gdbscan.h).

Argument marshalling only: every step of the clustering runs in the CUDA
library.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or fails to load, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgdbscan.so")

GD_OK, GD_EINVAL, GD_ERANGE, GD_ENOMEM, GD_ECUDA, GD_ETIMEOUT, GD_EBUSY = range(7)
VIEW_PERM, VIEW_CELL_START, VIEW_CELL_COORD, VIEW_NBR_START, VIEW_NBR, VIEW_CORE_SORTED, VIEW_CELL_CID = range(7)


class GdInstance(ctypes.Structure):
    """gd_instance of include/gdbscan.h."""
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int), ("eps2", ctypes.c_int64),
                ("minpts", ctypes.c_int32), ("labels", ctypes.c_void_p), ("is_core", ctypes.c_void_p),
                ("eps2_yes", ctypes.c_int64)]


class GdTuning(ctypes.Structure):
    """gd_tuning of include/gdbscan.h."""
    _fields_ = [("knob", ctypes.c_int32), ("d", ctypes.c_int32), ("n_max", ctypes.c_int64), ("value", ctypes.c_int32)]


# gd_knob of include/gdbscan.h
KNOBS = {"merge_budget": 1, "merge_lane": 2, "merge_small": 3, "core_bands": 4, "fm_blocks": 5, "walk_blocks": 6,
         "merge_order": 7, "core_mode": 8}
# tuning table shipped with the package (written by autotune.py on a GB300)
DEFAULT_TUNING = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


class GdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gdbscan error {status}: {msg}")
        self.status = status


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libgdbscan.so (built by paper_2210_07580_gb300._build).  Raises if
    it is absent: the clustering has no other implementation."""
    global _lib
    with _lib_lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgdbscan.so not found at {p}: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.gd_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
        lib.gd_create.restype = ctypes.c_int
        lib.gd_destroy.argtypes = [vp]
        lib.gd_destroy.restype = None
        lib.gd_workspace_bytes.argtypes = [i64, ctypes.c_int]
        lib.gd_workspace_bytes.restype = ctypes.c_size_t
        lib.gd_dbscan.argtypes = [vp, vp, i64, ctypes.c_int, i64, i32, vp, vp, vp]
        lib.gd_dbscan.restype = ctypes.c_int
        lib.gd_sync.argtypes = [vp, vp]
        lib.gd_sync.restype = ctypes.c_int
        lib.gd_dbscan_host.argtypes = [vp, vp, i64, ctypes.c_int, i64, i32, vp, vp, vp]
        lib.gd_dbscan_host.restype = ctypes.c_int
        lib.gd_dbscan_host_async.argtypes = [vp, vp, i64, ctypes.c_int, i64, i32, vp, vp, vp]
        lib.gd_dbscan_host_async.restype = ctypes.c_int
        lib.gd_status_str.argtypes = [ctypes.c_int]
        lib.gd_status_str.restype = ctypes.c_char_p
        lib.gd_last_error.argtypes = [vp]
        lib.gd_last_error.restype = ctypes.c_char_p
        lib.gd_last_sizes.argtypes = [vp, ctypes.POINTER(i64)]
        lib.gd_last_sizes.restype = ctypes.c_int
        lib.gd_copy_view.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
        lib.gd_copy_view.restype = ctypes.c_int
        lib.gd_set_timing.argtypes = [vp, ctypes.c_int]
        lib.gd_set_timing.restype = ctypes.c_int
        lib.gd_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.c_int]
        lib.gd_stage_times.restype = ctypes.c_int
        lib.gd_set_retry_limit.argtypes = [vp, i32]
        lib.gd_set_retry_limit.restype = ctypes.c_int
        lib.gd_inject_alloc_failure.argtypes = [vp, i32]
        lib.gd_inject_alloc_failure.restype = ctypes.c_int
        lib.gd_set_stats.argtypes = [vp, ctypes.c_int]
        lib.gd_set_stats.restype = ctypes.c_int
        lib.gd_run_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]
        lib.gd_run_stats.restype = ctypes.c_int
        lib.gd_distance_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.gd_distance_peak.restype = ctypes.c_int
        lib.gd_ctx_bytes.argtypes = [vp]
        lib.gd_ctx_bytes.restype = ctypes.c_size_t
        lib.gd_ctx_trim.argtypes = [vp]
        lib.gd_ctx_trim.restype = ctypes.c_int
        lib.gd_dbscan_batched.argtypes = [vp, ctypes.c_int, vp, vp]
        lib.gd_dbscan_batched.restype = ctypes.c_int
        lib.gd_dbscan_noalloc.argtypes = [vp, i64, ctypes.c_int, i64, i32, vp, vp, vp]
        lib.gd_dbscan_noalloc.restype = ctypes.c_int
        lib.gd_set_graphs.argtypes = [vp, ctypes.c_int]
        lib.gd_set_graphs.restype = ctypes.c_int
        lib.gd_graph_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        lib.gd_graph_stats.restype = ctypes.c_int
        lib.gd_set_tuning.argtypes = [vp, vp, ctypes.c_int]
        lib.gd_set_tuning.restype = ctypes.c_int
        lib.gd_get_knob.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, ctypes.POINTER(ctypes.c_int32)]
        lib.gd_get_knob.restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


def load_tuning(path: str):
    """A tuning table written by autotune.py: a list of (knob, d, n_max, value)."""
    import json
    with open(path) as f:
        doc = json.load(f)
    return [(e["knob"], e["d"], e["n_max"], e["value"]) for e in doc["entries"]]


def eps2_from_eps(eps) -> int:
    """floor(eps^2) computed exactly: for integer points dist <= eps exactly
    when dist^2 <= floor(eps^2).  Accepts int, float, Fraction or a decimal
    string."""
    f = Fraction(eps) if not isinstance(eps, float) else Fraction(eps)
    if f < 0:
        raise ValueError("eps must be >= 0")
    sq = f * f
    return sq.numerator // sq.denominator


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Context:
    """One gd_ctx: a device workspace reused across calls.  Not thread-safe."""

    def __init__(self, device: int = 0, tuning="default", graphs: bool = True, arena_bytes: int = 0):
        """tuning: "default" loads the table shipped with the package (if
        present), None keeps the built-in defaults, or a list of entries as
        for set_tuning.  graphs: launch each phase of a call as a CUDA graph
        kept by the context (gd_set_graphs).  arena_bytes: cap on the device
        memory the context may hold (0: none)."""
        self._lib = load_library()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = self._lib.gd_create(ctypes.byref(h), self.device, int(arena_bytes))
        if st != GD_OK:
            raise GdError(st, self._lib.gd_status_str(st).decode())
        self._h = h
        if graphs:
            self.set_graphs(True)
        if tuning == "default":
            if os.path.exists(DEFAULT_TUNING):
                self.set_tuning(load_tuning(DEFAULT_TUNING))
        elif tuning is not None:
            self.set_tuning(tuning)

    def set_tuning(self, entries):
        """Replace the tuning table: entries of (knob, d, n_max, value), knob
        a name of KNOBS or its number, d = 0 for any dimension.  The first
        entry matching a group's dimension and largest size wins."""
        arr = (GdTuning * max(len(entries), 1))()
        for i, (kn, d, n_max, value) in enumerate(entries):
            arr[i] = GdTuning(KNOBS[kn] if isinstance(kn, str) else int(kn), int(d), int(n_max), int(value))
        self._check(self._lib.gd_set_tuning(self._h, ctypes.cast(arr, ctypes.c_void_p), len(entries)))

    def set_graphs(self, enable: bool):
        """Launch each phase of a call as a CUDA graph kept by the context."""
        self._check(self._lib.gd_set_graphs(self._h, 1 if enable else 0))

    def graph_stats(self) -> dict:
        out = (ctypes.c_int64 * 3)()
        self._check(self._lib.gd_graph_stats(self._h, out))
        return {"launches": int(out[0]), "updates": int(out[1]), "instantiations": int(out[2])}

    def get_knob(self, knob, d: int, n: int) -> int:
        v = ctypes.c_int32()
        self._check(self._lib.gd_get_knob(self._h, KNOBS[knob] if isinstance(knob, str) else int(knob), int(d),
                                          int(n), ctypes.byref(v)))
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != GD_OK:
            msg = self._lib.gd_last_error(self._h).decode() or self._lib.gd_status_str(st).decode()
            raise GdError(st, msg)

    # -- clustering
    def sync(self, stream=None):
        """gd_sync: finish the queued call and raise GdError if it failed."""
        self._check(self._lib.gd_sync(self._h, _stream_handle(stream)))

    def dbscan(self, X, eps2: int, minpts: int, labels=None, is_core=None, stream=None, sync: bool = True,
               eps2_yes: int = 0):
        """Cluster the device tensor X (torch.int32, [n, d], contiguous, on this
        context's device).  Returns (labels int32 [n], is_core bool [n]) as
        device tensors (or fills the given ones; is_core must be uint8/bool).
        With sync=False the call only queues the work (gd_dbscan is
        asynchronous): the results are final after sync().  eps2_yes > 0
        selects approximate FastMerging (gd_instance.eps2_yes; a batch of one
        instance)."""
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.int32 and X.dim() == 2):
            raise TypeError("X must be a CUDA int32 tensor of shape [n, d]")
        X = X.contiguous()
        n, d = X.shape
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=X.device)
        if is_core is None:
            is_core = torch.empty(n, dtype=torch.uint8, device=X.device)
        if eps2_yes:
            one = (GdInstance * 1)(GdInstance(X.data_ptr(), n, d, int(eps2), int(minpts), labels.data_ptr(),
                                              is_core.data_ptr(), int(eps2_yes)))
            st = self._lib.gd_dbscan_batched(self._h, 1, ctypes.cast(one, ctypes.c_void_p), _stream_handle(stream))
        else:
            st = self._lib.gd_dbscan(self._h, X.data_ptr(), n, d, int(eps2), int(minpts), labels.data_ptr(),
                                     is_core.data_ptr(), _stream_handle(stream))
        self._check(st)
        if sync:
            self.sync(stream)
        return labels, is_core.view(torch.bool) if is_core.dtype == torch.uint8 else is_core

    def dbscan_batched(self, jobs, outputs=None, stream=None, sync: bool = True):
        """Cluster a batch of instances in one gd_dbscan_batched call.  jobs is a
        list of (X, eps2, minpts) or (X, eps2, minpts, eps2_yes) with X a CUDA
        int32 [n, d] tensor (n >= 1; eps2_yes as gd_instance.eps2_yes);
        returns a list of (labels, is_core) device tensors (or fills `outputs`,
        a list of (labels int32, is_core uint8) tensor pairs)."""
        import torch
        k = len(jobs)
        arr = (GdInstance * max(k, 1))()
        outs = []
        keep = []
        for i, job in enumerate(jobs):
            X, eps2, minpts = job[:3]
            eps2_yes = int(job[3]) if len(job) > 3 else 0
            if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.int32 and X.dim() == 2):
                raise TypeError("each X must be a CUDA int32 tensor of shape [n, d]")
            X = X.contiguous()
            keep.append(X)
            n, d = X.shape
            if outputs is not None:
                lab, core = outputs[i]
            else:
                lab = torch.empty(n, dtype=torch.int32, device=X.device)
                core = torch.empty(n, dtype=torch.uint8, device=X.device)
            outs.append((lab, core))
            arr[i] = GdInstance(X.data_ptr(), n, d, int(eps2), int(minpts), lab.data_ptr(), core.data_ptr(), eps2_yes)
        self._check(self._lib.gd_dbscan_batched(self._h, k, ctypes.cast(arr, ctypes.c_void_p),
                                                _stream_handle(stream)))
        if sync:
            self.sync(stream)
        return [(lab, core.view(torch.bool) if core.dtype == torch.uint8 else core) for lab, core in outs]

    def dbscan_host(self, X, eps2: int, minpts: int, labels=None, is_core=None, stream=None, sync: bool = True):
        """Cluster host points (numpy or CPU torch int32 [n, d]; pinned memory
        is fastest).  Copies in, clusters and copies the results out.  With
        sync=False the work is only queued (gd_dbscan_host_async): X must stay
        unchanged and the outputs are final after sync()."""
        import torch
        if isinstance(X, np.ndarray):
            X = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32))
        if X.is_cuda or X.dtype != torch.int32 or X.dim() != 2:
            raise TypeError("X must be a host int32 array of shape [n, d]")
        X = X.contiguous()
        n, d = X.shape
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32)
        if is_core is None:
            is_core = torch.empty(n, dtype=torch.uint8)
        fn = self._lib.gd_dbscan_host if sync else self._lib.gd_dbscan_host_async
        st = fn(self._h, X.data_ptr(), n, d, int(eps2), int(minpts), labels.data_ptr(), is_core.data_ptr(),
                _stream_handle(stream))
        self._check(st)
        return labels, is_core

    # -- memory
    def bytes_held(self) -> int:
        """Device bytes the context holds for reuse."""
        return int(self._lib.gd_ctx_bytes(self._h))

    def trim(self):
        """Release the context's cached buffers."""
        self._check(self._lib.gd_ctx_trim(self._h))

    # -- introspection
    def last_sizes(self) -> dict:
        out = (ctypes.c_int64 * 13)()
        self._check(self._lib.gd_last_sizes(self._h, out))
        keys = ["n", "d", "grids", "nnbr", "side", "key_bits", "launches", "pairs", "sort_passes", "digit_bits",
                "fastmerging_pairs", "key_class", "queued"]
        return {k: int(v) for k, v in zip(keys, out)}

    def copy_view(self, which: int, dtype, count: int) -> np.ndarray:
        a = np.empty(count, dtype=dtype)
        self._check(self._lib.gd_copy_view(self._h, int(which), a.ctypes.data, a.nbytes))
        return a

    def set_timing(self, enable: bool):
        self._check(self._lib.gd_set_timing(self._h, 1 if enable else 0))

    def set_retry_limit(self, limit: int):
        """Cap the union-find loops' iterations (0: the built-in limit); a
        call whose loops run out raises GdError with GD_ETIMEOUT."""
        self._check(self._lib.gd_set_retry_limit(self._h, int(limit)))

    def inject_alloc_failure(self, k: int):
        """Make the k-th device buffer request from now fail (0: cancel)."""
        self._check(self._lib.gd_inject_alloc_failure(self._h, int(k)))

    def set_stats(self, enable: bool):
        """Keep run statistics (merge outcomes, FastMerging rounds, count
        rows) for each following call; such calls are slower."""
        self._check(self._lib.gd_set_stats(self._h, 1 if enable else 0))

    def run_stats(self) -> dict:
        """The statistics of the last call (empty if it kept none)."""
        vals = (ctypes.c_int64 * 64)()
        names = (ctypes.c_char_p * 64)()
        k = self._lib.gd_run_stats(self._h, vals, names, 64)
        return {names[i].decode(): int(vals[i]) for i in range(k)}

    def stage_times(self) -> dict:
        ms = (ctypes.c_float * 32)()
        names = (ctypes.c_char_p * 32)()
        k = self._lib.gd_stage_times(self._h, ms, names, 32)
        return {names[i].decode(): float(ms[i]) for i in range(k)}


NOALLOC_MAX_POINTS = 65536


def dbscan_noalloc(X, eps2: int, minpts: int, labels=None, is_core=None, stream=None):
    """gd_dbscan_noalloc: cluster a CUDA int32 [n, d] tensor (n at most
    NOALLOC_MAX_POINTS) with the library's fixed static scratch instead of any
    device allocation.  The output tensors are allocated here by torch unless
    given; the library call itself allocates nothing."""
    import torch
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.int32 and X.dim() == 2):
        raise TypeError("X must be a CUDA int32 tensor of shape [n, d]")
    lib = load_library()
    X = X.contiguous()
    n, d = X.shape
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=X.device)
    if is_core is None:
        is_core = torch.empty(n, dtype=torch.uint8, device=X.device)
    with torch.cuda.device(X.device):
        st = lib.gd_dbscan_noalloc(X.data_ptr(), n, d, int(eps2), int(minpts), labels.data_ptr(),
                                   is_core.data_ptr(), _stream_handle(stream))
    if st != GD_OK:
        raise GdError(st, lib.gd_status_str(st).decode())
    return labels, is_core


def distance_peak(d: int, device: int = 0) -> float:
    """gd_distance_peak: squared distances per second the GPU can evaluate
    in d dimensions from registers alone (the ALU ceiling of the distance
    loops)."""
    lib = load_library()
    v = ctypes.c_double()
    st = lib.gd_distance_peak(int(device), int(d), ctypes.byref(v))
    if st != GD_OK:
        raise GdError(st, lib.gd_status_str(st).decode())
    return float(v.value)


def workspace_bytes(n: int, d: int) -> int:
    return int(load_library().gd_workspace_bytes(int(n), int(d)))


_default: dict[int, Context] = {}


def dbscan(X, eps2: int, minpts: int, stream=None):
    """Exact DBSCAN of a CUDA int32 [n, d] tensor with a per-device default
    context.  Returns (labels, is_core) device tensors."""
    dev = X.device.index if X.device.index is not None else 0
    ctx = _default.get(dev)
    if ctx is None:
        ctx = _default[dev] = Context(dev)
    return ctx.dbscan(X, eps2, minpts, stream=stream)
