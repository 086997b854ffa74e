"""Exact Euclidean DBSCAN on one GB300 (GriT-DBSCAN, arXiv 2210.07580).

The clustering runs in libgdbscan.so (hand-written CUDA for sm_103a behind the
C ABI of include/gdbscan.h); ``binding`` marshals arguments to it.  Importing
this package does not load the library; the first call does, and raises if
the library has not been built.
"""
from .binding import (Context, GdError, GdInstance, dbscan, eps2_from_eps, load_library,  # noqa: F401
                      workspace_bytes)
