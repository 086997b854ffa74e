"""The C ABI library builds, loads without a GPU and exports every function
include/gdbscan.h declares; host-side helpers of the binding."""
import ctypes
import os
import re
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gdbscan.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gd_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_07580_gb300 import _build, binding
    path = _build.build()
    return binding.load_library(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["gd_create", "gd_destroy", "gd_workspace_bytes", "gd_dbscan", "gd_dbscan_host",
                 "gd_status_str", "gd_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in gdbscan.h but not exported"


def test_status_strings_and_workspace(lib):
    for s in range(7):
        assert lib.gd_status_str(s)
    w1 = lib.gd_workspace_bytes(1000, 3)
    w2 = lib.gd_workspace_bytes(1_000_000, 3)
    w3 = lib.gd_workspace_bytes(1_000_000, 7)
    assert 0 < w1 < w2 < w3
    # linear in n with a fixed overhead of about a megabyte
    assert w1 < 4 << 20 and w2 < 1_000_000 * 512 and w3 < 1_000_000 * 512
    assert lib.gd_workspace_bytes(10, 9) == 0 and lib.gd_workspace_bytes(-1, 3) == 0


def test_null_context_is_rejected(lib):
    assert lib.gd_dbscan(None, None, 0, 3, 1, 1, None, None, None) == 1  # GD_EINVAL
    assert lib.gd_last_sizes(None, None) == 1


def test_eps2_from_eps_is_exact():
    from paper_2210_07580_gb300 import eps2_from_eps
    assert eps2_from_eps(800) == 640000
    assert eps2_from_eps(Fraction(3, 2)) == 2
    assert eps2_from_eps("2.5") == 6
    # sqrt(2) as a float is slightly above sqrt(2): its square floors to 2
    assert eps2_from_eps(2 ** 0.5) == 2
    x = 12345.678
    f = Fraction(x)
    assert eps2_from_eps(x) == (f * f).numerator // (f * f).denominator
    with pytest.raises(ValueError):
        eps2_from_eps(-1)
