"""The C-ABI library loads without a GPU and exports every function its
header declares; calls that need no device reject bad arguments."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "beor.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(beor_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_12928_gb300 import _build
    if not os.path.exists(_build.LIB):
        if shutil.which("nvcc") is None:
            pytest.skip("library not built and nvcc not available")
        _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("beor_create", "beor_precompute", "beor_lnl", "beor_lnl_multi", "beor_posterior_mean",
                 "beor_set_lookahead", "beor_dbar_factored_noalloc", "beor_mlp_train_step", "beor_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_argument_checks_without_a_device(lib):
    lib.beor_strerror.restype = ctypes.c_char_p
    lib.beor_strerror.argtypes = [ctypes.c_int]
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.beor_strerror(code)
    # null context / output pointers are rejected before any device work
    lib.beor_lnl.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3
    assert lib.beor_lnl(None, None, 1, None, None, None) == -1
    lib.beor_get_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.beor_get_stats(None, None) == -1
    lib.beor_set_lookahead.argtypes = [ctypes.c_int]
    assert lib.beor_set_lookahead(1) == 0
