"""The C ABI library builds for sm_103a, loads, and exports every entry point of
include/ofdft.h; the product path fails loudly without it (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "ofdft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ofdft_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2002_02985_gb300 import build as b
    return b.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ofdft_grid_create", "ofdft_energy_potential", "ofdft_forces", "ofdft_optimize_density"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2002_02985_gb300 import _lib as L
    assert sorted(L.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.ofdft_status_string.restype = ctypes.c_char_p
    lib.ofdft_version.restype = ctypes.c_char_p
    assert lib.ofdft_status_string(0) == b"ok"
    assert b"2^a 3^b 5^c" in lib.ofdft_status_string(-2)
    assert b"sm_103a" in lib.ofdft_version()


def test_missing_library_raises():
    from paper_2002_02985_gb300 import _lib as L
    saved = L._lib
    L._lib = None
    try:
        with pytest.raises(OSError):
            L.load("/nonexistent/libofdft.so")
    finally:
        L._lib = saved
