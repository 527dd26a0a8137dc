"""The polynomial forms of G_NL compiled into the FP32-mixed kernels (csrc/gnl_fit.cuh,
written by gen_gnl_fit.py) against the oracle's G_NL (Sec. 2.3, the G_NL definition below
Eq. MGP): the coefficients as the compiler rounds them (FP32), evaluated in FP64, stay
within 1e-7 of G_NL below eta = 1/2 and above eta = 2, the ranges where the kernels use them."""
import os
import re

import numpy as np
import pytest

from oracle.lindhard import G_NL

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2002_02985_gb300", "csrc",
                   "gnl_fit.cuh")


def _coefficients(name):
    src = open(HDR).read()
    body = re.search(name + r"\(float \w\) \{\s*return (.*?);\s*\}", src, re.S).group(1)
    lits = [np.float32(float(v.rstrip("f"))) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+f", body)]
    # the innermost literal is the highest coefficient; then one constant per fmaf, inside out
    return [float(c) for c in reversed(lits)]             # constant term first


def _horner(c, v):
    p = np.zeros_like(v)
    for ck in reversed(c):
        p = p * v + ck
    return p


def test_small_eta_polynomial_matches_g_nl():
    c = _coefficients("gnl_small_s")
    eta = np.linspace(1e-4, 0.5, 20001)
    y = eta * eta
    got = y * _horner(c, y)
    ref = G_NL(eta)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-7
    assert abs(c[0] + 8.0 / 3.0) < 1e-6                 # G_NL = -(8/3) eta^2 + O(eta^4)


def test_large_eta_polynomial_matches_g_nl():
    c = _coefficients("gnl_large_l")
    eta = np.concatenate([np.linspace(2.0, 50.0, 20001), np.geomspace(50.0, 1e6, 2001)])
    got = _horner(c, 1.0 / (eta * eta))
    ref = G_NL(eta)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-7
    assert abs(c[0] + 1.6) < 1e-6                       # G_NL(inf) = -8/5


def test_generator_reproduces_the_compiled_header(tmp_path, monkeypatch):
    """gen_gnl_fit.py (50-digit Chebyshev interpolation) writes exactly the committed header."""
    pytest.importorskip("mpmath")
    import importlib.util
    gen = os.path.join(os.path.dirname(HDR), "..", "gen_gnl_fit.py")
    spec = importlib.util.spec_from_file_location("gen_gnl_fit", gen)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = tmp_path / "gnl_fit.cuh"
    monkeypatch.setattr(mod, "OUT", str(out))
    mod.main()
    assert out.read_text() == open(HDR).read()
