"""The paper's printed parameters (tests/golden/paper_parameters.txt) against the values the
oracle, the workloads and the Python binding use.  Loads the binding module only (no GPU)."""
import math
import os

import pytest

import workloads as W
from oracle.lindhard import C_WT

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")
BOHR_ANGSTROM = 0.529177210903        # CODATA 2018


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = eval(v, {"pi": math.pi})     # arithmetic of the printed formulas only
    return out


def test_wang_teter_constant():
    assert abs(C_WT - _golden()["C_WT"]) < 1e-15 * C_WT


def test_fermi_wavevector_convention():
    from oracle.functionals import fermi_wavevector
    g = _golden()["kF_per_rho_cubed"]
    for rho in (1e-3, 0.02, 0.3):
        assert abs(float(fermi_wavevector(rho)) - (g * rho) ** (1 / 3)) < 1e-14


def test_mgp_presets_of_the_binding():
    pytest.importorskip("torch")
    import paper_2002_02985_gb300 as ofd
    g = _golden()
    for name in ("MGP", "MGPA", "MGPG"):
        x, y = g[name]
        assert getattr(ofd, name) == dict(mgp_x=x, mgp_y=y)


def test_aluminium_lattice_constant():
    """The workloads' conventional fcc cell edge, 7.65 bohr, is the paper's 4.05 Angstrom rounded
    to three significant figures in bohr."""
    a = _golden()["al_lattice_constant_angstrom"] / BOHR_ANGSTROM
    assert abs(W.A_AL / a - 1.0) < 1e-3
