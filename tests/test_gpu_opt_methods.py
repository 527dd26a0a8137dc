"""GPU tests of the optimiser's truncated-Newton and L-BFGS directions (Sec. 2.4, step 1).

The trajectories are parity unpinned (the inner solves, line search and finite-difference
Hessian products are readings); the end points are checked:
- vW + local PP is a quadratic form in psi, so its constrained minimum is N_e times the
  lowest eigenvalue of -lap/2 + v_ext on the grid (Lanczos on the spectral operator);
- TF + vW + Hartree + PP (convex in rho): the oracle's minimum;
- the full LWT functional with frozen knots: the oracle's CG minimum (the spline's kinks
  make this functional non-convex; nearby stationary points differ by < 1e-7 Ha/atom).
"""
import ctypes as ct
import math

import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn
from oracle.evaluate import Functional as OFunc
from oracle.grid import Grid as OGrid
from oracle.optimize import optimize_density as ooptimize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402

WL = "fcc-al-4/32"
METHODS = ("cg", "tn", "lbfgs")


@pytest.fixture(scope="module")
def case():
    wl = W.workload(WL)
    rho = W.model_density(wl)
    og = OGrid(wl["cell"], wl["shape"])
    Vg = ofn.external_potential_G(og, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    return wl, rho, og, Vg


def _grid(wl):
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
    return g


def _run(wl, rho, func, method, tol, max_iter=400, update="rotate", objective="energy"):
    g = _grid(wl)
    dt = torch.float64 if func.precision == L.FP64 else torch.float32
    psi = torch.from_numpy(np.sqrt(rho)).to("cuda", dt).contiguous()
    rep = g.optimize_density(psi, func, wl["n_electrons"], tol_per_atom=tol, max_iter=max_iter, method=method,
                             update=update, objective=objective)
    charge = float((psi.double() ** 2).sum()) * g.dV
    assert abs(charge - wl["n_electrons"]) <= (1e-10 if func.precision == L.FP64 else 1e-6) * wl["n_electrons"]
    return rep


@pytest.fixture(scope="module")
def ground_state(case):
    """N_e * lowest eigenvalue of H = -lap/2 + v_ext (spectral Laplacian; cubic cell)."""
    import scipy.sparse.linalg as sla
    wl, _, og, Vg = case
    v = og.ifft(Vg)

    def mv(x):
        x = x.reshape(og.shape)
        return (0.5 * og.ifft(og.G2 * og.fft(x)) + v * x).reshape(-1)

    w = sla.eigsh(sla.LinearOperator((og.N, og.N), matvec=mv, dtype=np.float64), k=1, which="SA", tol=1e-14)[0]
    return wl["n_electrons"] * float(w[0])


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("precision", [L.FP64, L.FP32_MIXED])
def test_methods_reach_the_schroedinger_ground_state(case, ground_state, method, precision):
    wl, rho, _, _ = case
    f = ofd.Functional(terms=L.TERM_VW | L.TERM_PP, precision=precision)
    rep = _run(wl, rho, f, method, 1e-13 if precision == L.FP64 else 1e-8)
    err = abs(rep["energy"] - ground_state)
    if precision == L.FP64:
        assert err <= 1e-9 * abs(ground_state), (method, rep)
    else:
        assert err / wl["n_atoms"] <= 1e-6, (method, rep)


@pytest.fixture(scope="module")
def convex_minimum(case):
    wl, rho, og, Vg = case
    r = ooptimize(og, np.sqrt(rho), OFunc(terms=("TF", "VW", "HARTREE", "PP")), Vg, wl["n_electrons"],
                  wl["n_atoms"], tol=1e-12, max_iter=400, method="tn")
    return r["E"]


@pytest.mark.parametrize("method", ("tn", "lbfgs"))
@pytest.mark.parametrize("precision,tol", [(L.FP64, 1e-9), (L.FP32_MIXED, 1e-6)])
def test_tn_and_lbfgs_reach_the_oracle_minimum_convex(case, convex_minimum, method, precision, tol):
    wl, rho, _, _ = case
    f = ofd.Functional(terms=L.TERM_TF | L.TERM_VW | L.TERM_HARTREE | L.TERM_PP, precision=precision)
    rep = _run(wl, rho, f, method, 1e-12 if precision == L.FP64 else 1e-8)
    assert abs(rep["energy"] - convex_minimum) / wl["n_atoms"] <= tol, (method, rep, convex_minimum)


@pytest.fixture(scope="module")
def lwt_minimum(case):
    wl, rho, og, Vg = case
    knots = ofn.make_knots(rho, wl["n_knots"])
    r = ooptimize(og, np.sqrt(rho), OFunc(n_knots=wl["n_knots"], knots=knots), Vg, wl["n_electrons"],
                  wl["n_atoms"], tol=1e-12, max_iter=400)
    return knots, r["E"]


@pytest.mark.parametrize("method", ("tn", "lbfgs"))
@pytest.mark.parametrize("precision", [L.FP64, L.FP32_MIXED])
def test_tn_and_lbfgs_on_the_lwt_functional(case, lwt_minimum, method, precision):
    wl, rho, _, _ = case
    knots, E_or = lwt_minimum
    f = ofd.Functional(n_knots=wl["n_knots"], knots=knots, precision=precision)
    rep = _run(wl, rho, f, method, 1e-12 if precision == L.FP64 else 1e-7)
    assert abs(rep["energy"] - E_or) / wl["n_atoms"] <= 1e-6, (method, rep, E_or)
    assert rep["residual"] < (1e-4 if precision == L.FP64 else 1e-2)


@pytest.mark.parametrize("method", ("cg", "tn"))
def test_scaling_update_reaches_the_same_minima(case, ground_state, convex_minimum, method):
    """Sec. 2.4's scaling scheme (psi + t p renormalised, p not orthogonalised)."""
    wl, rho, _, _ = case
    f = ofd.Functional(terms=L.TERM_VW | L.TERM_PP, precision=L.FP64)
    rep = _run(wl, rho, f, method, 1e-13, update="scale")
    assert abs(rep["energy"] - ground_state) <= 1e-9 * abs(ground_state), (method, rep)
    f = ofd.Functional(terms=L.TERM_TF | L.TERM_VW | L.TERM_HARTREE | L.TERM_PP, precision=L.FP32_MIXED)
    rep = _run(wl, rho, f, method, 1e-8, update="scale")
    assert abs(rep["energy"] - convex_minimum) / wl["n_atoms"] <= 1e-6, (method, rep, convex_minimum)


@pytest.mark.parametrize("method", ("cg", "tn"))
def test_residual_minimisation_reaches_the_same_minima(case, ground_state, convex_minimum, method):
    """Sec. 2.4's second way: each step lowers the norm of the residual of Eq. euler2."""
    wl, rho, _, _ = case
    f = ofd.Functional(terms=L.TERM_VW | L.TERM_PP, precision=L.FP64)
    rep = _run(wl, rho, f, method, 1e-13, max_iter=800, objective="residual")
    assert abs(rep["energy"] - ground_state) <= 1e-9 * abs(ground_state), (method, rep)
    f = ofd.Functional(terms=L.TERM_TF | L.TERM_VW | L.TERM_HARTREE | L.TERM_PP, precision=L.FP32_MIXED)
    rep = _run(wl, rho, f, method, 1e-8, max_iter=800, objective="residual")
    assert abs(rep["energy"] - convex_minimum) / wl["n_atoms"] <= 1e-6, (method, rep, convex_minimum)


def test_tn_needs_fewer_outer_iterations_than_cg(case):
    wl, rho, _, _ = case
    f = ofd.Functional(terms=L.TERM_TF | L.TERM_VW | L.TERM_HARTREE | L.TERM_PP, precision=L.FP64)
    cg = _run(wl, rho, f, "cg", 1e-12)
    tn = _run(wl, rho, f, "tn", 1e-12)
    assert tn["iterations"] < cg["iterations"], (tn, cg)


def test_optimiser_options_out_of_range_are_rejected(case):
    wl, rho, _, _ = case
    g = _grid(wl)
    psi = torch.from_numpy(np.sqrt(rho)).to("cuda", torch.float32).contiguous()
    c, keep = ofd.Functional().to_c()
    rep = L.COptReport()
    for bad in (L.COptOptions(7, 1, 0, 0, 0), L.COptOptions(L.OPT_TN, 1, 101, 0, 0), L.COptOptions(L.OPT_LBFGS, 1, 0, 33, 0),
                L.COptOptions(L.OPT_TN, 1, -1, 0, 0), L.COptOptions(L.OPT_CG, 1, 0, 0, 2),
                L.COptOptions(L.OPT_CG, 1, 0, 0, 0, 2)):
        st = g.lib.ofdft_optimize_density_ex(g.h, ct.c_void_p(psi.data_ptr()), ct.byref(c), wl["n_electrons"], 1e-6,
                                             10, ct.byref(bad), ct.byref(rep))
        assert st == L.OFDFT_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        g.optimize_density(psi, ofd.Functional(), wl["n_electrons"], method="newton")
    with pytest.raises(ValueError):
        g.optimize_density(psi, ofd.Functional(), wl["n_electrons"], update="shift")
    with pytest.raises(ValueError):
        g.optimize_density(psi, ofd.Functional(), wl["n_electrons"], objective="force")
    del keep
