"""Pins of the oracle's psi = sqrt(rho) optimiser (Sec. 2.4, Eq. euler2).

The trajectory is parity unpinned (the line search is a reading); what the
method fixes is checked: charge conservation of the cos/sin update, monotone
energy decrease, and the Euler-Lagrange residual (V - mu) psi at convergence.
"""
import math

import numpy as np

import workloads as W
from oracle import functionals as fn
from oracle.evaluate import Functional, evaluate
from oracle.grid import Grid
from oracle.optimize import optimize_density


def _small_al():
    cell, pos = W.fcc_positions(1)
    g = Grid(cell, (16, 16, 16))
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, g.shape, pos, 3.0, 1.0), 0.05, 7), cell, 12.0)
    Vg = fn.external_potential_G(g, pos, np.zeros(4, int), [3.0], [0.8])
    return g, rho, Vg


def test_optimizer_conserves_charge_and_decreases_energy():
    """With frozen knots E[psi^2] is one fixed functional: the CG must descend monotonically.
    (With knots recomputed every iteration the functional itself moves between iterations.)"""
    g, rho, Vg = _small_al()
    f = Functional(n_knots=6, knots=fn.make_knots(rho, 6))
    res = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-9, max_iter=60)
    psi = res["psi"]
    assert abs(np.sum(psi * psi) * g.dV - 12.0) < 1e-11
    h = np.array(res["history"])
    assert np.all(np.diff(h) <= 1e-12)
    assert h[-1] < h[0] - 1e-3
    # Euler-Lagrange residual: V - mu small where the density lives
    E, V = evaluate(g, psi * psi, f, Vg)
    mu = np.sum(psi * psi * V) * g.dV / 12.0
    resid = math.sqrt(np.sum(((V - mu) * psi) ** 2) * g.dV)
    resid0 = math.sqrt(np.sum(((evaluate(g, rho, f, Vg)[1] - mu) * np.sqrt(rho)) ** 2) * g.dV)
    assert resid < 1e-2 * resid0


def test_orthogonal_update_is_exactly_norm_preserving():
    g, rho, _ = _small_al()
    psi = np.sqrt(rho)
    p = np.random.default_rng(5).standard_normal(g.shape)
    p -= np.sum(p * psi) / np.sum(psi * psi) * psi
    p *= math.sqrt(12.0 / (np.sum(p * p) * g.dV))
    for lam in (0.01, 0.3, 1.2):
        q = psi * math.cos(lam) + p * math.sin(lam)
        assert abs(np.sum(q * q) * g.dV - 12.0) < 1e-11


def test_multistep_reaches_the_single_level_minimum():
    """Coarse (16^3) then fine (32^3): the fine level ends at the minimum a direct fine
    optimisation reaches (knots frozen, so both minimise the same functional)."""
    from oracle.optimize import optimize_multistep
    wl = W.workload("fcc-al-4/32")
    rho = W.model_density(wl)
    gf, gc = Grid(wl["cell"], wl["shape"]), Grid(wl["cell"], (16, 16, 16))
    Vf = fn.external_potential_G(gf, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    Vc = fn.external_potential_G(gc, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    f = Functional(n_knots=wl["n_knots"], knots=fn.make_knots(rho, wl["n_knots"]))
    direct = optimize_density(gf, np.sqrt(rho), f, Vf, wl["n_electrons"], wl["n_atoms"], tol=1e-10, max_iter=400)
    multi = optimize_multistep([gc, gf], np.sqrt(rho), f, [Vc, Vf], wl["n_electrons"], wl["n_atoms"],
                               tol=1e-10, max_iter=400)
    assert abs(multi["E"] - direct["E"]) / wl["n_atoms"] < 1e-8
    assert multi["levels"][1] < direct["iterations"]
