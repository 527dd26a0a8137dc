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


# --------------------------------------------------------------------------- TN / L-BFGS
def _schroedinger_case(n=10):
    """vW + local PP only: E[psi^2] = dV psi^T (K/2 + diag v) psi with K the spectral
    -Laplacian, a quadratic form.  Under int psi^2 = N_e its minimum is N_e times the
    lowest eigenvalue of H = K/2 + diag v (the one-orbital Schroedinger ground state,
    Sec. 2.4's psi = sqrt(rho) picture), found here by dense diagonalisation."""
    cell, pos = W.fcc_positions(1)
    g = Grid(cell, (n, n, n))
    Vg = fn.external_potential_G(g, pos, np.zeros(4, int), [3.0], [0.9])
    v = g.ifft(Vg).reshape(-1)
    N = g.N
    K = np.empty((N, N))
    e = np.zeros(N)
    for j in range(N):               # columns of the spectral -Laplacian (cubic cell: symmetric)
        e[j] = 1.0
        K[:, j] = g.ifft(g.G2 * g.fft(e.reshape(g.shape))).reshape(-1)
        e[j] = 0.0
    H = 0.5 * K + np.diag(v)
    return g, Vg, H


def test_dense_hamiltonian_is_symmetric_with_a_nodeless_ground_state():
    g, _, H = _schroedinger_case(8)
    assert np.max(np.abs(H - H.T)) < 1e-10 * np.max(np.abs(H))
    w, U = np.linalg.eigh(H)
    u0 = U[:, 0] * np.sign(U[0, 0])
    assert np.all(u0 > 0.0)          # ground state of a local Hamiltonian has no node
    assert w[1] - w[0] > 1e-3        # and is non-degenerate here


def test_hessian_vector_equals_dense_lagrangian_hessian():
    """For the quadratic vW + PP functional the Lagrangian Hessian is exactly
    2 dV (H - mu); the finite-difference product must reproduce it."""
    from oracle.optimize import hessian_vector
    g, Vg, H = _schroedinger_case(8)
    rng = np.random.default_rng(3)
    psi = 1.0 + 0.2 * rng.random(g.shape)
    x = rng.standard_normal(g.shape)
    f = Functional(terms=("VW", "PP"))
    mu = 0.37
    Hx, _ = hessian_vector(g, psi, x, f, Vg, mu)
    ref = 2.0 * g.dV * (H @ x.reshape(-1) - mu * x.reshape(-1))
    assert np.max(np.abs(Hx.reshape(-1) - ref)) < 1e-7 * np.max(np.abs(ref))


def test_hessian_vector_matches_second_differences_of_the_energy():
    """TF + vW + Hartree + PP (nonlinear in psi): x.Hx from differences of the gradient
    equals d^2/dt^2 of the Lagrangian E[(psi + t x)^2] - mu int (psi + t x)^2 from
    differences of the ENERGY alone, and the product is symmetric (y.Hx = x.Hy).
    (The LWT term is left out: its linear spline in k_F has kinks wherever k_F crosses
    a knot, so its second derivative along a line is not a smooth function of t.)"""
    from oracle.optimize import hessian_vector
    g, rho, Vg = _small_al()
    f = Functional(terms=("TF", "VW", "HARTREE", "PP"))
    psi = np.sqrt(rho)
    rng = np.random.default_rng(11)
    x = psi * rng.standard_normal(g.shape) * 0.3
    y = psi * rng.standard_normal(g.shape) * 0.3
    mu = 0.21
    Hx, _ = hessian_vector(g, psi, x, f, Vg, mu)
    Hy, _ = hessian_vector(g, psi, y, f, Vg, mu)
    h = 1e-3

    def L(t):
        q = psi + t * x
        return evaluate(g, q * q, f, Vg)[0]["total"] - mu * np.sum(q * q) * g.dV

    d2 = (-L(2 * h) + 16 * L(h) - 30 * L(0.0) + 16 * L(-h) - L(-2 * h)) / (12 * h * h)
    xHx = float(np.sum(x * Hx))
    assert abs(xHx - d2) < 1e-7 * abs(d2)
    assert abs(float(np.sum(y * Hx)) - float(np.sum(x * Hy))) < 1e-6 * abs(xHx)


def test_every_method_reaches_the_schroedinger_ground_state():
    g, Vg, H = _schroedinger_case(10)
    E0 = 4.0 * np.linalg.eigvalsh(H)[0]
    rng = np.random.default_rng(2)
    psi0 = 1.0 + 0.3 * rng.random(g.shape)
    f = Functional(terms=("VW", "PP"))
    for method in ("cg", "tn", "lbfgs"):
        res = optimize_density(g, psi0, f, Vg, 4.0, 4, tol=1e-13, max_iter=500, method=method)
        assert abs(res["E"] - E0) < 1e-9 * abs(E0), (method, res["E"], E0, res["iterations"])


def _residual(g, psi, f, Vg, ne):
    E, V = evaluate(g, psi * psi, f, Vg)
    mu = np.sum(psi * psi * V) * g.dV / ne
    return math.sqrt(np.sum(((V - mu) * psi) ** 2) * g.dV)


def test_tn_and_lbfgs_reach_the_cg_minimum_in_fewer_iterations():
    """TF + vW + Hartree + PP: a convex problem in rho, one minimum for all three
    methods; Newton-CG's curvature information shows as far fewer outer iterations."""
    g, rho, Vg = _small_al()
    f = Functional(terms=("TF", "VW", "HARTREE", "PP"))
    out = {m: optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400, method=m)
           for m in ("cg", "tn", "lbfgs")}
    for m in ("tn", "lbfgs"):
        assert abs(out[m]["E"] - out["cg"]["E"]) / 4 < 1e-10, (m, out[m]["E"], out["cg"]["E"])
        assert _residual(g, out[m]["psi"], f, Vg, 12.0) < 1e-4
    assert out["tn"]["iterations"] < out["cg"]["iterations"] / 2
    assert out["lbfgs"]["iterations"] <= out["cg"]["iterations"]


def test_methods_end_at_stationary_points_of_the_lwt_functional():
    """With the LWT term (knots frozen) the functional is not convex: its linear spline
    in k_F has kinks, and on this small noisy cell CG and TN settle in two different
    local minima 3e-5 Ha apart, each stable when the other method is restarted from
    it.  What holds for every method: a stationary point (small Euler-Lagrange
    residual), at an energy far below the start and within 1e-5 Ha/atom of the others."""
    g, rho, Vg = _small_al()
    f = Functional(n_knots=6, knots=fn.make_knots(rho, 6))
    E0 = evaluate(g, rho, f, Vg)[0]["total"]
    Es = []
    for m in ("cg", "tn", "lbfgs"):
        r = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400, method=m)
        assert _residual(g, r["psi"], f, Vg, 12.0) < 3e-5, m
        assert abs(np.sum(r["psi"] ** 2) * g.dV - 12.0) < 1e-10
        Es.append(r["E"])
    assert max(Es) < E0 - 1e-2
    assert (max(Es) - min(Es)) / 4 < 1e-5


# --------------------------------------------------------------------------- scaling update
def test_scaling_update_stays_normalised_and_its_derivative_is_exact():
    from oracle.optimize import update_curve
    g, rho, _ = _small_al()
    psi = np.sqrt(rho)
    d = np.random.default_rng(4).standard_normal(g.shape) * psi      # not orthogonal to psi
    p = d * math.sqrt(12.0 / (np.sum(d * d) * g.dV))
    for t in (0.0, 0.2, 0.9):
        q, dq = update_curve(psi, p, t, g.dV, 12.0, "scale")
        assert abs(np.sum(q * q) * g.dV - 12.0) < 1e-11
        h = 1e-5
        fd = (update_curve(psi, p, t + h, g.dV, 12.0, "scale")[0]
              - update_curve(psi, p, t - h, g.dV, 12.0, "scale")[0]) / (2 * h)
        assert np.max(np.abs(fd - dq)) < 1e-7 * np.max(np.abs(dq))
        # the renormalised point is psi + t p scaled: parallel to it
        r = psi + t * p
        assert np.max(np.abs(q * (np.sum(r * r) / np.sum(q * r)) - r)) < 1e-12 * np.max(np.abs(r))


def test_scaling_with_orthogonal_p_is_the_rotation_at_atan_t():
    from oracle.optimize import update_curve
    g, rho, _ = _small_al()
    psi = np.sqrt(rho)
    d = np.random.default_rng(9).standard_normal(g.shape) * psi
    p = d - np.sum(d * psi) / np.sum(psi * psi) * psi
    p *= math.sqrt(12.0 / (np.sum(p * p) * g.dV))
    for t in (0.1, 0.7, 2.0):
        a = update_curve(psi, p, t, g.dV, 12.0, "scale")[0]
        b = update_curve(psi, p, math.atan(t), g.dV, 12.0, "rotate")[0]
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_scaling_update_reaches_the_same_minima():
    g, Vg, H = _schroedinger_case(10)
    E0 = 4.0 * np.linalg.eigvalsh(H)[0]
    psi0 = 1.0 + 0.3 * np.random.default_rng(2).random(g.shape)
    for method in ("cg", "tn"):
        r = optimize_density(g, psi0, Functional(terms=("VW", "PP")), Vg, 4.0, 4, tol=1e-13, max_iter=500,
                             method=method, update="scale")
        assert abs(r["E"] - E0) < 1e-9 * abs(E0), (method, r["E"], E0)
    g, rho, Vg = _small_al()
    f = Functional(terms=("TF", "VW", "HARTREE", "PP"))
    a = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400)
    b = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400, update="scale")
    assert abs(a["E"] - b["E"]) / 4 < 1e-10


# --------------------------------------------------------------------------- residual minimisation
def test_residual_minimisation_reaches_the_same_minima():
    """Sec. 2.4's second way (the step lowers the norm of Eq. euler2's residual): the
    Schroedinger ground state and the convex minimum, with CG and TN directions."""
    g, Vg, H = _schroedinger_case(10)
    E0 = 4.0 * np.linalg.eigvalsh(H)[0]
    psi0 = 1.0 + 0.3 * np.random.default_rng(2).random(g.shape)
    for method in ("cg", "tn"):
        r = optimize_density(g, psi0, Functional(terms=("VW", "PP")), Vg, 4.0, 4, tol=1e-13, max_iter=800,
                             method=method, objective="residual")
        assert abs(r["E"] - E0) < 1e-9 * abs(E0), (method, r["E"], E0, r["iterations"])
    g, rho, Vg = _small_al()
    f = Functional(terms=("TF", "VW", "HARTREE", "PP"))
    a = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400)
    b = optimize_density(g, np.sqrt(rho), f, Vg, 12.0, 4, tol=1e-11, max_iter=400, method="tn",
                         objective="residual")
    assert abs(a["E"] - b["E"]) / 4 < 1e-10
    assert _residual(g, b["psi"], f, Vg, 12.0) < 1e-5


def test_residual_minimisation_lowers_the_residual_every_step():
    g, rho, Vg = _small_al()
    f = Functional(terms=("TF", "VW", "HARTREE", "PP"))
    psi = np.sqrt(rho)
    res = [_residual(g, psi, f, Vg, 12.0)]
    for _ in range(6):
        r = optimize_density(g, psi, f, Vg, 12.0, 4, max_iter=1, fixed_iter=1, method="tn", objective="residual")
        psi = r["psi"]
        res.append(_residual(g, psi, f, Vg, 12.0))
    assert all(b < a for a, b in zip(res, res[1:])), res
    assert res[-1] < 1e-2 * res[0]
