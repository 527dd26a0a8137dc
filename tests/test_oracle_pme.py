"""Pins of the oracle's smooth-PME structure factor (Sec. 2.5; Essmann et al. 1995)
against the definition S(G) = sum_I exp(-iG.R_I), partition of unity, and finite
differences of the PME energy (its forces)."""
import numpy as np
import pytest

import workloads as W
from oracle import functionals as fn, pme
from oracle.forces import forces as direct_forces
from oracle.grid import Grid


def setup():
    wl = W.workload("fcc-al-4/32")
    rho = W.model_density(wl)
    cell = np.array([[7.65, 0.0, 0.0], [0.4, 7.3, 0.0], [-0.2, 0.5, 7.9]])      # non-orthogonal
    g = Grid(cell, (32, 30, 36))
    pos = np.random.default_rng(0).uniform(0, 1, (5, 3)) @ cell
    rho = W.renormalise(W.gaussian_density(cell, g.shape, pos, 3.0, 1.0), cell, 15.0)
    return g, pos, rho


def test_bspline_partition_of_unity_and_support():
    x = np.linspace(0, 1, 17)
    for p in (4, 8, 12):
        tot = sum(pme.bspline(p, x + j) for j in range(p))
        assert np.allclose(tot, 1.0, atol=1e-14)
        assert np.all(pme.bspline(p, np.array([-0.1, p + 0.1])) == 0.0)
    g, pos, _ = setup()
    assert abs(pme.charge_grid(g, pos, 8).sum() - len(pos)) < 1e-12


@pytest.mark.parametrize("p,tol_e", [(8, 1e-7), (12, 1e-10)])
def test_pme_converges_to_direct_structure_factor(p, tol_e):
    g, pos, rho = setup()
    sp = [0] * len(pos)
    Ed = fn.local_pseudopotential(g, rho, fn.external_potential_G(g, pos, sp, [3.0], [0.8]))[0]
    Ep = fn.local_pseudopotential(g, rho, pme.external_potential_G(g, pos, sp, [3.0], [0.8], p))[0]
    assert abs(Ep - Ed) <= tol_e * abs(Ed)
    Fd = direct_forces(g, rho, pos, sp, [3.0], [0.8])
    Fp = pme.forces(g, rho, pos, sp, [3.0], [0.8], p)
    assert np.max(np.abs(Fp - Fd)) <= 100 * tol_e * max(1.0, np.max(np.abs(Fd)))


def test_pme_forces_are_the_derivative_of_the_pme_energy():
    g, pos, rho = setup()
    sp = [0] * len(pos)
    p, h = 6, 1e-5            # low order: PME differs from the direct S, FD must follow PME
    F = pme.forces(g, rho, pos, sp, [3.0], [0.8], p)
    for I, a in [(0, 0), (3, 2), (4, 1)]:
        Es = []
        for sgn in (1, -1):
            q = pos.copy()
            q[I, a] += sgn * h
            Es.append(fn.local_pseudopotential(g, rho, pme.external_potential_G(g, q, sp, [3.0], [0.8], p))[0])
        assert abs(-(Es[0] - Es[1]) / (2 * h) - F[I, a]) <= 1e-8 * max(1.0, abs(F[I, a]))
