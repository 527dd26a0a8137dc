"""Pins of the oracle's LDA exchange-correlation (Dirac exchange, Perdew-Zunger
correlation; the xc of the paper's benchmarks, Sec. 3.1) against facts that do
not come from its own formulas."""
import numpy as np
import pytest

from oracle import xc
from oracle.grid import Grid


def _uniform(rho0, n=6, L=7.0):
    g = Grid(np.diag([L, L, L]), (n, n, n))
    return g, np.full(g.shape, rho0)


@pytest.mark.parametrize("rs", [0.5, 1.0, 2.0, 4.0])
def test_uniform_gas_exchange_is_minus_three_kf_over_four_pi(rs):
    """Exchange energy per electron of the uniform gas, -3 k_F / (4 pi) with
    k_F = (9 pi / 4)^(1/3) / r_s (the textbook form through the Fermi wavevector)."""
    rho0 = 3.0 / (4.0 * np.pi * rs ** 3)
    g, rho = _uniform(rho0)
    Ex = np.sum(rho * xc.eps_x(rho)) * g.dV
    kf = (9.0 * np.pi / 4.0) ** (1.0 / 3.0) / rs
    assert abs(Ex / (rho0 * g.omega) - (-3.0 * kf / (4.0 * np.pi))) <= 1e-13 * kf


def test_exchange_scales_linearly_under_uniform_compression():
    """E_x[lambda^3 rho(lambda r)] = lambda E_x[rho]: the density values scale by
    lambda^3 and the cell by 1/lambda (exact coordinate scaling of exchange)."""
    rng = np.random.default_rng(2)
    cell = np.array([[6.0, 0.0, 0.0], [0.9, 5.5, 0.0], [-0.4, 0.3, 6.3]])
    rho = 0.01 + 0.05 * rng.random((8, 9, 10))
    g = Grid(cell, rho.shape)
    lam = 1.7
    g2 = Grid(cell / lam, rho.shape)
    E1 = np.sum(rho * xc.eps_x(rho)) * g.dV
    E2 = np.sum(lam ** 3 * rho * xc.eps_x(lam ** 3 * rho)) * g2.dV
    assert abs(E2 - lam * E1) <= 1e-13 * abs(E1)


def test_pz_branches_join_at_rs_one():
    """The two Perdew-Zunger branches are fitted to meet at r_s = 1: energy and
    potential agree there to the fit's precision (a few 1e-5 Ha)."""
    lo, hi = 1.0 - 1e-12, 1.0
    assert abs(xc.eps_c(lo) - xc.eps_c(hi)) < 1e-4
    rho_lo = 3.0 / (4.0 * np.pi * lo ** 3)
    rho_hi = 3.0 / (4.0 * np.pi * hi ** 3)
    vlo = xc.xc_potential(np.array([rho_lo])) - xc.eps_x(rho_lo) * 4.0 / 3.0
    vhi = xc.xc_potential(np.array([rho_hi])) - xc.eps_x(rho_hi) * 4.0 / 3.0
    assert abs(vlo[0] - vhi[0]) < 1e-4


def test_pz_high_density_coefficient_is_gell_mann_brueckner():
    """eps_c -> A ln r_s as r_s -> 0 with A = (1 - ln 2) / pi^2 (Gell-Mann and Brueckner);
    Perdew and Zunger's A is that number to three digits."""
    r1, r2 = 1e-6, 1e-7
    slope = (xc.eps_c(r1) - xc.eps_c(r2)) / (np.log(r1) - np.log(r2))
    assert abs(slope / ((1.0 - np.log(2.0)) / np.pi ** 2) - 1.0) < 1e-3


def test_xc_potential_is_the_derivative_of_the_energy_density():
    """V_xc(rho) = d(rho eps_xc)/d rho by central differences over both branches."""
    rho = np.geomspace(1e-5, 10.0, 400)
    h = 1e-6 * rho
    fd = (xc.xc_energy_density(rho + h) - xc.xc_energy_density(rho - h)) / (2.0 * h)
    V = xc.xc_potential(rho)
    assert np.max(np.abs(fd - V) / np.abs(V)) < 1e-8


def test_exchange_potential_is_four_thirds_of_the_energy_per_electron():
    rho = np.geomspace(1e-4, 5.0, 50)
    rs = xc.wigner_seitz_radius(rho)
    Vx = xc.eps_x(rho) - rs / 3.0 * xc.deps_x_drs(rs)
    assert np.allclose(Vx, 4.0 / 3.0 * xc.eps_x(rho), rtol=1e-14, atol=0.0)
