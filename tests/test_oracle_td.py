"""Pins of the oracle's real-time TD-OFDFT (Sec. "Time-Dependent OFDFT", Eq. cn).

What the mathematics fixes, independent of the oracle's own arithmetic:
- Crank-Nicolson with a Hermitian H is unitary; its residual is checked with a
  Hamiltonian applied through full complex FFTs (not the oracle's real-part splitting);
- a plane wave in v = 0 and an eigenstate of a fixed potential pick up the CN phase
  ((1 - i tau e) / (1 + i tau e))^n exactly (eigenstate from Lanczos);
- CN with a fixed H is reversible (dt then -dt);
- after a kick e^{ikx} of a real psi, d<x>/dt = N_e k (continuity equation);
- the dipole of a displaced Gaussian is N_e times the displacement;
- the spectrum of a sampled damped sinusoid is a geometric series.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import functionals as fn
from oracle import td
from oracle.evaluate import Functional
from oracle.grid import Grid


def _box(n=24, L=14.0):
    return Grid(np.diag([L, L, L]), (n, n, n))


def _blob(g, centre=(0.0, 0.0, 0.0), sigma=1.6, ne=2.0):
    r = td.positions(g) - np.asarray(centre)
    rho = np.exp(-(r ** 2).sum(-1) / (2 * sigma ** 2))
    return rho * ne / (rho.sum() * g.dV)


def _h_full_fft(g, psi, v):
    """H psi with the full complex FFT (cubic cell): an independent kinetic operator."""
    n = g.shape
    m = [np.fft.fftfreq(k, 1.0 / k) for k in n]
    for a in range(3):
        if n[a] % 2 == 0:
            m[a][n[a] // 2] = n[a] / 2      # Nyquist as +n/2: G^2 is the same either way
    mm = np.meshgrid(*m, indexing="ij")
    G = 2 * np.pi * (mm[0][..., None] * g.recip[0] + mm[1][..., None] * g.recip[1] + mm[2][..., None] * g.recip[2])
    G2 = (G ** 2).sum(-1)
    return np.fft.ifftn(0.5 * G2 * np.fft.fftn(psi)) + v * psi


def test_cn_step_is_unitary_and_solves_the_system():
    g = _box(16, 10.0)
    rng = np.random.default_rng(1)
    v = 2.0 * np.cos(2 * np.pi * td.positions(g)[..., 0] / 10.0) + 0.5 * rng.random(g.shape)
    psi = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    dt = 0.2
    x, its = td.cn_solve(g, psi, v, dt)
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(psi) ** 2)) < 1e-11 * np.sum(np.abs(psi) ** 2)
    tau = dt / 2
    r = x + 1j * tau * _h_full_fft(g, x, v) - (psi - 1j * tau * _h_full_fft(g, psi, v))
    assert np.sqrt(np.sum(np.abs(r) ** 2)) < 1e-11 * np.sqrt(np.sum(np.abs(psi) ** 2))


def test_plane_wave_in_zero_potential_takes_the_cn_phase():
    g = _box(16, 10.0)
    G = 2 * np.pi * np.array([2.0, -1.0, 3.0]) / 10.0
    psi0 = np.exp(1j * (td.positions(g) @ G))
    rho0 = np.abs(psi0) ** 2
    dt, n = 0.3, 7
    psi, dip = td.propagate(g, psi0, rho0, Functional(terms=("VW",)), None, dt, n, n_corrector=1)
    e = 0.5 * G @ G
    phase = ((1 - 0.5j * dt * e) / (1 + 0.5j * dt * e)) ** n
    assert np.max(np.abs(psi - phase * psi0)) < 1e-11
    assert np.max(np.abs(dip)) < 1e-10


def test_eigenstate_of_a_fixed_potential_takes_the_cn_phase():
    import scipy.sparse.linalg as sla
    cell, pos = W.fcc_positions(1)
    g = Grid(cell, (16, 16, 16))
    Vg = fn.external_potential_G(g, pos, np.zeros(4, int), [3.0], [0.9])
    v = g.ifft(Vg)

    def mv(x):
        x = x.reshape(g.shape)
        return (0.5 * g.ifft(g.G2 * g.fft(x)) + v * x).reshape(-1)

    w, U = sla.eigsh(sla.LinearOperator((g.N, g.N), matvec=mv, dtype=np.float64), k=1, which="SA", tol=1e-14)
    psi0 = U[:, 0].reshape(g.shape)
    psi0 *= math.sqrt(12.0 / (np.sum(psi0 ** 2) * g.dV))
    dt, n = 0.1, 5
    psi, _ = td.propagate(g, psi0.astype(complex), psi0 ** 2, Functional(terms=("VW", "PP")), Vg, dt, n)
    phase = ((1 - 0.5j * dt * w[0]) / (1 + 0.5j * dt * w[0])) ** n
    assert np.max(np.abs(psi - phase * psi0)) < 1e-8 * np.max(np.abs(psi0))


def test_fixed_potential_propagation_is_reversible():
    g = _box(16, 10.0)
    rho0 = _blob(g, sigma=1.4)
    Vg = np.zeros(g.G2.shape, complex)
    psi0 = td.kick(g, np.sqrt(rho0), [0.1, 0.0, 0.05])
    f = Functional(terms=("VW",))
    fwd, _ = td.propagate(g, psi0, rho0, f, Vg, 0.2, 6)
    back, _ = td.propagate(g, fwd, rho0, f, Vg, -0.2, 6)
    assert np.max(np.abs(back - psi0)) < 1e-11 * np.max(np.abs(psi0))


def test_nonlinear_propagation_conserves_charge():
    g = _box(20, 12.0)
    rho0 = _blob(g, sigma=1.5, ne=3.0)
    psi0 = td.kick(g, np.sqrt(rho0), [0.05, 0.0, 0.0])
    f = Functional(terms=("TF", "VW", "HARTREE"))
    psi, dip = td.propagate(g, psi0, rho0, f, None, 0.05, 4, n_corrector=2)
    assert abs(np.sum(np.abs(psi) ** 2) * g.dV - 3.0) < 1e-11
    assert dip[-1][0] > 0.0


def test_initial_dipole_velocity_is_ne_k():
    """d<x>/dt at t = 0+ equals int j_x = N_e k for a kicked real psi (continuity): the
    one-step dipole velocity differs from it at O(dt^2) (the blob's acceleration vanishes by
    symmetry), so the Richardson extrapolation of two steps hits N_e k."""
    g = _box(24, 14.0)
    rho0 = _blob(g, sigma=1.0, ne=2.0)
    k = 0.01
    f = Functional(terms=("TF", "VW", "HARTREE"))
    err = []
    for dt in (0.02, 0.01):
        _, dip = td.propagate(g, td.kick(g, np.sqrt(rho0), [k, 0, 0]), rho0, f, None, dt, 1, n_corrector=2)
        err.append(dip[1][0] / dt / (2.0 * k) - 1.0)
        assert abs(dip[1][1]) < 1e-10 and abs(dip[1][2]) < 1e-10
    assert abs(err[1]) < 2e-4
    assert abs(4.0 * err[1] - err[0]) / 3.0 < 1e-5, err


def test_dipole_of_a_displaced_gaussian_and_kick_modulus():
    g = _box(24, 14.0)
    rho0 = _blob(g, sigma=1.0, ne=2.0)
    d = np.array([0.4, -0.3, 0.2])
    rho1 = _blob(g, centre=d, sigma=1.0, ne=2.0)
    assert np.max(np.abs(td.dipole(g, rho1, rho0) - 2.0 * d)) < 1e-8
    psi = td.kick(g, np.sqrt(rho0), [0.3, 0.1, -0.2])
    assert np.max(np.abs(np.abs(psi) ** 2 - rho0)) < 1e-14


def test_spectrum_of_a_sampled_damped_sinusoid():
    dt, n, w0, A, gam = 0.1, 400, 1.3, 0.7, 0.02
    t = np.arange(n) * dt
    dmu = A * np.sin(w0 * t)
    omega = np.array([0.5, 1.0, 1.3, 2.0])
    got = td.spectrum(dmu, dt, omega, gam)
    ref = []
    for w in omega:
        s = 0.0
        for sgn in (1, -1):
            q = np.exp((1j * (w + sgn * w0) - gam) * dt)
            s += sgn * (1 - q ** n) / (1 - q) / (2j)
        ref.append(w * (A * s * dt).imag)
    assert np.max(np.abs(got - np.array(ref))) < 1e-10
    assert got[2] > 0.0                      # absorption peak at w0 is positive
