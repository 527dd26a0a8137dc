"""Real-time TD-OFDFT of the oracle (test infrastructure only).

Sec. "Time-Dependent OFDFT" of the paper: a collective orbital psi = sqrt(rho) e^{iS}
obeys i dpsi/dt = H psi with H = -lap/2 + dT_Pauli/drho + v_s in the adiabatic
approximation.  For the energy functional E of Eq. efunc (T_vW included) this is

    H psi = -lap psi / 2 + v_eff[rho] psi,   v_eff = d(E - T_vW)/drho = V - V_vW,

so that H psi = V psi = mu psi at a ground state (Eq. of-ham).  Eq. cn advances psi by
one Crank-Nicolson step, solved as a linear system; the paper wraps it in a
predictor-corrector and kicks the ground state with a phase e^{ikx}; the dipole
change and its transform give the oscillator strength.

Readings (the paper states the equations only):
- CN sign: (1 + i dt/2 H) psi(t+dt) = (1 - i dt/2 H) psi(t), the step that integrates
  i dpsi/dt = H psi as printed.  The printed Eq. cn has the two signs exchanged; with the
  printed kick e^{-ikx} it gives the complex conjugate of this scheme's psi under the
  kick e^{+ikx}, hence the same rho(t), dipole and spectrum.  Here the kick is e^{+ik.r}.
- Predictor-corrector: the predictor solves the step with v_eff[rho(t)]; each corrector
  pass solves it again from psi(t) with (v_eff[rho(t)] + v_eff[rho_last(t+dt)]) / 2.
- The linear system is solved by the fixed-point iteration of the splitting
  (1 + i tau (K + vbar)) x = b - i tau (v - vbar) x, tau = dt/2, K = -lap/2 (diagonal in
  G), vbar = the midpoint of v's range; it contracts when tau max|v - vbar| < 1 (checked),
  and stops on the residual of the unsplit system.
- Positions are cell-centred: r = A^T (f - 1/2) for the fractional grid coordinates
  f = (i0/n0, i1/n1, i2/n2); they define the kick phase and the dipole.
- Dipole: delta mu(t) = sum_r r (rho(r, t) - rho0(r)) dV.
- Spectrum: delta mu~(w) = sum_n delta mu(t_n) e^{i w t_n} e^{-gamma t_n} dt over the
  recorded steps (gamma a damping the paper does not give), sigma(w) = w Im delta mu~(w).
Complex psi is stored as one complex array; -lap acts on its real and imaginary parts
as the real-field operator of oracle.grid (irfftn of the half spectrum).
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from .evaluate import Functional, evaluate
from .grid import Grid


def positions(g: Grid) -> np.ndarray:
    """Cell-centred Cartesian coordinates of the grid points, (n0, n1, n2, 3)."""
    f = np.meshgrid(*[np.arange(n) / n - 0.5 for n in g.shape], indexing="ij")
    return np.stack(f, -1) @ g.cell


def kinetic(g: Grid, psi):
    """K psi = -lap psi / 2 (spectral, on real and imaginary parts)."""
    def k(x):
        return 0.5 * g.ifft(g.G2 * g.fft(x))
    return k(psi.real) + 1j * k(psi.imag)


def effective_potential(g: Grid, rho, func: Functional, Vext_G):
    """v_eff = d(E - T_vW)/drho: the potential of every term of func but von Weizsaecker."""
    terms = tuple(t for t in func.terms if t != "VW")
    if not terms:
        return np.zeros(g.shape)
    return evaluate(g, rho, replace(func, terms=terms), Vext_G)[1]


def apply_h(g: Grid, psi, v):
    return kinetic(g, psi) + v * psi


def cn_solve(g: Grid, psi, v, dt: float, tol: float = 1e-13, max_iter: int = 500):
    """psi(t+dt) from (1 + i dt/2 H) x = (1 - i dt/2 H) psi, H = K + v (v fixed)."""
    tau = 0.5 * dt
    b = psi - 1j * tau * apply_h(g, psi, v)
    vbar = 0.5 * (float(v.max()) + float(v.min()))
    dv = v - vbar
    if tau * float(np.max(np.abs(dv))) >= 0.9:
        raise ValueError("time step too long for the splitting iteration")
    # (1 + i tau (K + vbar))^{-1} on real and imaginary parts' half spectra
    m = 1.0 / (1.0 + 1j * tau * (0.5 * g.G2 + vbar))

    def minv(y):
        a, c = g.fft(y.real), g.fft(y.imag)
        # the complex field's spectrum is a + i c; scale it by m and split back
        return g.ifft(m.real * a - m.imag * c) + 1j * g.ifft(m.real * c + m.imag * a)

    x = psi.copy()
    nb = math.sqrt(float(np.sum(np.abs(b) ** 2)))
    for it in range(max_iter):
        x = minv(b - 1j * tau * dv * x)
        r = x + 1j * tau * apply_h(g, x, v) - b
        if math.sqrt(float(np.sum(np.abs(r) ** 2))) <= tol * nb:
            return x, it + 1
    raise RuntimeError("Crank-Nicolson solve did not converge")


def td_step(g: Grid, psi, func: Functional, Vext_G, dt: float, n_corrector: int = 1, v_t=None):
    """One predictor-corrector Crank-Nicolson step; returns (psi(t+dt), v_eff at rho(t+dt))."""
    if v_t is None:
        v_t = effective_potential(g, np.abs(psi) ** 2, func, Vext_G)
    x, _ = cn_solve(g, psi, v_t, dt)
    v_new = effective_potential(g, np.abs(x) ** 2, func, Vext_G)
    for _ in range(n_corrector):
        x, _ = cn_solve(g, psi, 0.5 * (v_t + v_new), dt)
        v_new = effective_potential(g, np.abs(x) ** 2, func, Vext_G)
    return x, v_new


def kick(g: Grid, psi, k):
    """psi(r) e^{i k . r} with cell-centred r."""
    return psi * np.exp(1j * (positions(g) @ np.asarray(k, dtype=np.float64)))


def dipole(g: Grid, rho, rho0):
    """delta mu = sum_r r (rho - rho0) dV, a 3-vector."""
    return np.tensordot(rho - rho0, positions(g), axes=([0, 1, 2], [0, 1, 2])) * g.dV


def propagate(g: Grid, psi0, rho0, func: Functional, Vext_G, dt: float, n_steps: int, n_corrector: int = 1):
    """n_steps steps from psi0; returns (psi, dipoles [n_steps + 1][3])."""
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    dip = [dipole(g, np.abs(psi) ** 2, rho0)]
    v = None
    for _ in range(n_steps):
        psi, v = td_step(g, psi, func, Vext_G, dt, n_corrector, v)
        dip.append(dipole(g, np.abs(psi) ** 2, rho0))
    return psi, np.array(dip)


def spectrum(dmu, dt: float, omega, gamma: float):
    """sigma(w) = w Im sum_n dmu_n e^{(i w - gamma) t_n} dt, t_n = n dt."""
    dmu = np.asarray(dmu, dtype=np.float64)
    t = np.arange(len(dmu)) * dt
    out = []
    for w in np.asarray(omega, dtype=np.float64):
        out.append(w * float(np.sum(dmu * np.exp((1j * w - gamma) * t)).imag) * dt)
    return np.array(out)
