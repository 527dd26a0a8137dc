"""LDA exchange-correlation energy and potential (test infrastructure only).

The paper's benchmarks use LDA exchange-correlation with the Perdew-Zunger
parametrisation (Sec. 3.1, its reference to Perdew and Zunger, 1981): Dirac
exchange plus the Perdew-Zunger fit of the Ceperley-Alder correlation energy of
the uniform electron gas, spin unpolarised.  Hartree atomic units; with the
Wigner-Seitz radius r_s = (3 / (4 pi rho))^(1/3):

  exchange     eps_x(rho) = -(3/4) (3/pi)^(1/3) rho^(1/3)
  correlation  eps_c(r_s) = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)        r_s >= 1
               eps_c(r_s) = A ln r_s + B + C r_s ln r_s + D r_s              r_s <  1
  energy       E_xc = sum_r rho eps_xc(rho) dV
  potential    V_xc = d(rho eps_xc)/d rho = eps_xc - (r_s / 3) d eps_xc / d r_s

The potential is written out from that definition (the derivative of each
branch taken by hand below), not from the simplified closed forms.  The density
is floored at RHO_FLOOR as for the other terms.
"""
from __future__ import annotations

import numpy as np

from .functionals import RHO_FLOOR
from .grid import Grid

# Perdew-Zunger (1981) unpolarised constants (Hartree)
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
C_X = 0.75 * (3.0 / np.pi) ** (1.0 / 3.0)


def wigner_seitz_radius(rho):
    return (3.0 / (4.0 * np.pi * np.maximum(rho, RHO_FLOOR))) ** (1.0 / 3.0)


def eps_x(rho):
    return -C_X * np.maximum(rho, RHO_FLOOR) ** (1.0 / 3.0)


def deps_x_drs(rs):
    # eps_x = -C_X (3/(4 pi))^(1/3) / r_s
    return C_X * (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0) / rs ** 2


def eps_c(rs):
    rs = np.asarray(rs, dtype=np.float64)
    hi = PZ_GAMMA / (1.0 + PZ_BETA1 * np.sqrt(rs) + PZ_BETA2 * rs)
    lrs = np.log(rs)
    lo = PZ_A * lrs + PZ_B + PZ_C * rs * lrs + PZ_D * rs
    return np.where(rs >= 1.0, hi, lo)


def deps_c_drs(rs):
    rs = np.asarray(rs, dtype=np.float64)
    den = 1.0 + PZ_BETA1 * np.sqrt(rs) + PZ_BETA2 * rs
    hi = -PZ_GAMMA * (0.5 * PZ_BETA1 / np.sqrt(rs) + PZ_BETA2) / den ** 2
    lo = PZ_A / rs + PZ_C * (np.log(rs) + 1.0) + PZ_D
    return np.where(rs >= 1.0, hi, lo)


def xc_energy_density(rho):
    """rho eps_xc(rho) per unit volume."""
    r = np.maximum(np.asarray(rho, dtype=np.float64), RHO_FLOOR)
    return r * (eps_x(r) + eps_c(wigner_seitz_radius(r)))


def xc_potential(rho):
    r = np.maximum(np.asarray(rho, dtype=np.float64), RHO_FLOOR)
    rs = wigner_seitz_radius(r)
    eps = eps_x(r) + eps_c(rs)
    return eps - rs / 3.0 * (deps_x_drs(rs) + deps_c_drs(rs))


def lda_xc(g: Grid, rho):
    """E_xc = sum rho eps_xc dV and V_xc (Sec. 3.1's LDA, Perdew-Zunger correlation)."""
    rho = np.asarray(rho, dtype=np.float64)
    return float(np.sum(xc_energy_density(rho)) * g.dV), xc_potential(rho)
