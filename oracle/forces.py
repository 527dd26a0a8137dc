"""Ionic forces of the oracle (test infrastructure only).

E_PP = int rho v_ext = Omega sum_G conj(rho_hat(G)) V_ext(G) with
V_ext(G) = (1/Omega) sum_I v(|G|) exp(-i G.R_I) (Sec. 2.5 structure factor);
differentiating the phase gives

    F_I = -dE/dR_I = -sum_G G v(|G|) Im[conj(rho_hat(G)) exp(-i G.R_I)].

Only the electron-ion term depends on R_I: Eq. efunc has no ion-ion term.
"""
from __future__ import annotations

import numpy as np

from .functionals import pp_form_factor
from .grid import Grid


def forces(g: Grid, rho, positions, species, Z, rc):
    rh = g.fft(np.asarray(rho, dtype=np.float64))
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    species = np.asarray(species, dtype=int).reshape(-1)
    F = np.zeros_like(pos)
    for I in range(len(pos)):
        s = species[I]
        v = pp_form_factor(g.Gnorm, Z[s], rc[s])
        im = np.imag(np.conj(rh) * np.exp(-1j * (g.G @ pos[I])))
        F[I] = -np.einsum("ijk,ijkc->c", g.weights * v * im, g.G)
    return F
