"""Ion-ion electrostatic energy and forces by Ewald summation (test infrastructure only).

The total energy of the paper's Eq. efunc becomes a full total energy, for
structures and forces, with the ion-ion term of point charges Z_I in a uniform
neutralising background (the electrons neutralise the cell).  Ewald's split with
parameter eta, over the lattice vectors L and the reciprocal vectors G != 0:

  E = 1/2 sum_{I,J,L}' Z_I Z_J erfc(eta r) / r                r = |R_I - R_J + L|
    + (2 pi / Omega) sum_G |S(G)|^2 exp(-G^2 / (4 eta^2)) / G^2,   S(G) = sum_I Z_I e^{i G.R_I}
    - (eta / sqrt(pi)) sum_I Z_I^2 - pi (sum_I Z_I)^2 / (2 Omega eta^2)

(the prime drops I = J at L = 0).  E does not depend on eta; both sums are cut
where their terms fall below ~1e-16.  F_I = -dE/dR_I:

  F_I = Z_I sum_{J,L}' Z_J [erfc(eta r)/r^2 + 2 eta/sqrt(pi) exp(-eta^2 r^2)/r] (R_I - R_J + L)/r
      + (4 pi / Omega) Z_I sum_G G exp(-G^2/(4 eta^2))/G^2 Im[conj(S(G)) e^{i G.R_I}]
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

CUT = 6.0     # erfc(6) ~ 2e-17, exp(-36) ~ 2e-16


def ewald(cell, positions, charges, eta=None):
    """Returns (E [Ha], F [N][3] Ha/bohr)."""
    A = np.asarray(cell, dtype=np.float64)
    R = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    Z = np.asarray(charges, dtype=np.float64).reshape(-1)
    N = len(Z)
    omega = abs(np.linalg.det(A))
    B = 2.0 * np.pi * np.linalg.inv(A).T                   # rows: reciprocal basis
    if eta is None:
        eta = math.sqrt(math.pi) * (max(N, 1) / omega ** 2) ** (1.0 / 6.0)
    rc, gc = CUT / eta, 2.0 * eta * CUT
    # ---- real space: every image shift whose cell can hold a pair within rc
    width = omega / np.linalg.norm(np.cross(A[[1, 2, 0]], A[[2, 0, 1]]), axis=1)   # plane spacings
    nimg = np.ceil(rc / width).astype(int) + 1
    E_real = 0.0
    F = np.zeros((N, 3))
    d0 = R[:, None, :] - R[None, :, :]                       # R_I - R_J
    ZZ = Z[:, None] * Z[None, :]
    for i in range(-nimg[0], nimg[0] + 1):
        for j in range(-nimg[1], nimg[1] + 1):
            for k in range(-nimg[2], nimg[2] + 1):
                L = i * A[0] + j * A[1] + k * A[2]
                d = d0 + L
                r = np.linalg.norm(d, axis=-1)
                if i == j == k == 0:
                    np.fill_diagonal(r, np.inf)
                m = r < rc
                if not m.any():
                    continue
                rr = np.where(m, r, 1.0)
                e = np.where(m, ZZ * erfc(eta * rr) / rr, 0.0)
                E_real += 0.5 * e.sum()
                fr = np.where(m, ZZ * (erfc(eta * rr) / rr ** 2
                                       + 2.0 * eta / math.sqrt(math.pi) * np.exp(-(eta * rr) ** 2) / rr) / rr, 0.0)
                F += (fr[..., None] * d).sum(axis=1)
    # ---- reciprocal space: G = m . B inside the sphere |G| < gc
    mmax = np.ceil(gc / (2.0 * np.pi / np.linalg.norm(A, axis=1))).astype(int) + 1
    E_rec = 0.0
    for i in range(-mmax[0], mmax[0] + 1):
        for j in range(-mmax[1], mmax[1] + 1):
            for k in range(-mmax[2], mmax[2] + 1):
                if i == j == k == 0:
                    continue
                G = i * B[0] + j * B[1] + k * B[2]
                G2 = G @ G
                if G2 >= gc * gc:
                    continue
                f = math.exp(-G2 / (4.0 * eta * eta)) / G2
                ph = np.exp(1j * (R @ G))
                S = np.sum(Z * ph)
                E_rec += 2.0 * np.pi / omega * f * abs(S) ** 2
                F += (4.0 * np.pi / omega * f * Z * np.imag(np.conj(S) * ph))[:, None] * G[None, :]
    E_self = -eta / math.sqrt(math.pi) * np.sum(Z * Z)
    E_bg = -math.pi * np.sum(Z) ** 2 / (2.0 * omega * eta * eta)
    return E_real + E_rec + E_self + E_bg, F
