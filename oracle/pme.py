"""Smooth particle-mesh Ewald structure factor (test infrastructure only).

Sec. 2.5 of the paper: for more than ~1000 ions the structure factor
S(G) = sum_I exp(-i G.R_I) is computed by PME (Essmann et al. 1995).  With
fractional coordinates f and u_a = n_a f_a, each axis factor is interpolated by
cardinal B-splines M_p of even order p (support [0, p]):

    exp(-2 pi i m u / n)  ~  conj(b(m)) sum_k M_p(u - k) exp(-2 pi i m k / n),
    b(m) = exp(2 pi i (p-1) m / n) / sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / n)

(the complex conjugate of Essmann's Eq. 4.4 for our exp(-iG.R) sign), so that

    S(G) ~ prod_a conj(b_a(m_a)) * sum_k Q(k) exp(-2 pi i m.k / n),
    Q(k) = sum_I prod_a M_p(u_{a,I} - k_a)    (k periodic).

Energy and forces of the PME approximation follow from this S(G) exactly
(E_PP = sum_k Q(k) phi(k); F_I = -sum_k phi(k) dQ(k)/dR_I).
"""
from __future__ import annotations

import numpy as np

from .functionals import pp_form_factor
from .grid import Grid


def bspline(p: int, x):
    """Cardinal B-spline M_p(x) (support [0, p]) by the recursion
    M_p(x) = x/(p-1) M_{p-1}(x) + (p-x)/(p-1) M_{p-1}(x-1),  M_2(x) = 1 - |x - 1|."""
    x = np.asarray(x, dtype=np.float64)
    if p == 2:
        return np.where((x >= 0) & (x <= 2), 1.0 - np.abs(x - 1.0), 0.0)
    return (x * bspline(p - 1, x) + (p - x) * bspline(p - 1, x - 1.0)) / (p - 1)


def bspline_deriv(p: int, x):
    """dM_p/dx = M_{p-1}(x) - M_{p-1}(x - 1)."""
    return bspline(p - 1, x) - bspline(p - 1, x - 1.0)


def b_factor(n: int, p: int, m):
    m = np.asarray(m, dtype=np.float64)
    k = np.arange(p - 1)
    den = (bspline(p, k + 1.0)[None, :] * np.exp(2j * np.pi * m[:, None] * k[None, :] / n)).sum(1)
    return np.exp(2j * np.pi * (p - 1) * m / n) / den


def charge_grid(g: Grid, positions, p: int):
    """Q(k) = sum_I prod_a M_p(u_aI - k_a), spread on the full real grid."""
    frac = np.asarray(positions, dtype=np.float64).reshape(-1, 3) @ g.recip.T
    Q = np.zeros(g.shape)
    n = np.array(g.shape)
    for f in frac:
        u = (f % 1.0) * n
        ks, ws = [], []
        for a in range(3):
            k = np.floor(u[a]).astype(int) - np.arange(p)           # grid points with 0 < u - k < p
            ks.append(k % n[a])
            ws.append(bspline(p, u[a] - k))
        Q[np.ix_(ks[0], ks[1], ks[2])] += ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    return Q


def b_product(g: Grid, p: int):
    """prod_a conj(b_a(m_a)) on the half spectrum (indices k, not wrapped frequencies)."""
    n0, n1, n2 = g.shape
    b0 = np.conj(b_factor(n0, p, np.arange(n0)))
    b1 = np.conj(b_factor(n1, p, np.arange(n1)))
    b2 = np.conj(b_factor(n2, p, np.arange(n2 // 2 + 1)))
    return b0[:, None, None] * b1[None, :, None] * b2[None, None, :]


def structure_factor(g: Grid, positions, p: int):
    """PME approximation of S(G) = sum_I exp(-iG.R_I) on the half spectrum."""
    Q = charge_grid(g, positions, p)
    return b_product(g, p) * np.fft.rfftn(Q)


def external_potential_G(g: Grid, positions, species, Z, rc, p: int):
    """V_ext(G) = (1/Omega) sum_s v_s(|G|) S_s(G) with PME S_s; G = 0 uses the exact
    S(0) = number of ions of the species."""
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    species = np.asarray(species, dtype=int).reshape(-1)
    Vg = np.zeros(g.G2.shape, dtype=np.complex128)
    for s in range(len(Z)):
        sel = pos[species == s]
        if len(sel) == 0:
            continue
        S = structure_factor(g, sel, p)
        S[0, 0, 0] = len(sel)
        Vg += pp_form_factor(g.Gnorm, Z[s], rc[s]) * S
    return Vg / g.omega


def forces(g: Grid, rho, positions, species, Z, rc, p: int):
    """F_I = -dE_PP/dR_I of the PME energy: E_PP(G != 0) = sum_s sum_k Q_s(k) phi_s(k),
    phi_s = IFFT(rho_hat conj(prod conj b) v_s), gathered with the B-spline derivatives."""
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    species = np.asarray(species, dtype=int).reshape(-1)
    rh = g.fft(np.asarray(rho, dtype=np.float64))
    B = b_product(g, p)
    n = np.array(g.shape)
    F = np.zeros_like(pos)
    for s in range(len(Z)):
        v = pp_form_factor(g.Gnorm, Z[s], rc[s])
        Fs = rh * np.conj(B) * v
        Fs[0, 0, 0] = 0.0
        phi = g.ifft(Fs)
        for I in np.nonzero(species == s)[0]:
            u = ((pos[I] @ g.recip.T) % 1.0) * n
            ks, ws, ds = [], [], []
            for a in range(3):
                k = np.floor(u[a]).astype(int) - np.arange(p)
                ks.append(k % n[a])
                ws.append(bspline(p, u[a] - k))
                ds.append(bspline_deriv(p, u[a] - k))
            blk = phi[np.ix_(ks[0], ks[1], ks[2])]
            du = np.array([
                np.einsum("ijk,i,j,k->", blk, ds[0], ws[1], ws[2]),
                np.einsum("ijk,i,j,k->", blk, ws[0], ds[1], ws[2]),
                np.einsum("ijk,i,j,k->", blk, ws[0], ws[1], ds[2])])
            # du_a/dR = n_a b_a  ->  dE/dR = sum_a du_a n_a b_a
            F[I] = -(du * n) @ g.recip
    return F
