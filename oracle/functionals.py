"""Energy functionals and their potentials (test infrastructure only).

Each function returns (E [Ha], V [Ha/e] on the real grid), V = dE/drho as a
functional derivative, i.e. dE/drho_r = V_r * dV for the discrete energy.
All arithmetic is FP64 and follows the paper (Sec. 1 Eqs. efunc/euler,
Sec. 2.3 Eqs. nl2, WT, the G_NL definition and steps s1-s4, Sec. 2.4
Eq. euler2) together with the readings listed where the paper is silent.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .lindhard import C_WT, G_NL
from .mgp import kernel as mgp_kernel

C_TF = 0.3 * (3.0 * np.pi ** 2) ** (2.0 / 3.0)
RHO_FLOOR = 1e-20     # reading: guard for rho^(alpha-1), 1/psi and kF (paper silent)


# --------------------------------------------------------------------------- semilocal
def thomas_fermi(g: Grid, rho):
    """T_TF = C_TF int rho^(5/3),  V_TF = (5/3) C_TF rho^(2/3)  (Sec. 2.3, Sec. 3.2)."""
    E = C_TF * np.sum(rho ** (5.0 / 3.0)) * g.dV
    V = (5.0 / 3.0) * C_TF * rho ** (2.0 / 3.0)
    return E, V


def von_weizsaecker(g: Grid, rho):
    """T_vW in the psi = sqrt(rho) form of Sec. 2.4:

        T_vW = 1/2 int psi (-lap psi) = (Omega/2) sum_G G^2 |psi_hat|^2,
        V_vW = (-lap psi) / (2 psi),   lap psi = IFFT(-G^2 psi_hat).

    Reading: the spectral Laplacian with the Nyquist plane kept; this is the
    exact derivative of the discrete energy."""
    psi = np.sqrt(rho)
    ph = g.fft(psi)
    E = 0.5 * g.omega * g.gsum(g.G2 * np.abs(ph) ** 2)
    minus_lap = g.ifft(g.G2 * ph)
    V = minus_lap / (2.0 * np.maximum(psi, np.sqrt(RHO_FLOOR)))
    return E, V


def hartree(g: Grid, rho):
    """E_H = (Omega/2) sum_{G!=0} 4 pi |rho_hat|^2 / G^2,  V_H = IFFT(4 pi rho_hat / G^2).

    Reading: the G = 0 term is dropped (neutralising background)."""
    rh = g.fft(rho)
    with np.errstate(divide="ignore", invalid="ignore"):
        kern = np.where(g.G2 > 0.0, 4.0 * np.pi / g.G2, 0.0)
    E = 0.5 * g.omega * g.gsum(kern * np.abs(rh) ** 2)
    V = g.ifft(kern * rh)
    return E, V


# --------------------------------------------------------------------------- ions
def pp_form_factor(q, Z: float, rc: float):
    """v(q) = -4 pi Z exp(-(q rc)^2 / 4) / q^2 for q > 0 (real space -Z erf(r/rc)/r).

    Reading for q = 0 (paper silent): the finite part pi Z rc^2 of
    v(q) + 4 pi Z / q^2, i.e. the Coulomb tail is neutralised like E_H."""
    q = np.asarray(q, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -4.0 * np.pi * Z * np.exp(-(q * rc) ** 2 / 4.0) / (q * q)
    return np.where(q > 0.0, v, np.pi * Z * rc * rc)


def external_potential_G(g: Grid, positions, species, Z, rc):
    """V_ext(G) = (1/Omega) sum_I v_{s(I)}(|G|) exp(-i G.R_I): direct structure factor (Sec. 2.5)."""
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    species = np.asarray(species, dtype=int).reshape(-1)
    Vg = np.zeros(g.G2.shape, dtype=np.complex128)
    for s in range(len(Z)):
        S = np.zeros(g.G2.shape, dtype=np.complex128)
        for I in np.nonzero(species == s)[0]:
            S += np.exp(-1j * (g.G @ pos[I]))
        Vg += pp_form_factor(g.Gnorm, Z[s], rc[s]) * S
    return Vg / g.omega


def local_pseudopotential(g: Grid, rho, Vext_G):
    """E_PP = int v_ext rho,  V_PP = v_ext(r) = IFFT(V_ext(G))  (Eq. efunc)."""
    vext = g.ifft(Vext_G)
    return np.sum(vext * rho) * g.dV, vext


# --------------------------------------------------------------------------- nonlocal
def fermi_wavevector(rho):
    """kF = (3 pi^2 rho)^(1/3) (Sec. 2.3, below Eq. WT), rho floored at RHO_FLOOR."""
    return np.cbrt(3.0 * np.pi ** 2 * np.maximum(rho, RHO_FLOOR))


def make_knots(rho, n_knots: int, spacing: str = "log"):
    """Step s1: M knots spanning [kF_min, kF_max] of the density.

    'log' is the geometric progression k_m = kmin (kmax/kmin)^(m/(M-1)), with
    the last knot set to kmax exactly; 'arith' the arithmetic progression."""
    kmin = float(fermi_wavevector(np.min(rho)))
    kmax = float(fermi_wavevector(np.max(rho)))
    m = np.arange(n_knots, dtype=np.float64)
    if spacing == "log":
        k = kmin * np.exp(m * (np.log(kmax / kmin) / (n_knots - 1)))
    else:
        k = kmin + m * ((kmax - kmin) / (n_knots - 1))
    k[0], k[-1] = kmin, kmax
    return k


def spline_weights(kF, knots):
    """Step s4 linear spline in kF: interval j with k_j <= kF < k_{j+1} (kF clamped to
    [k_0, k_{M-1}], j clamped to [0, M-2], so kF = k_{M-1} gives j = M-2, t = 1),
    t = (kF - k_j)/(k_{j+1} - k_j); h_j = 1 - t, h_{j+1} = t, h'_j = -1/dk, h'_{j+1} = +1/dk.
    A zero-width interval (all knots equal) gets t = 0 and slope 0.

    Returns (j, t, inv_dk, inside) with `inside` = kF within the knot range."""
    M = len(knots)
    inside = (kF >= knots[0]) & (kF <= knots[-1])
    kc = np.clip(kF, knots[0], knots[-1])
    j = np.clip(np.searchsorted(knots, kc, side="right") - 1, 0, M - 2)
    dk = knots[j + 1] - knots[j]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_dk = np.where(dk > 0.0, 1.0 / dk, 0.0)
    t = (kc - knots[j]) * inv_dk
    return j, t, inv_dk, inside


def nonlocal_lwt(g: Grid, rho, knots, alpha=5.0 / 6.0, beta=5.0 / 6.0, potential="exact", mgp=(0.0, 5.0 / 6.0)):
    """Density-dependent-kernel KEDF (LWT) through steps s1-s4 (Sec. 2.3).

    Energy (reading of Eq. nl2 with the kernel at the local kF(r)):
        T_NL = sum_r rho^alpha(r) Phi(r) dV,  Phi = sum_j h_j(kF(r)) y_j(r),
        y_j = K_j * rho^beta   (step s3, one convolution per knot).
    Potential 'exact' = the derivative of that discrete energy:
        V = alpha rho^(alpha-1) Phi + beta rho^(beta-1) sum_j K_j * (h_j rho^alpha)
            + rho^alpha Psi kF/(3 rho),   Psi = sum_j h'_j(kF) y_j.
    Potential 'interpolated' = the paper's s3->s4 blend of per-knot WT
    potentials, 2 alpha rho^(alpha-1) Phi (alpha = beta only): same energy,
    not the exact derivative.
    mgp = (x, y): the knots' kernels are those of Eq. MGP (x = 0: Eq. WT), giving LMGP/A/G."""
    rf = np.maximum(rho, RHO_FLOOR)
    kF = fermi_wavevector(rho)
    j, t, inv_dk, inside = spline_weights(kF, knots)
    M = len(knots)
    rb_hat = g.fft(rf ** beta)
    ra = rf ** alpha
    Phi = np.zeros_like(rf)
    Psi = np.zeros_like(rf)
    T2 = np.zeros_like(rf)
    for m in range(M):                      # one knot at a time: memory O(N)
        K = mgp_kernel(g.Gnorm / (2.0 * knots[m]), *mgp)    # step s2
        y = g.ifft(K * rb_hat)                               # step s3
        h = np.where(j == m, 1.0 - t, 0.0) + np.where(j == m - 1, t, 0.0)
        hp = np.where(j == m, -inv_dk, 0.0) + np.where(j == m - 1, inv_dk, 0.0)
        Phi += h * y                                         # step s4
        Psi += hp * y
        if potential == "exact":
            T2 += g.ifft(K * g.fft(h * ra))
    E = np.sum(ra * Phi) * g.dV
    if potential == "interpolated":
        if alpha != beta:
            raise ValueError("interpolated potential needs alpha == beta")
        return E, 2.0 * alpha * rf ** (alpha - 1.0) * Phi
    V = alpha * rf ** (alpha - 1.0) * Phi + beta * rf ** (beta - 1.0) * T2 \
        + np.where(inside, ra * Psi * kF / (3.0 * rf), 0.0)
    return E, V


def nonlocal_wt_global(g: Grid, rho, alpha=5.0 / 6.0, beta=5.0 / 6.0, rho0=None, mgp=(0.0, 5.0 / 6.0)):
    """Wang-Teter with one kernel at kF(rho0), rho0 = N_e/Omega (Eq. nl2 with Eq. WT; with
    mgp = (x, y), x != 0, the kernel of Eq. MGP: the MGP/A/G functionals):
        E = int rho^alpha (K * rho^beta),
        V = alpha rho^(alpha-1) (K * rho^beta) + beta rho^(beta-1) (K * rho^alpha)."""
    rf = np.maximum(rho, RHO_FLOOR)
    if rho0 is None:
        rho0 = np.sum(rho) * g.dV / g.omega
    K = mgp_kernel(g.Gnorm / (2.0 * float(fermi_wavevector(rho0))), *mgp)
    cb = g.ifft(K * g.fft(rf ** beta))
    ca = g.ifft(K * g.fft(rf ** alpha))
    E = np.sum(rf ** alpha * cb) * g.dV
    V = alpha * rf ** (alpha - 1.0) * cb + beta * rf ** (beta - 1.0) * ca
    return E, V
