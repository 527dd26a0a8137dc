"""Lindhard function and Wang-Teter kernel (test infrastructure only).

Sec. 2.3, Eq. WT and the G_NL definition below Eq. MGP:
    G_NL(eta) = (1/2 + (1 - eta^2)/(4 eta) ln|(1+eta)/(1-eta)|)^-1 - 3 eta^2 - 1,
    omega_WT(q) = C_WT G_NL(q / 2kF),   C_WT = (6/25)(3 pi^2)^(2/3).

F(eta) (the bracket) is evaluated from its closed form for 0.5 <= eta <= 2
and from the exact convergent expansions of the logarithm elsewhere,
    F = 1 - sum_{m>=1} eta^(2m)/(4m^2-1)        (eta < 1)
    F =     sum_{m>=1} eta^(-2m)/(4m^2-1)       (eta > 1),
obtained by inserting ln((1+x)/(1-x)) = 2 sum x^(2k+1)/(2k+1) into the
closed form.  For eta > 2 the difference 1/F - 3 eta^2 - 1 cancels; with
x = 1/eta^2 it is rewritten exactly as
    G_NL = -(sum_{m>=1} d_m x^m) / F,   d_m = 1/(4m^2-1) + 3/(4(m+1)^2-1),
(multiply F's series by 3/x + 1 and collect powers of x).
Special values: G_NL(0) = 0, G_NL(1) = -2, G_NL(inf) = -8/5.
"""
from __future__ import annotations

import numpy as np

C_WT = 6.0 / 25.0 * (3.0 * np.pi ** 2) ** (2.0 / 3.0)


def _series(x: np.ndarray, n_terms: int = 40) -> np.ndarray:
    """sum_{m>=1} x^m / (4 m^2 - 1) for 0 <= x <= 1/4 (terms below 1e-25 at 40)."""
    out = np.zeros_like(x)
    xm = np.ones_like(x)
    for m in range(1, n_terms + 1):
        xm = xm * x
        out += xm / (4.0 * m * m - 1.0)
    return out


def lindhard_F(eta) -> np.ndarray:
    eta = np.asarray(eta, dtype=np.float64)
    F = np.empty_like(eta)
    lo = eta < 0.5
    hi = eta > 2.0
    mid = ~(lo | hi)
    F[lo] = 1.0 - _series(eta[lo] ** 2)
    F[hi] = _series(1.0 / eta[hi] ** 2)
    e = eta[mid]
    with np.errstate(divide="ignore", invalid="ignore"):
        Fm = 0.5 + (1.0 - e * e) / (4.0 * e) * np.log(np.abs((1.0 + e) / (1.0 - e)))
    Fm = np.where(e == 1.0, 0.5, Fm)
    F[mid] = Fm
    return F


def G_NL(eta) -> np.ndarray:
    """G_NL(eta) of the paper; G_NL(0) = 0 exactly."""
    eta = np.asarray(eta, dtype=np.float64)
    F = lindhard_F(eta)
    g = 1.0 / F - 3.0 * eta * eta - 1.0
    hi = eta > 2.0
    if np.any(hi):
        x = 1.0 / eta[hi] ** 2
        num = np.zeros_like(x)
        xm = np.ones_like(x)
        for m in range(1, 41):
            xm = xm * x
            num += xm * (1.0 / (4.0 * m * m - 1.0) + 3.0 / (4.0 * (m + 1) ** 2 - 1.0))
        g[hi] = -num / F[hi]
    return np.where(eta == 0.0, 0.0, g)


def wt_kernel(q, kF: float) -> np.ndarray:
    """omega_WT(q) = C_WT G_NL(q / (2 kF))  (Eq. WT)."""
    return C_WT * G_NL(np.asarray(q, dtype=np.float64) / (2.0 * kF))
