"""MGP-family kernels of the oracle (test infrastructure only).

Eq. MGP of Sec. 2.3:
    omega_{x,y}(q) = omega_WT(q) - x C_WT int_0^1 dt t^y dG_NL(eta(q, t))/dt,
with MGP (x, y) = (1, 5/6), MGPA (1/2, 5/6), MGPG (1, 5/3); with the spline steps s1-s4
the same kernels at the local k_F give LMGP/A/G.

Reading (the text leaves eta(q, t) undefined): eta(q, t) = q / (2 k_F t^(1/3)), the
reduced wavevector at the Fermi wavevector of the scaled density t rho, the path
rho_t = t rho of the functional integration the correction term comes from.

With t = s^3 and an integration by parts (t^y G vanishes at t = 0: G_NL is bounded),
    I_y(eta) = int_0^1 t^y dG/dt dt = G_NL(eta) - 3y J_y(eta),
    J_y(eta) = int_0^1 s^(3y-1) G_NL(eta/s) ds = 2 int_0^1 r^(6y-1) G_NL(eta/r^2) dr  (s = r^2),
and J_y is evaluated by tanh-sinh (double-exponential) quadrature on [0, sqrt(eta)] and
[sqrt(eta), 1] (split at the logarithmic kink of G_NL at argument 1; one piece when
eta >= 1), vectorised over the distinct eta values.
    omega = C_WT (G_NL(eta) - x I_y(eta)) = C_WT ((1 - x) G_NL(eta) + 3 x y J_y(eta)).
"""
from __future__ import annotations

import numpy as np

from .lindhard import C_WT, G_NL


def _ts_rule(h: float = 1.0 / 64.0, tmax: float = 3.2):
    """Tanh-sinh abscissae on [-1, 1] as distances to the nearer end, with weights."""
    t = np.arange(-tmax, tmax + 0.5 * h, h)
    u = 0.5 * np.pi * np.sinh(t)
    w = h * 0.5 * np.pi * np.cosh(t) / np.cosh(u) ** 2
    d = 2.0 / (np.exp(2.0 * np.abs(u)) + 1.0)          # 1 - |x|, without cancellation
    return np.sign(t), d, w


def _piece(eta, a, b, y, rule):
    """2 int_a^b r^(6y-1) G_NL(eta/r^2) dr for arrays eta, a, b."""
    sgn, d, w = rule
    half = 0.5 * (b - a)[:, None]
    r = np.where(sgn[None, :] < 0, a[:, None] + half * d[None, :], b[:, None] - half * d[None, :])
    f = 2.0 * r ** (6.0 * y - 1.0) * G_NL(eta[:, None] / (r * r))
    return half[:, 0] * np.sum(w[None, :] * f, axis=1)


def mgp_J(eta, y: float) -> np.ndarray:
    """J_y(eta) = int_0^1 s^(3y-1) G_NL(eta/s) ds, elementwise (J_y(0) = 0)."""
    eta = np.asarray(eta, dtype=np.float64)
    u, inv = np.unique(eta.ravel(), return_inverse=True)
    out = np.zeros_like(u)
    pos = u > 0.0
    e = u[pos]
    rule = _ts_rule()
    k = np.sqrt(np.minimum(e, 1.0))
    out[pos] = _piece(e, np.zeros_like(e), k, y, rule) + np.where(e < 1.0, _piece(e, k, np.ones_like(e), y, rule), 0.0)
    return out[inv].reshape(eta.shape)


def mgp_correction(eta, y: float) -> np.ndarray:
    """I_y(eta) = int_0^1 t^y dG_NL(eta t^(-1/3))/dt dt = G_NL(eta) - 3y J_y(eta)."""
    eta = np.asarray(eta, dtype=np.float64)
    return G_NL(eta) - 3.0 * y * mgp_J(eta, y)


def kernel(eta, x: float = 0.0, y: float = 5.0 / 6.0) -> np.ndarray:
    """C_WT (G_NL(eta) - x I_y(eta)); x = 0 is the Wang-Teter kernel of Eq. WT."""
    eta = np.asarray(eta, dtype=np.float64)
    if x == 0.0:
        return C_WT * G_NL(eta)
    return C_WT * ((1.0 - x) * G_NL(eta) + 3.0 * x * y * mgp_J(eta, y))
