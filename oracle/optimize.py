"""psi = sqrt(rho) density optimiser of the oracle (test infrastructure only).

Sec. 2.4: minimise E[psi^2] subject to int psi^2 = N_e (Eq. euler2), repeating
(1) a search direction p_k, (2) a line search for lambda_k, (3) the update
psi_{k+1} = psi_k cos(lambda_k) + p_k sin(lambda_k) with p_k orthogonal to
psi_k and normalised to N_e, which conserves the charge exactly.

Step (1) offers the three direction methods the paper names (Sec. 2.4):
nonlinear conjugate gradient, truncated Newton (TN) and limited-memory BFGS.

Readings (the paper leaves them to SciPy and to its references):
- CG: Polak-Ribiere+, restarted on loss of descent and every 50 iterations.
- TN: the Newton equation H x = -g is solved approximately by an inner CG
  (Newton-CG, stopped when |r| < min(0.5, sqrt(res)) |g| with res the RMS
  Euler-Lagrange residual per electron, |g| / (2 sqrt(dV N_e)), or at the first
  direction of non-positive curvature), in the tangent space of the sphere
  int psi^2 = N_e; H is the Hessian of the Lagrangian E - mu (int psi^2 - N_e),
  applied by central finite differences of the gradient 2 psi V[psi^2] dV.
- L-BFGS: two-loop recursion over the last m pairs (s, y) of steps in psi and
  changes of the projected gradient, initial inverse Hessian (s.y / y.y) I;
  a pair with s.y <= 0 is not stored; the memory is cleared on a failed search.
- Step (3), the update: the orthogonal psi cos(lambda) + p sin(lambda) (default), or
  the scaling scheme psi + t p renormalised to N_e with p not orthogonalised (with p
  orthogonal to psi the two are one curve, t = tan(lambda)).
- The paper's two ways to optimise: the step minimises the energy (default) or the norm of
  the residual of Eq. euler2, |2 psi (V - mu) dV| (backtracking from the first trial by
  halves until the norm falls by the factor 1 - c1; the directions are the same).
- Step (2): a strong-Wolfe line search on lambda (c1 = 1e-4, c2 = 0.2, at most
  10 evaluations per search, cubic interpolation).  A TN or L-BFGS direction
  built from curvature starts from the length of its step,
  lambda = atan(|x_perp| / |psi|), which the rotation maps psi + x_perp onto;
  CG and steepest-descent fallbacks from the last accepted lambda.
- The spline knots are recomputed at the start of every iteration and frozen
  inside its line search; convergence when |E_k - E_{k-1}| < tol * n_atoms for
  3 consecutive iterations.
Parity unpinned for the trajectory: only the converged energy is compared.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from . import functionals as fn
from .evaluate import Functional, evaluate
from .grid import Grid


def _cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic through (a, fa, da), (b, fb, db); None if not defined."""
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def hessian_vector(g: Grid, psi, x, func: Functional, Vext_G, mu: float, h: float = 1e-4):
    """Hessian of the Lagrangian E[psi^2] - mu (int psi^2 - N_e) applied to x, by
    central differences of the gradient dE/dpsi = 2 psi V[psi^2] dV:

        H x = (grad(psi + e x) - grad(psi - e x)) / (2 e) - 2 mu dV x,
        e = h |psi| / |x|.

    Returns (H x, number of evaluations used)."""
    e = h * math.sqrt(np.sum(psi * psi) / np.sum(x * x))
    gp = 2.0 * (psi + e * x) * evaluate(g, (psi + e * x) ** 2, func, Vext_G)[1] * g.dV
    gm = 2.0 * (psi - e * x) * evaluate(g, (psi - e * x) ** 2, func, Vext_G)[1] * g.dV
    return (gp - gm) / (2.0 * e) - 2.0 * mu * g.dV * x, 2


def update_curve(psi, p, t: float, dV: float, n_electrons: float, update: str = "rotate"):
    """Step (3) of Sec. 2.4: the trial psi at step t along p and its derivative in t.
    rotate: psi cos t + p sin t (p orthogonal to psi, int p^2 = N_e);
    scale:  psi_t = c (psi + t p), c = sqrt(N_e / n), n = int (psi + t p)^2, so that
            d psi_t / dt = c p - (n' / 2n) psi_t with n' = 2 int (psi + t p) p."""
    if update == "rotate":
        return psi * math.cos(t) + p * math.sin(t), -psi * math.sin(t) + p * math.cos(t)
    q = psi + t * p
    n = np.sum(q * q) * dV
    c = math.sqrt(n_electrons / n)
    psi_t = c * q
    return psi_t, c * p - (np.sum(q * p) * dV / n) * psi_t


def _tangent(v, psi):
    """Component of v orthogonal to psi."""
    return v - (np.sum(v * psi) / np.sum(psi * psi)) * psi


def optimize_density(g: Grid, psi0, func: Functional, Vext_G, n_electrons: float, n_atoms: int,
                     tol: float = 1e-6, max_iter: int = 200, c1: float = 1e-4, c2: float = 0.2,
                     max_ls: int = 10, fixed_iter: int | None = None, method: str = "cg",
                     max_inner: int = 20, lbfgs_m: int = 5, update: str = "rotate", objective: str = "energy"):
    """method: 'cg' | 'tn' | 'lbfgs'; update: 'rotate' (psi cos + p sin, p orthogonal to psi)
    or 'scale' (psi + t p renormalised, p not orthogonalised); objective of the line search:
    'energy' (direct minimisation) or 'residual' (the norm of Eq. euler2's residual).
    Returns dict(psi, E, energies, iterations, evals, history)."""
    if method not in ("cg", "tn", "lbfgs"):
        raise ValueError("unknown method %r" % method)
    if update not in ("rotate", "scale"):
        raise ValueError("unknown update %r" % update)
    if objective not in ("energy", "residual"):
        raise ValueError("unknown objective %r" % objective)
    psi = np.asarray(psi0, dtype=np.float64).copy()
    psi *= math.sqrt(n_electrons / (np.sum(psi * psi) * g.dV))
    evals = 0

    def energy(psi_l, f):
        nonlocal evals
        evals += 1
        E, V = evaluate(g, psi_l * psi_l, f, Vext_G)
        return E, V

    def frozen(psi_l):
        if "NL" in func.terms and func.kernel == "lwt" and func.knots is None:
            return replace(func, knots=fn.make_knots(psi_l * psi_l, func.n_knots, func.spacing))
        return func

    f_it = frozen(psi)
    E, V = energy(psi, f_it)
    history = [E["total"]]
    d_prev = None
    g_prev = None
    pairs = []                    # L-BFGS memory: (s, y, 1 / s.y)
    psi_prev = None
    lam_prev = 0.05
    small = 0
    it = 0
    while it < max_iter:
        it += 1
        dEdpsi = 2.0 * psi * V * g.dV
        mu = np.sum(psi * dEdpsi) / (2.0 * n_electrons)
        grad = dEdpsi - 2.0 * mu * psi * g.dV
        newton = False                # direction built from curvature information
        if method == "cg":
            if d_prev is None or it % 50 == 1:
                d = -grad
            else:
                beta = max(0.0, float(np.sum(grad * (grad - g_prev)) / np.sum(g_prev * g_prev)))
                d = -grad + beta * d_prev
                if np.sum(d * grad) >= 0.0:
                    d = -grad
        elif method == "tn":
            # inner CG on H x = -grad (tangent space), forcing term eta |grad|
            gn = math.sqrt(np.sum(grad * grad))
            stop = min(0.5, math.sqrt(gn / (2.0 * math.sqrt(g.dV * n_electrons)))) * gn
            x = np.zeros_like(psi)
            r = grad.copy()
            q = -r
            for j in range(max_inner):
                Hq, ne = hessian_vector(g, psi, q, f_it, Vext_G, mu)
                evals += ne
                Hq = _tangent(Hq, psi)
                curv = float(np.sum(q * Hq))
                if curv <= 0.0:
                    if j == 0:
                        x = -grad
                    break
                newton = True
                a = float(np.sum(r * r)) / curv
                x = x + a * q
                r_new = r + a * Hq
                if math.sqrt(np.sum(r_new * r_new)) < stop:
                    break
                q = -r_new + (np.sum(r_new * r_new) / np.sum(r * r)) * q
                r = r_new
            if np.sum(x * grad) < 0.0:
                d = x
            else:
                d, newton = -grad, False
        else:
            # L-BFGS two-loop recursion
            if psi_prev is not None:
                s_k, y_k = psi - psi_prev, grad - g_prev
                sy = float(np.sum(s_k * y_k))
                if sy > 0.0:
                    pairs.append((s_k, y_k, 1.0 / sy))
                    if len(pairs) > lbfgs_m:
                        pairs.pop(0)
            q = grad.copy()
            alphas = []
            for s_k, y_k, rh in reversed(pairs):
                a = rh * float(np.sum(s_k * q))
                alphas.append(a)
                q = q - a * y_k
            if pairs:
                s_k, y_k, _ = pairs[-1]
                q = q * (float(np.sum(s_k * y_k)) / float(np.sum(y_k * y_k)))
            for (s_k, y_k, rh), a in zip(pairs, reversed(alphas)):
                b = rh * float(np.sum(y_k * q))
                q = q + (a - b) * s_k
            newton = bool(pairs) and np.sum(q * grad) > 0.0
            d = -q if newton else -grad
        g_prev, d_prev, psi_prev = grad, d, psi
        if update == "rotate":
            p = d - (np.sum(d * psi) / np.sum(psi * psi)) * psi
            p_len = math.sqrt(np.sum(p * p) * g.dV / n_electrons)     # |p_perp| / |psi|
            step0 = math.atan(p_len)                                 # psi + p_perp on the rotation
        else:
            p = d.copy()
            p_len = math.sqrt(np.sum(p * p) * g.dV / n_electrons)     # |d| / |psi|
            step0 = p_len                                            # psi + d at t = |d| / |psi|
        p *= math.sqrt(n_electrons / (np.sum(p * p) * g.dV))
        phi0 = E["total"]
        dphi0 = float(np.sum(grad * p))
        if dphi0 >= 0.0:
            d_prev = None
            pairs = []
            continue

        def phi(lam):
            psi_l, dpsi = update_curve(psi, p, lam, g.dV, n_electrons, update)
            E_l, V_l = energy(psi_l, f_it)
            return E_l, V_l, psi_l, float(np.sum(2.0 * psi_l * V_l * g.dV * dpsi))

        lam = min(max(step0 if newton else lam_prev, 1e-4), 0.5)
        if objective == "residual":
            # the step lowers the norm of the residual of Eq. euler2, |2 psi (V - mu) dV|:
            # backtracking from the first trial until it falls by the factor (1 - c1)
            r0 = math.sqrt(float(np.sum(grad * grad)))
            best = None
            for _ in range(max_ls):
                psi_l, _ = update_curve(psi, p, lam, g.dV, n_electrons, update)
                E_l, V_l = energy(psi_l, f_it)
                mu_l = np.sum(psi_l * psi_l * V_l) * g.dV / n_electrons
                r_l = math.sqrt(float(np.sum((2.0 * psi_l * (V_l - mu_l) * g.dV) ** 2)))
                if best is None or r_l < best[0]:
                    best = (r_l, lam, E_l, V_l, psi_l)
                if r_l <= (1.0 - c1) * r0:
                    break
                lam *= 0.5
            improved = best[0] < r0
            _, lam, E_new, V_new, psi_new = best
        else:
            improved, lam, E_new, V_new, psi_new = _wolfe_search(phi, phi0, dphi0, lam, c1, c2, max_ls)
        if not improved:
            d_prev = None            # no decrease: restart with steepest descent
            pairs = []
            psi_prev = None
            if fixed_iter is None and small >= 3:
                break
            small += 1
            continue
        lam_prev = lam
        psi = psi_new
        dE = abs(E_new["total"] - E["total"])
        E, V = E_new, V_new
        history.append(E["total"])
        f_it = frozen(psi)
        if f_it is not func:
            E, V = energy(psi, f_it)   # knots moved: re-evaluate at the new knots
        if fixed_iter is not None:
            if it >= fixed_iter:
                break
            continue
        small = small + 1 if dE < tol * n_atoms else 0
        if small >= 3:
            break
    return dict(psi=psi, E=E["total"], energies=E, iterations=it, evals=evals, history=history)


def _wolfe_search(phi, phi0, dphi0, lam, c1, c2, max_ls):
    """Strong-Wolfe search on phi(lam) = (E, V, psi, dE/dlam) (bracketing + zoom with cubic
    interpolation).  Returns (decreased, lam, E, V, psi) of the lowest trial."""
    lam_lo, f_lo, d_lo = 0.0, phi0, dphi0
    best = None
    n_ls = 0
    lam_hi = None
    while n_ls < max_ls:
        n_ls += 1
        E_l, V_l, psi_l, dl = phi(lam)
        fl = E_l["total"]
        if best is None or fl < best[0]:
            best = (fl, lam, E_l, V_l, psi_l)
        if fl > phi0 + c1 * lam * dphi0 or (lam_hi is None and fl >= f_lo and lam_lo > 0.0):
            lam_hi, f_hi, d_hi = lam, fl, dl
        elif abs(dl) <= -c2 * dphi0:
            break
        elif dl >= 0.0:
            lam_hi, f_hi, d_hi = lam_lo, f_lo, d_lo
            lam_lo, f_lo, d_lo = lam, fl, dl
        else:
            lam_lo, f_lo, d_lo = lam, fl, dl
            if lam_hi is None:
                lam = min(2.0 * lam, math.pi / 2.0)
                continue
        c = _cubic_min(lam_lo, f_lo, d_lo, lam_hi, f_hi, d_hi)
        lo, hi = min(lam_lo, lam_hi), max(lam_lo, lam_hi)
        if c is None or not (lo + 0.1 * (hi - lo) <= c <= hi - 0.1 * (hi - lo)):
            c = 0.5 * (lam_lo + lam_hi)
        lam = c
    fl, lam, E_new, V_new, psi_new = best
    return fl < phi0, lam, E_new, V_new, psi_new


def optimize_multistep(grids, psi0, func: Functional, Vext_list, n_electrons: float, n_atoms: int,
                       tol: float = 1e-6, max_iter: int = 200):
    """Sec. 2.4's multi-step scheme: psi0 (on the finest grid, grids[-1]) is carried to
    the coarsest grid, optimised there, and each converged psi is interpolated
    (oracle.interp) to the next finer grid and optimised again.  Returns the finest
    level's result dict (with 'levels': the per-level iteration counts)."""
    from .interp import fourier_interpolate
    psi = fourier_interpolate(psi0, grids[0].shape)
    levels = []
    res = None
    for li, (g, Vg) in enumerate(zip(grids, Vext_list)):
        if li > 0:
            psi = fourier_interpolate(res["psi"], g.shape)
        res = optimize_density(g, psi, func, Vg, n_electrons, n_atoms, tol=tol, max_iter=max_iter)
        levels.append(res["iterations"])
    res["levels"] = levels
    return res
