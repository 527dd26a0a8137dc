"""Generate csrc/gnl_fit.cuh: polynomial forms of the Lindhard-derived kernel G_NL for the
FP32-mixed kernels.

G_NL(eta) = 1/F(eta) - 3 eta^2 - 1, F(eta) = 1/2 + (1 - eta^2)/(4 eta) ln|(1+eta)/(1-eta)|
(Sec. 2.3, the G_NL definition below Eq. MGP) is analytic in y = eta^2 on eta < 1 and in
x = 1/eta^2 on eta > 1, its only real singularity being the kink at eta = 1 (y = x = 1).
Away from the kink it is therefore approximated to far below FP32 rounding by short
polynomials:

    eta <= 1/2:  G_NL = y * S(y),   S a polynomial of degree DS on y in [0, 1/4]
    eta >= 2  :  G_NL = L(x),       L a polynomial of degree DL on x in [0, 1/4]

each the Chebyshev interpolant (in the polynomial's variable, on [0, 1/4]) of the closed
form evaluated with 50 significant digits, converted to monomial coefficients for Horner's
rule.  The degrees are the smallest whose largest error on a dense sample of the interval
is below 2e-9 of |G_NL| (FP32 rounding is 6e-8).  Between 1/2 and 2 the kernels keep the
closed form.

Run from the repository root: python paper_2002_02985_gb300/gen_gnl_fit.py
"""
from __future__ import annotations

import os

import mpmath as mp

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "gnl_fit.cuh")
TOL = 2e-9


def gnl(eta):
    eta = mp.mpf(eta)
    F = mp.mpf(1) / 2 + (1 - eta * eta) / (4 * eta) * mp.log(abs((1 + eta) / (1 - eta)))
    return 1 / F - 3 * eta * eta - 1


def small(y):                      # S(y) = G_NL(sqrt y) / y
    return gnl(mp.sqrt(y)) / y


def large(x):                      # L(x) = G_NL(1 / sqrt x)
    return gnl(1 / mp.sqrt(x))


def cheb_monomial(f, a, b, deg):
    """Monomial coefficients c_0..c_deg (in the original variable) of the Chebyshev
    interpolant of f at deg + 1 Chebyshev points of the first kind on [a, b]."""
    n = deg + 1
    nodes = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    vals = [f((b - a) / 2 * t + (b + a) / 2) for t in nodes]
    # Chebyshev coefficients a_j = (2/n) sum_k f_k T_j(t_k)  (a_0 halved)
    cj = []
    for j in range(n):
        s = mp.fsum(vals[k] * mp.cos(j * mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n))
        cj.append(2 * s / n)
    cj[0] /= 2
    # sum_j a_j T_j(t) as a polynomial in t (T_{j+1} = 2 t T_j - T_{j-1}) ...
    poly_t = [mp.mpf(0)] * n
    Tm, T = [mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]
    for j in range(n):
        P = Tm if j == 0 else (T if j == 1 else None)
        if j >= 2:
            P = [mp.mpf(0)] * (j + 1)
            for i, c in enumerate(T):
                P[i + 1] += 2 * c
            for i, c in enumerate(Tm):
                P[i] -= c
            Tm, T = T, P
        for i, c in enumerate(P):
            poly_t[i] += cj[j] * c
    # ... then in the variable v = (b - a)/2 t + (b + a)/2, i.e. t = alpha v + beta
    alpha, beta = 2 / (b - a), -(b + a) / (b - a)
    out = [mp.mpf(0)] * n
    for i, c in enumerate(poly_t):            # c (alpha v + beta)^i
        for k in range(i + 1):
            out[k] += c * mp.binomial(i, k) * alpha ** k * beta ** (i - k)
    return out


def horner(c, v):
    p = mp.mpf(0)
    for ck in reversed(c):
        p = p * v + ck
    return p


def fit(f, scale, name):
    a, b = mp.mpf(0), mp.mpf(1) / 4
    sample = [b * (k + mp.mpf(1) / 2) / 4000 for k in range(4000)]
    for deg in range(3, 20):
        c = cheb_monomial(f, a, b, deg)
        err = max(abs(horner(c, v) - f(v)) / abs(scale(v)) for v in sample[::7])
        if err < TOL:
            err = max(abs(horner(c, v) - f(v)) / abs(scale(v)) for v in sample)
            if err < TOL:
                print(f"{name}: degree {deg}, max relative error {float(err):.2e}")
                return c, float(err)
    raise RuntimeError(name)


def main():
    cs, es = fit(small, small, "S(y)")                    # relative to |S| (G_NL = y S)
    cl, el = fit(large, large, "L(x)")
    def horner_src(c, v):
        src = f"{float(c[-1]):.9e}f"
        for ck in reversed(c[:-1]):
            src = f"fmaf({src}, {v}, {float(ck):.9e}f)"
        return src
    text = f"""// Generated by gen_gnl_fit.py (do not edit): polynomial forms of the kernel G_NL of
// Sec. 2.3 for the FP32-mixed kernels.  eta <= 1/2: G_NL = y S(y), y = eta^2; eta >= 2:
// G_NL = L(x), x = 1/eta^2; S (degree {len(cs) - 1}) and L (degree {len(cl) - 1}) are Chebyshev
// interpolants on [0, 1/4] of the closed form (largest relative error {es:.1e} and {el:.1e},
// below FP32 rounding), evaluated by Horner's rule.
#pragma once

namespace ofdft {{
__device__ __forceinline__ float gnl_small_s(float y) {{
    return {horner_src(cs, "y")};
}}
__device__ __forceinline__ float gnl_large_l(float x) {{
    return {horner_src(cl, "x")};
}}
}}  // namespace ofdft
"""
    with open(OUT, "w") as fh:
        fh.write(text)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
