"""Total energy and potential of the oracle (test infrastructure only).

E[rho] = T_TF + T_vW + T_NL + E_H + E_PP (+ E_xc)   (Eq. efunc)
V      = dE/drho                                     (Eq. euler)
E_xc (LDA, Perdew-Zunger) is included when "XC" is among the terms.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import functionals as fn
from . import xc as fxc
from .grid import Grid

TERMS_ALL = ("TF", "VW", "NL", "HARTREE", "PP")


@dataclass
class Functional:
    """Which terms to evaluate and how (mirrors the library's functional record)."""
    terms: tuple = TERMS_ALL
    alpha: float = 5.0 / 6.0
    beta: float = 5.0 / 6.0
    n_knots: int = 10
    spacing: str = "log"              # 'log' | 'arith'
    knots: np.ndarray | None = None   # frozen knots (e.g. for finite differences)
    potential: str = "exact"          # 'exact' | 'interpolated'
    kernel: str = "lwt"               # 'lwt' | 'wt_global'
    mgp_x: float = 0.0                # Eq. MGP's (x, y): x = 0 is Wang-Teter; (1, 5/6) MGP,
    mgp_y: float = 5.0 / 6.0          # (1/2, 5/6) MGPA, (1, 5/3) MGPG
    extra: dict = field(default_factory=dict)


def evaluate(g: Grid, rho, func: Functional, Vext_G=None):
    """Returns (energies dict with keys total, TF, vW, NL, H, PP, XC;  V on the grid)."""
    rho = np.asarray(rho, dtype=np.float64)
    E = dict(TF=0.0, vW=0.0, NL=0.0, H=0.0, PP=0.0, XC=0.0)
    V = np.zeros_like(rho)
    if "TF" in func.terms:
        e, v = fn.thomas_fermi(g, rho)
        E["TF"] = e
        V += v
    if "VW" in func.terms:
        e, v = fn.von_weizsaecker(g, rho)
        E["vW"] = e
        V += v
    if "NL" in func.terms:
        if func.kernel == "wt_global":
            e, v = fn.nonlocal_wt_global(g, rho, func.alpha, func.beta, mgp=(func.mgp_x, func.mgp_y))
        else:
            knots = func.knots if func.knots is not None else fn.make_knots(rho, func.n_knots, func.spacing)
            e, v = fn.nonlocal_lwt(g, rho, np.asarray(knots, dtype=np.float64), func.alpha, func.beta,
                                   func.potential, mgp=(func.mgp_x, func.mgp_y))
        E["NL"] = e
        V += v
    if "HARTREE" in func.terms:
        e, v = fn.hartree(g, rho)
        E["H"] = e
        V += v
    if "PP" in func.terms and Vext_G is not None:
        e, v = fn.local_pseudopotential(g, rho, Vext_G)
        E["PP"] = e
        V += v
    if "XC" in func.terms:
        e, v = fxc.lda_xc(g, rho)
        E["XC"] = e
        V += v
    E["total"] = E["TF"] + E["vW"] + E["NL"] + E["H"] + E["PP"] + E["XC"]
    return E, V
