"""GPU parity at the benchmark's own workloads and launch configurations.

The bench times FP32-mixed evaluations of fcc-al-256/128 (16 knots), mg147/192
(30 knots) and fcc-al-1m/1024 (12 knots, PME order 10).  These tests put each of
those configurations, with the kernels the bench launches, against the FP64
oracle (Sec. 2.3 s1-s4; Eqs. efunc, euler):

  energies : every term within 1e-6 Ha/atom;
  potential: ||dV||_2 / ||V||_2 <= 1e-4 away from points whose kF is within 1e-5
             (relative) of a knot (there the spline interval is a floating-point
             decision each side takes in its own precision).

The 1024^3 grid is too large for the oracle; it is pinned by supercell invariance
instead: a noise-free perfect crystal of 64^3 conventional cells has exactly the
period of one cell, so its energy per atom and its potential equal those of the
4-atom cell on a 16^3 grid (same knots: same min/max density), which the oracle
computes.
"""
import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn
from oracle.evaluate import Functional as OFunc, evaluate
from oracle.grid import Grid as OGrid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402


def _near_knot_mask(rho, n_knots, rtol=1e-5):
    """Points whose kF is not within rtol of an interior knot.  (The end knots are kF of the
    minimum and maximum density; the knot-range decision is taken on the density itself,
    identically in both precisions, so the floored vacuum of a cluster, all at the first
    knot, is compared too.)"""
    k = ofn.make_knots(rho, n_knots)[1:-1]
    kF = ofn.fermi_wavevector(rho)
    # nearest knot per point without an [N, M] temporary
    d = np.full(rho.shape, np.inf)
    for kk in k:
        d = np.minimum(d, np.abs(kF / kk - 1.0))
    return d > rtol


def _gpu_and_oracle(wl, kw):
    rho32 = W.model_density(wl).astype(np.float32)
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
    f = ofd.Functional(n_knots=wl["n_knots"], precision=L.FP32_MIXED, **kw)
    E, V = g.energy_potential(torch.from_numpy(rho32).cuda(), f)
    V = V.double().cpu().numpy()
    og = OGrid(wl["cell"], wl["shape"])
    Vg = ofn.external_potential_G(og, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    pot = "exact" if kw.get("nl_potential", L.NLPOT_EXACT) == L.NLPOT_EXACT else "interpolated"
    Eo, Vo = evaluate(og, rho32.astype(np.float64), OFunc(n_knots=wl["n_knots"], potential=pot), Vg)
    return rho32.astype(np.float64), E, V, Eo, Vo


def _check(wl, rho, E, V, Eo, Vo, rho_min=0.0):
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] - Eo[k]) / wl["n_atoms"] <= 1e-6, (k, E[k], Eo[k])
    m = _near_knot_mask(rho, wl["n_knots"])
    assert m.mean() > 0.999
    # the potential as the optimiser uses it, in the gradient 2 psi V dV: psi-weighted
    w = np.sqrt(rho)
    relw = np.linalg.norm((w * (V - Vo))[m]) / np.linalg.norm((w * Vo)[m])
    assert relw <= 1e-4, relw
    m &= rho >= rho_min
    rel = np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m])
    assert rel <= 1e-4, rel
    return relw, rel


@pytest.mark.parametrize("kw", [dict(), dict(nl_potential=L.NLPOT_INTERP)])
def test_bench_workload_fcc_al_256_128_matches_oracle(kw):
    """The headline configuration: 128^3 on every axis (row, n1-pencil and reciprocal-space
    kernels specialised for 128 points), 16 knots, FP32-mixed."""
    wl = W.workload("fcc-al-256/128")
    _check(wl, *_gpu_and_oracle(wl, kw))


def test_cluster_mg147_192_matches_oracle():
    """The isolated-cluster configuration: 192^3, 30 knots, density spanning 1e-8..0.05.
    Every energy term within 1e-6 Ha/atom; the potential psi-weighted over the whole grid (the
    optimiser's gradient 2 psi V dV) and unweighted where rho >= 1e-3 (43 % of the points,
    99.1 % of the charge).  In the tail the von Weizsaecker
    potential -lap(psi)/(2 psi) divides the FP32 noise floor of the spectral Laplacian (about
    1e-7 of the field times G_max^2) by psi: 4e-4 relative where rho >= 1e-6, 5e-3 Ha at
    rho = 1e-6, where V carries no weight in any energy or gradient."""
    wl = W.workload("mg147/192")
    _check(wl, *_gpu_and_oracle(wl, {}), rho_min=1e-3)


def test_supercell_1024_matches_the_cell_oracle():
    """1,048,576 atoms on 1024^3 (12 knots, PME order 10 as in the bench) against the
    4-atom cell on 16^3: energy per atom and the potential of three 16^3 blocks."""
    wl = W.workload("fcc-al-1m/1024")
    wl1 = W.workload("fcc-al-4/16")
    dev = torch.device("cuda", 0)
    rho = W.tiled_density_torch(wl1, 64, 0.0, 5, dev, torch.float32)
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"], pme_order=10)
    E, V = g.energy_potential(rho, ofd.Functional(n_knots=12, precision=L.FP32_MIXED))
    og = OGrid(wl1["cell"], wl1["shape"])
    Vg = ofn.external_potential_G(og, wl1["positions"], wl1["species"], wl1["Z"], wl1["rc"])
    r1 = W.model_density(wl1).astype(np.float32).astype(np.float64)
    E1, V1 = evaluate(og, r1, OFunc(n_knots=12), Vg)
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] / wl["n_atoms"] - E1[k] / 4) <= 1e-6, (k, E[k] / wl["n_atoms"], E1[k] / 4)
    m = _near_knot_mask(r1, 12)
    for a, b, c in ((0, 0, 0), (512, 256, 768), (1008, 1008, 1008)):
        blk = V[a:a + 16, b:b + 16, c:c + 16].double().cpu().numpy()
        rel = np.linalg.norm((blk - V1)[m]) / np.linalg.norm(V1[m])
        assert rel <= 1e-4, (a, b, c, rel)
    del V, rho
    torch.cuda.empty_cache()
