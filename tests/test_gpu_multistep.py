"""GPU Fourier interpolation between grids and the multi-step optimisation (Sec. 2.4)
against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn
from oracle.evaluate import Functional as OFunc
from oracle.grid import Grid as OGrid
from oracle.interp import fourier_interpolate
from oracle.optimize import optimize_density as ooptimize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402

CELL = np.array([[6.0, 0.0, 0.0], [0.8, 5.5, 0.0], [-0.5, 0.4, 7.0]])


@pytest.mark.parametrize("small,big", [((12, 10, 16), (24, 20, 32)), ((9, 15, 10), (18, 30, 20)),
                                       ((16, 16, 16), (32, 32, 32))])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
def test_interpolation_matches_oracle(small, big, dtype, tol):
    rng = np.random.default_rng(sum(small))
    fs = 0.5 + rng.random(small)
    fb = 0.5 + rng.random(big)
    gs, gb = ofd.Grid(CELL, small), ofd.Grid(CELL, big)
    up = gs.interpolate(torch.from_numpy(fs).to("cuda", dtype), gb).double().cpu().numpy()
    down = gb.interpolate(torch.from_numpy(fb).to("cuda", dtype), gs).double().cpu().numpy()
    fs_in = fs.astype(np.float32).astype(np.float64) if dtype == torch.float32 else fs
    fb_in = fb.astype(np.float32).astype(np.float64) if dtype == torch.float32 else fb
    assert np.max(np.abs(up - fourier_interpolate(fs_in, big))) <= tol * np.max(np.abs(fs))
    assert np.max(np.abs(down - fourier_interpolate(fb_in, small))) <= tol * np.max(np.abs(fb))


@pytest.fixture(scope="module")
def fine_optimum():
    """Oracle minimum on 32^3 with the knots frozen at the starting density's."""
    wl = W.workload("fcc-al-4/32")
    rho = W.model_density(wl)
    og = OGrid(wl["cell"], wl["shape"])
    Vg = ofn.external_potential_G(og, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    knots = ofn.make_knots(rho, wl["n_knots"])
    res = ooptimize(og, np.sqrt(rho), OFunc(n_knots=wl["n_knots"], knots=knots), Vg, wl["n_electrons"],
                    wl["n_atoms"], tol=1e-12, max_iter=400)
    return wl, rho, knots, res


@pytest.mark.parametrize("precision,tol", [(L.FP64, 1e-8), (L.FP32_MIXED, 1e-6)])
def test_multistep_reaches_the_fine_minimum(fine_optimum, precision, tol):
    wl, rho, knots, ores = fine_optimum
    dt = torch.float64 if precision == L.FP64 else torch.float32
    grids = []
    for shape in ((16, 16, 16), wl["shape"]):
        g = ofd.Grid(wl["cell"], shape)
        g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
        grids.append(g)
    f = ofd.Functional(n_knots=wl["n_knots"], knots=knots, precision=precision)
    psi = torch.from_numpy(np.sqrt(rho)).to("cuda", dt).contiguous()
    rep = ofd.optimize_density_multistep(grids, psi, f, wl["n_electrons"],
                                         tol_per_atom=1e-12 if precision == L.FP64 else 1e-7, max_iter=400)
    assert abs(rep["energy"] - ores["E"]) / wl["n_atoms"] <= tol, (rep["energy"], ores["E"], rep)
    charge = float((psi.double() ** 2).sum()) * grids[-1].dV
    assert abs(charge - wl["n_electrons"]) <= (1e-10 if precision == L.FP64 else 1e-6) * wl["n_electrons"]
