"""GPU smooth-PME structure factor and forces against the oracle's PME (same
approximation: tight) and against the direct structure factor (order 12)."""
import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn, pme as opme
from oracle.evaluate import Functional as OFunc, evaluate
from oracle.grid import Grid as OGrid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402


def case():
    cell = np.array([[9.2, 0.0, 0.0], [0.6, 8.8, 0.0], [-0.4, 0.7, 10.1]])
    shape = (40, 36, 48)
    rng = np.random.default_rng(21)
    pos = rng.uniform(0, 1, (7, 3)) @ cell
    species = np.array([0, 1, 0, 1, 1, 0, 0], np.int32)
    Z, rc = [3.0, 2.0], [0.8, 1.0]
    q = np.array([Z[s] for s in species])
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, q, 1.0) + 1e-3, 0.05, 3), cell, q.sum())
    return cell, shape, pos, species, Z, rc, rho


@pytest.mark.parametrize("precision,order", [(L.FP64, 8), (L.FP32_MIXED, 8), (L.FP64, 12)])
def test_pme_energy_and_forces_match_oracle_pme(precision, order):
    cell, shape, pos, species, Z, rc, rho = case()
    dt = torch.float64 if precision == L.FP64 else torch.float32
    rin = rho if precision == L.FP64 else rho.astype(np.float32).astype(np.float64)
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, species, Z, rc, pme_order=order)
    f = ofd.Functional(n_knots=6, precision=precision)
    r = torch.from_numpy(rin).to("cuda", dt).contiguous()
    E, V = g.energy_potential(r, f)
    F = g.forces(r, precision)
    og = OGrid(cell, shape)
    Vg = opme.external_potential_G(og, pos, species, Z, rc, order)
    Eo, Vo = evaluate(og, rin, OFunc(n_knots=6), Vg)
    Fo = opme.forces(og, rin, pos, species, Z, rc, order)
    if precision == L.FP64:
        assert abs(E["PP"] - Eo["PP"]) <= 1e-10 * abs(Eo["PP"])
        assert abs(E["total"] - Eo["total"]) <= 1e-10 * abs(Eo["total"])
        assert np.max(np.abs(V.cpu().numpy() - Vo)) <= 1e-9 * np.max(np.abs(Vo))
        assert np.max(np.abs(F - Fo)) <= 1e-9 * max(1.0, np.max(np.abs(Fo)))
    else:
        assert abs(E["PP"] - Eo["PP"]) / len(pos) <= 1e-6
        assert abs(E["total"] - Eo["total"]) / len(pos) <= 1e-6
        assert np.max(np.abs(F - Fo)) <= 2e-5 * max(1.0, np.max(np.abs(Fo)))


def test_pme_order12_matches_direct_structure_factor_on_gpu():
    cell, shape, pos, species, Z, rc, rho = case()
    r = torch.from_numpy(rho).cuda()
    f = ofd.Functional(n_knots=6, precision=L.FP64)
    g1 = ofd.Grid(cell, shape)
    g1.set_ions(pos, species, Z, rc)
    g2 = ofd.Grid(cell, shape)
    g2.set_ions(pos, species, Z, rc, pme_order=12)
    E1, _ = g1.energy_potential(r, f)
    E2, _ = g2.energy_potential(r, f)
    assert abs(E1["PP"] - E2["PP"]) <= 1e-9 * abs(E1["PP"])
    F1, F2 = g1.forces(r, L.FP64), g2.forces(r, L.FP64)
    assert np.max(np.abs(F1 - F2)) <= 1e-7 * max(1.0, np.max(np.abs(F1)))


def test_pme_charge_grid_is_bit_reproducible():
    cell, shape, pos, species, Z, rc, rho = case()
    r = torch.from_numpy(rho.astype(np.float32)).cuda()
    out = []
    for _ in range(2):
        g = ofd.Grid(cell, shape)
        g.set_ions(pos, species, Z, rc, pme_order=8)
        out.append(g.energy_potential(r, ofd.Functional(n_knots=6))[0])
    assert out[0] == out[1]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("precision", [L.FP64, L.FP32_MIXED])
def test_pme_long_axis_supercell_matches_the_cell(axis, precision):
    """A 4-atom FCC cell repeated 64 times along one axis (1024 points there, 16 on the others):
    the PME structure factor runs one-channel transforms of length 1024 along that axis, and
    the perfect supercell's energy per atom equals that of the cell (oracle, direct S(G))."""
    wl1 = W.workload("fcc-al-4/16")
    reps = [1, 1, 1]
    reps[axis] = 64
    cell = np.diag([wl1["cell"][a][a] * reps[a] for a in range(3)])
    shape = tuple(16 * r for r in reps)
    ijk = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    pos = (ijk[:, None, :] * np.diag(wl1["cell"])[None, None, :] + wl1["positions"][None]).reshape(-1, 3)
    r1 = W.model_density(wl1)
    rho = np.tile(r1, reps)
    dt = torch.float64 if precision == L.FP64 else torch.float32
    if precision == L.FP32_MIXED:
        r1 = r1.astype(np.float32).astype(np.float64)
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, np.zeros(len(pos), np.int32), wl1["Z"], wl1["rc"], pme_order=10)
    E, V = g.energy_potential(torch.from_numpy(rho).to("cuda", dt).contiguous(),
                              ofd.Functional(n_knots=12, precision=precision))
    og = OGrid(wl1["cell"], wl1["shape"])
    Vg = ofn.external_potential_G(og, wl1["positions"], wl1["species"], wl1["Z"], wl1["rc"])
    E1, _ = evaluate(og, r1, OFunc(n_knots=12), Vg)
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] / len(pos) - E1[k] / 4) <= 1e-6, (k, E[k] / len(pos), E1[k] / 4)
