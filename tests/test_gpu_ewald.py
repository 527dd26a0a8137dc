"""GPU ion-ion Ewald energy and forces (FP64, through the C ABI) against the oracle's
Ewald sum, which uses its own split parameter and its own G and image sums."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.ewald import ewald as oewald

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402

FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def _random_case():
    rng = np.random.default_rng(11)
    cell = np.array([[6.5, 0.0, 0.0], [1.2, 5.8, 0.0], [-0.9, 0.7, 6.9]])
    pos = rng.uniform(0, 1, (7, 3)) @ cell
    species = np.array([0, 1, 2, 0, 1, 0, 2], np.int32)
    Z = (3.0, 2.0, 1.0)
    return cell, pos, species, Z


def _gpu(cell, shape, pos, species, Z, pme_order=0):
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, species, Z, tuple(0.8 for _ in Z), pme_order=pme_order)
    return g.ewald()


def test_ewald_matches_oracle():
    cell, pos, species, Z = _random_case()
    E, F = _gpu(cell, (24, 20, 27), pos, species, Z)
    Eo, Fo = oewald(cell, pos, np.asarray(Z)[species])
    assert abs(E - Eo) <= 1e-10 * abs(Eo), (E, Eo)
    assert np.max(np.abs(F - Fo)) <= 1e-9 * np.max(np.abs(Fo))


def test_ewald_fcc_and_rock_salt_lattice_sums():
    """FCC Al (Z = 3) in its background: E per ion = -0.895873615195 Z^2 / r_s; rock
    salt with charges +-1: E per ion pair = -1.747564594633 / d."""
    a = 7.65
    E, F = _gpu(np.eye(3) * a, (32, 32, 32), FCC * a, np.zeros(4, np.int32), (3.0,))
    rs = a * (3.0 / (16.0 * math.pi)) ** (1.0 / 3.0)
    assert abs(E / 4 * rs / 9.0 - (-0.895873615195)) < 1e-10
    assert np.max(np.abs(F)) < 1e-9
    R = np.vstack([FCC, FCC + [0.5, 0.0, 0.0]]) * a
    E, F = _gpu(np.eye(3) * a, (30, 30, 30), R, np.array([0] * 4 + [1] * 4, np.int32), (1.0, -1.0))
    assert abs(-E / 4 * (0.5 * a) - 1.747564594633) < 1e-10
    assert np.max(np.abs(F)) < 1e-9


def test_ewald_with_pme_structure_factor():
    cell, pos, species, Z = _random_case()
    E, F = _gpu(cell, (24, 20, 27), pos, species, Z, pme_order=12)
    Eo, Fo = oewald(cell, pos, np.asarray(Z)[species])
    assert abs(E - Eo) <= 1e-8 * abs(Eo), (E, Eo)
    assert np.max(np.abs(F - Fo)) <= 1e-6 * np.max(np.abs(Fo))


def test_ewald_256_atom_workload():
    wl = W.workload("fcc-al-256/128")
    rng = np.random.default_rng(3)
    pos = wl["positions"] + rng.normal(0.0, 0.1, wl["positions"].shape)
    E, F = _gpu(wl["cell"], wl["shape"], pos, wl["species"], tuple(wl["Z"]))
    Eo, Fo = oewald(wl["cell"], pos, np.asarray(wl["Z"])[wl["species"]])
    assert abs(E - Eo) <= 1e-10 * abs(Eo), (E, Eo)
    assert np.max(np.abs(F - Fo)) <= 1e-9 * np.max(np.abs(Fo))
