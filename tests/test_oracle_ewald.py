"""Pins of the oracle's Ewald ion-ion energy and forces against tabulated lattice
sums (Madelung constants) and exact properties of the Ewald split."""
import math

import numpy as np
import pytest

from oracle.ewald import ewald

FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
ALPHA_SC = 2.837297479480619        # simple-cubic jellium constant, pinned in test_oracle_pins


def test_rock_salt_madelung_constant():
    """NaCl, charges +-1, nearest-neighbour distance d: E per ion pair = -1.747564594633 / d."""
    R = np.vstack([FCC, FCC + [0.5, 0.0, 0.0]])
    Z = np.array([1.0] * 4 + [-1.0] * 4)
    E, F = ewald(np.eye(3), R, Z)
    assert abs(-E / 4 * 0.5 - 1.747564594633) < 1e-11
    assert np.max(np.abs(F)) < 1e-12


def test_caesium_chloride_madelung_constant():
    """CsCl, d = sqrt(3)/2 a: E per ion pair = -1.762674773071 / d."""
    E, _ = ewald(np.eye(3), np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]), np.array([1.0, -1.0]))
    assert abs(-E * math.sqrt(3.0) / 2.0 - 1.762674773071) < 1e-11


@pytest.mark.parametrize("name,pos,value", [
    ("sc", np.zeros((1, 3)), -ALPHA_SC / 2.0 * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)),
    ("bcc", np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]), -0.895929255682),
    ("fcc", FCC, -0.895873615195),
])
def test_jellium_lattice_energies(name, pos, value):
    """Point charges in a neutralising background: E per ion = value Z^2 / r_s
    (Wigner-Seitz radius r_s); BCC and FCC constants of Coldwell-Horsfall and
    Maradudin (1960), SC from the simple-cubic constant."""
    n = len(pos)
    for a, Zv in ((1.0, 1.0), (7.65, 3.0)):
        E, F = ewald(np.eye(3) * a, pos * a, np.full(n, Zv))
        rs = a * (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
        assert abs(E / n * rs / Zv ** 2 - value) < 1e-11
        assert np.max(np.abs(F)) < 1e-11 * Zv ** 2


def _random_case():
    rng = np.random.default_rng(7)
    cell = np.array([[6.5, 0.0, 0.0], [1.2, 5.8, 0.0], [-0.9, 0.7, 6.9]])
    pos = rng.uniform(0, 1, (5, 3)) @ cell
    Z = np.array([3.0, 3.0, 2.0, 1.0, 3.0])
    return cell, pos, Z


def test_energy_and_forces_do_not_depend_on_the_split():
    cell, pos, Z = _random_case()
    E1, F1 = ewald(cell, pos, Z, eta=0.6)
    E2, F2 = ewald(cell, pos, Z, eta=1.4)
    assert abs(E1 - E2) < 1e-12 * abs(E1)
    assert np.max(np.abs(F1 - F2)) < 1e-11 * np.max(np.abs(F1))


def test_forces_are_minus_the_energy_gradient_and_sum_to_zero():
    cell, pos, Z = _random_case()
    E, F = ewald(cell, pos, Z)
    h = 1e-5
    for I, a in [(0, 0), (2, 1), (4, 2), (1, 2)]:
        Es = []
        for sgn in (1, -1):
            p = pos.copy()
            p[I, a] += sgn * h
            Es.append(ewald(cell, p, Z)[0])
        assert abs(-(Es[0] - Es[1]) / (2 * h) - F[I, a]) < 1e-7 * max(1.0, abs(F[I, a]))
    assert np.max(np.abs(F.sum(axis=0))) < 1e-11 * np.max(np.abs(F))


def test_translation_and_lattice_shift_invariance():
    cell, pos, Z = _random_case()
    E0, F0 = ewald(cell, pos, Z)
    E1, F1 = ewald(cell, pos + np.array([0.37, -1.1, 2.3]), Z)
    p2 = pos.copy()
    p2[3] += cell[0] - 2 * cell[2]
    E2, F2 = ewald(cell, p2, Z)
    assert abs(E1 - E0) < 1e-12 * abs(E0) and abs(E2 - E0) < 1e-12 * abs(E0)
    assert np.max(np.abs(F1 - F0)) < 1e-11 * np.max(np.abs(F0))
    assert np.max(np.abs(F2 - F0)) < 1e-11 * np.max(np.abs(F0))
