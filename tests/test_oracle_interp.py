"""Pins of the oracle's Fourier interpolation between grids (multi-step optimisation)."""
import numpy as np
import pytest

from oracle.interp import fourier_interpolate


def _plane_waves(shape, modes, phase=0.3):
    idx = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    f = np.full(shape, 0.7)
    for amp, m in modes:
        f += amp * np.cos(2 * np.pi * (m[0] * idx[0] + m[1] * idx[1] + m[2] * idx[2]) + phase)
    return f


MODES = [(0.4, (1, 0, 2)), (-0.25, (3, -2, 1)), (0.1, (-2, 3, -3))]


@pytest.mark.parametrize("small,big", [((8, 10, 12), (16, 20, 24)), ((9, 10, 15), (18, 25, 30))])
def test_band_limited_fields_interpolate_exactly(small, big):
    """A field whose frequencies lie inside both grids is reproduced exactly both ways."""
    fs, fb = _plane_waves(small, MODES), _plane_waves(big, MODES)
    assert np.max(np.abs(fourier_interpolate(fs, big) - fb)) < 1e-12
    assert np.max(np.abs(fourier_interpolate(fb, small) - fs)) < 1e-12


def test_interpolant_passes_through_the_coarse_samples():
    """Any coarse field (Nyquist terms included) is reproduced at the coarse points of the
    fine grid, and going back down returns it unchanged."""
    rng = np.random.default_rng(4)
    fc = rng.standard_normal((8, 6, 10))
    ff = fourier_interpolate(fc, (16, 12, 20))
    assert np.max(np.abs(ff[::2, ::2, ::2] - fc)) < 1e-12
    assert np.max(np.abs(fourier_interpolate(ff, (8, 6, 10)) - fc)) < 1e-12


def test_mean_is_preserved():
    rng = np.random.default_rng(5)
    f = rng.random((12, 9, 10))
    assert abs(fourier_interpolate(f, (24, 18, 20)).mean() - f.mean()) < 1e-14
    assert abs(fourier_interpolate(f, (6, 9, 5)).mean() - f.mean()) < 1e-14
