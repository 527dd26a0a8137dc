"""Fourier interpolation of a real periodic field between two grids of one cell
(test infrastructure only).

Sec. 2.4's multi-step optimisation converges the density on a coarse grid and
carries it to a finer one.  The oracle's reading of "interpolate": the unique
band-limited (trigonometric) interpolant.  With the normalised transform
f_hat(m) = (1/N) sum_r f(r) e^{-2 pi i m.r/n}, the coefficients of every
frequency present on both grids are copied; on the way up, a Nyquist coefficient
of the smaller grid (m_a = n_a/2, even n_a) stands for the cosine at that
frequency and is shared equally between +n_a/2 and -n_a/2 of the larger grid (so
the interpolant passes through the coarse samples); on the way down the two
become one again (their sum) and everything beyond is dropped.
"""
from __future__ import annotations

import numpy as np


def _axis_map(n_from: int, n_to: int):
    """(index_from, index_to, weight) triples for one full (complex) axis."""
    out = []
    small = min(n_from, n_to)
    for m in range(-(small // 2), small // 2 + 1):
        if small % 2 == 0 and abs(m) == small // 2:
            if m < 0:
                continue
            if n_to > n_from:            # split the smaller grid's Nyquist term
                out.append((m % n_from, m % n_to, 0.5))
                out.append((m % n_from, (-m) % n_to, 0.5))
            elif n_to < n_from:          # fold both signs into the Nyquist term
                out.append((m % n_from, m % n_to, 1.0))
                out.append(((-m) % n_from, m % n_to, 1.0))
            else:
                out.append((m % n_from, m % n_to, 1.0))
        else:
            out.append((m % n_from, m % n_to, 1.0))
    return out


def fourier_interpolate(field, shape_to):
    """Band-limited interpolant of `field` (real, periodic) sampled on `shape_to`."""
    f = np.asarray(field, dtype=np.float64)
    n_from, n_to = f.shape, tuple(shape_to)
    F = np.fft.fftn(f) / f.size                      # full complex spectrum, normalised
    T = np.zeros(n_to, dtype=np.complex128)
    maps = [_axis_map(n_from[a], n_to[a]) for a in range(3)]
    for i0, j0, w0 in maps[0]:
        for i1, j1, w1 in maps[1]:
            for i2, j2, w2 in maps[2]:
                T[j0, j1, j2] += w0 * w1 * w2 * F[i0, i1, i2]
    return np.real(np.fft.ifftn(T) * np.prod(n_to))
