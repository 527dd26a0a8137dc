"""Grid conventions of the oracle (test infrastructure only).

Follows the paper's Grid/Field description (Sec. 2.1 "DFTpy classes"):
a periodic cell with lattice vectors a_i (rows of `cell`, bohr) sampled on
n0 x n1 x n2 points, C order (n2 fastest).  Fourier coefficients use

    f_hat(G) = (1/N) sum_r f(r) exp(-i G.r),      f(r) = sum_G f_hat(G) exp(i G.r)

stored as the half spectrum n0 x n1 x (n2//2 + 1) of a real field.  The
integer frequency of index k along an axis of n points is k if k <= n/2,
else k - n (the Nyquist index keeps +n/2), and G = 2 pi (m0 b0 + m1 b1 + m2 b2)
with b = rows of inv(cell)^T.  A sum over the full set of G of a quantity
with Hermitian symmetry is the half-spectrum sum with weights w = 1 on the
k2 = 0 and k2 = n2/2 planes and 2 elsewhere.
"""
from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, cell, shape):
        self.cell = np.asarray(cell, dtype=np.float64).reshape(3, 3)
        self.shape = tuple(int(n) for n in shape)
        self.N = int(np.prod(self.shape))
        self.omega = abs(float(np.linalg.det(self.cell)))
        self.dV = self.omega / self.N
        self.recip = np.linalg.inv(self.cell).T          # rows b_i, a_i . b_j = delta_ij
        n0, n1, n2 = self.shape
        m = [self.int_freq(n0), self.int_freq(n1), np.arange(n2 // 2 + 1, dtype=np.float64)]
        mm = np.meshgrid(*m, indexing="ij")
        self.G = 2.0 * np.pi * (mm[0][..., None] * self.recip[0] + mm[1][..., None] * self.recip[1]
                                + mm[2][..., None] * self.recip[2])          # (n0, n1, n2h, 3)
        self.G2 = (self.G ** 2).sum(-1)
        self.Gnorm = np.sqrt(self.G2)
        w = np.full(self.G2.shape, 2.0)
        w[..., 0] = 1.0
        if n2 % 2 == 0:
            w[..., n2 // 2] = 1.0
        self.weights = w

    @staticmethod
    def int_freq(n: int) -> np.ndarray:
        k = np.arange(n, dtype=np.float64)
        return np.where(k <= n / 2.0, k, k - n)

    def points(self) -> np.ndarray:
        """Cartesian coordinates of all grid points, (n0, n1, n2, 3)."""
        f = np.meshgrid(*[np.arange(n) / n for n in self.shape], indexing="ij")
        return np.stack(f, -1) @ self.cell

    def fft(self, f: np.ndarray) -> np.ndarray:
        """f_hat on the half spectrum, normalised by 1/N."""
        return np.fft.rfftn(f) / self.N

    def ifft(self, F: np.ndarray) -> np.ndarray:
        """Real field sum_G F(G) e^{iG.r} from its half spectrum (inverse of `fft`)."""
        return np.fft.irfftn(F, s=self.shape, axes=(0, 1, 2)) * self.N

    def gsum(self, q: np.ndarray) -> float:
        """Sum over the full G set of a Hermitian-symmetric quantity given on the half spectrum."""
        return float((self.weights * q).sum())
