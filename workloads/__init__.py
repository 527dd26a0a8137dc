"""Seeded synthetic inputs for the OFDFT energy/potential path.

This module is shared by the oracle tests, the GPU tests and the benchmark.
It builds ionic structures, a counter-based noise stream and Gaussian model
densities.  It holds none of the method's arithmetic (no functional, FFT
convention, kernel or potential): it only produces the inputs both sides read.

Every workload stands in for the paper's BLPS-based Al/Mg systems (Sec. 3,
"Applications"), which need pseudopotential files that are not available:
ions carry an analytic local pseudopotential with charge Z and core radius rc,
and the density is a sum of atom-centred Gaussians with multiplicative noise.
"""
from __future__ import annotations

import math

import numpy as np

A_AL = 7.65          # bohr, conventional FCC cell edge (a = 4.05 Angstrom)
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_uniform(seed: int, idx: np.ndarray) -> np.ndarray:
    """Uniform [0,1) numbers u_i = mix(seed + (i+1)*gamma) >> 11 * 2^-53.

    This is the i-th output of Steele, Lea & Flood's SplitMix64 generator
    (OOPSLA 2014) seeded with `seed`, so any position of the stream can be
    produced without the others (a GPU kernel can regenerate it in place).
    """
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + (idx + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _lsr(z, s: int):
    """Logical right shift of int64 tensors (torch shifts arithmetically)."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def splitmix64_uniform_torch(seed: int, start: int, count: int, device):
    """The same stream as splitmix64_uniform for indices start .. start+count-1, computed
    with wrapping int64 tensor arithmetic on `device` (so a GPU can regenerate the noise
    of a 1024^3 grid without a host transfer)."""
    import torch
    idx = torch.arange(start, start + count, dtype=torch.int64, device=device)
    z = _i64(seed & _MASK64) + (idx + 1) * _i64(_GAMMA)
    z = (z ^ _lsr(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _i64(0x94D049BB133111EB)
    z = z ^ _lsr(z, 31)
    return _lsr(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def tiled_density_torch(wl_cell: dict, reps: int, noise: float, seed: int, device, dtype):
    """Density of a reps^3 supercell of a periodic unit cell: the unit cell's model
    density tiled, then the multiplicative SplitMix64 noise of the full grid (flat C
    index), then renormalised to reps^3 times the cell's electrons.  Built plane by
    plane on `device` in FP64, returned in `dtype`."""
    import torch
    rho1 = torch.from_numpy(model_density(wl_cell)).to(device)
    n = rho1.shape[0]
    Nn = n * reps
    out = torch.empty((Nn, Nn, Nn), dtype=dtype, device=device)
    plane = rho1.repeat(1, reps, reps)                       # (n, Nn, Nn) block of n planes
    total = 0.0
    for i0 in range(Nn):
        p = plane[i0 % n]
        if noise:
            u = splitmix64_uniform_torch(seed, i0 * Nn * Nn, Nn * Nn, device).view(Nn, Nn)
            p = p * (1.0 + noise * (2.0 * u - 1.0))
        total += float(p.sum())
        out[i0] = p.to(dtype)
    omega = abs(float(np.linalg.det(wl_cell["cell"]))) * reps ** 3
    scale = wl_cell["n_electrons"] * reps ** 3 / (total * omega / Nn ** 3)
    out.mul_(scale)
    return out


def fcc_positions(n_cells, a: float = A_AL) -> tuple[np.ndarray, np.ndarray]:
    """Cubic FCC supercell of n_cells (int or 3-tuple) conventional cells.

    Returns (cell [3x3, rows = lattice vectors, bohr], positions [n,3] bohr)."""
    nc = np.broadcast_to(np.asarray(n_cells, dtype=int), (3,))
    ijk = np.stack(np.meshgrid(*[np.arange(n) for n in nc], indexing="ij"), -1).reshape(-1, 3)
    frac = (ijk[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3)
    cell = np.diag(nc * a).astype(np.float64)
    return cell, frac * a


def mackay_icosahedron(n_shells: int = 3, nn: float = 6.0) -> np.ndarray:
    """Mackay icosahedron with 1 + sum_k (10 k^2 + 2) atoms (147 for 3 shells).

    Shell k has the 12 icosahedron vertices at radius k*nn (nn is the radial
    distance of the first shell), k-1 atoms on each of the 30 edges and the
    triangular interior points of the 20 faces, all on the flat facets."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    v = np.array(v)
    v /= np.linalg.norm(v[0])
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    edge2 = np.min(d2[d2 > 1e-9])
    edges = [(i, j) for i in range(12) for j in range(i + 1, 12) if abs(d2[i, j] - edge2) < 1e-6]
    faces = [(i, j, k) for (i, j) in edges for k in range(j + 1, 12)
             if abs(d2[i, k] - edge2) < 1e-6 and abs(d2[j, k] - edge2) < 1e-6]
    assert len(edges) == 30 and len(faces) == 20
    pts = [np.zeros(3)]
    for k in range(1, n_shells + 1):
        r = k * nn
        pts += list(v * r)
        for (i, j) in edges:
            for m in range(1, k):
                pts.append(r * (v[i] + (v[j] - v[i]) * m / k))
        for (i, j, l) in faces:
            for a in range(1, k):
                for b in range(1, k - a):
                    pts.append(r * (v[i] + (v[j] - v[i]) * a / k + (v[l] - v[i]) * b / k))
    out = np.array(pts)
    assert len(out) == 1 + sum(10 * k * k + 2 for k in range(1, n_shells + 1))
    return out


def _periodic_gauss_1d(x: np.ndarray, centre: np.ndarray, length: float, sigma: float) -> np.ndarray:
    """exp(-(x - c + s L)^2 / 2 sigma^2) summed over images s within 8 sigma."""
    s_max = int(math.ceil(8.0 * sigma / length)) + 1
    d = x[None, :] - centre[:, None]
    out = np.zeros_like(d)
    for s in range(-s_max, s_max + 1):
        out += np.exp(-((d + s * length) ** 2) / (2.0 * sigma * sigma))
    return out


def gaussian_density(cell, shape, positions, charges, sigma: float) -> np.ndarray:
    """Sum of normalised atom-centred Gaussians rho_I = Z (2 pi s^2)^-3/2 e^{-r^2/2 s^2}.

    Periodic images within 8 sigma are included.  Orthorhombic cells use the
    separable form; other cells sum images explicitly (small grids only)."""
    cell = np.asarray(cell, dtype=np.float64)
    shape = tuple(int(n) for n in shape)
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    q = np.broadcast_to(np.asarray(charges, dtype=np.float64), (len(pos),))
    norm = (2.0 * math.pi * sigma * sigma) ** -1.5
    if np.allclose(cell, np.diag(np.diag(cell)), atol=1e-12 * np.abs(cell).max()):
        L = np.diag(cell)
        g = [_periodic_gauss_1d(np.arange(n) * (L[a] / n), pos[:, a], L[a], sigma) for a, n in enumerate(shape)]
        t = (q * norm)[:, None, None] * g[0][:, :, None] * g[1][:, None, :]
        rho = t.reshape(len(pos), -1).T @ g[2]
        return rho.reshape(shape)
    # general cell: explicit images on the full grid
    frac = np.stack(np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij"), -1)
    r = frac @ cell
    rho = np.zeros(shape)
    heights = 1.0 / np.linalg.norm(np.linalg.inv(cell), axis=0)   # plane spacing per axis
    smax = [int(math.ceil(8.0 * sigma / h)) + 1 for h in heights]
    for I in range(len(pos)):
        for s0 in range(-smax[0], smax[0] + 1):
            for s1 in range(-smax[1], smax[1] + 1):
                for s2 in range(-smax[2], smax[2] + 1):
                    c = pos[I] + np.array([s0, s1, s2]) @ cell
                    d2 = ((r - c) ** 2).sum(-1)
                    rho += q[I] * norm * np.exp(-d2 / (2.0 * sigma * sigma))
    return rho


def apply_noise(rho: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """rho_i <- rho_i (1 + a (2 u_i - 1)), u_i from the SplitMix64 stream (flat C index i)."""
    if amplitude == 0.0:
        return rho
    u = splitmix64_uniform(seed, np.arange(rho.size, dtype=np.uint64)).reshape(rho.shape)
    return rho * (1.0 + amplitude * (2.0 * u - 1.0))


def renormalise(rho: np.ndarray, cell, n_electrons: float) -> np.ndarray:
    """Scale rho so that sum(rho) * Omega / N = n_electrons."""
    omega = abs(np.linalg.det(np.asarray(cell, dtype=np.float64)))
    return rho * (n_electrons / (rho.sum() * omega / rho.size))


def model_density(wl: dict) -> np.ndarray:
    """FP64 model density of a workload dict (see `workload`)."""
    rho = gaussian_density(wl["cell"], wl["shape"], wl["positions"], wl["charges"], wl["sigma"])
    if wl.get("density_floor", 0.0) > 0.0:
        rho = np.maximum(rho, wl["density_floor"])
    rho = apply_noise(rho, wl.get("noise", 0.0), wl.get("seed", 0))
    return renormalise(rho, wl["cell"], wl["n_electrons"])


def _al_workload(n_cells, shape, noise, seed, n_knots, jitter=0.0, jitter_seed=0):
    cell, pos = fcc_positions(n_cells)
    if jitter > 0.0:
        pos = pos + np.random.default_rng(jitter_seed).normal(0.0, jitter, pos.shape)
    n = len(pos)
    return dict(cell=cell, shape=tuple(shape), positions=pos, species=np.zeros(n, dtype=np.int32),
                Z=np.array([3.0]), rc=np.array([0.8]), charges=np.full(n, 3.0), n_electrons=3.0 * n,
                sigma=1.0, noise=noise, seed=seed, n_knots=n_knots, n_atoms=n)


def workload(name: str, index: int = 0) -> dict:
    """Named synthetic workloads (the benchmark and test cases).

    fcc-al-4/32      4-atom FCC Al cell, 32^3 grid, 5% noise, 10 knots
    fcc-al-256/128   4x4x4 FCC Al cells (256 atoms), 128^3, 2% noise, 16 knots
    mg147/192        Mackay icosahedron Mg147 in a 40 bohr box, 192^3, 30 knots
    fcc-al-108-snap  snapshot `index` (0..63) of jittered 108-atom FCC Al,
                     grid drawn from {64,80,96,120}^3, 16 knots
    fcc-al-1m/1024   64^3 FCC Al cells (1,048,576 atoms), 1024^3, 12 knots
    mg55/128         Mackay icosahedron Mg55 in a 40 bohr box, 128^3 (>= 9 bohr of vacuum
                     around the outer shell: an isolated cluster for dipoles and spectra)
    """
    if name == "fcc-al-4/32":
        return _al_workload(1, (32, 32, 32), 0.05, 1, 10)
    if name == "fcc-al-256/128":
        return _al_workload(4, (128, 128, 128), 0.02, 2, 16)
    if name == "fcc-al-108-snap":
        sizes = (64, 80, 96, 120)
        n = sizes[int(np.random.default_rng(1000 + index).integers(0, 4))]
        return _al_workload(3, (n, n, n), 0.02, 40 + index, 16, jitter=0.2, jitter_seed=4 + index)
    if name == "fcc-al-1m/1024":
        return _al_workload(64, (1024, 1024, 1024), 0.02, 5, 12)
    if name == "fcc-al-4/16":
        return _al_workload(1, (16, 16, 16), 0.0, 5, 12)
    if name == "mg147/192":
        L = 40.0
        pos = mackay_icosahedron(3, 6.0) + L / 2.0
        n = len(pos)
        return dict(cell=np.diag([L, L, L]), shape=(192, 192, 192), positions=pos,
                    species=np.zeros(n, dtype=np.int32), Z=np.array([2.0]), rc=np.array([1.0]),
                    charges=np.full(n, 2.0), n_electrons=2.0 * n, sigma=1.4, noise=0.0, seed=3,
                    density_floor=1e-8, n_knots=30, n_atoms=n)
    if name == "mg55/128":
        L = 40.0
        pos = mackay_icosahedron(2, 5.5) + L / 2.0
        n = len(pos)
        return dict(cell=np.diag([L, L, L]), shape=(128, 128, 128), positions=pos,
                    species=np.zeros(n, dtype=np.int32), Z=np.array([2.0]), rc=np.array([1.0]),
                    charges=np.full(n, 2.0), n_electrons=2.0 * n, sigma=1.4, noise=0.0, seed=3,
                    density_floor=1e-8, n_knots=16, n_atoms=n)
    raise KeyError(name)
