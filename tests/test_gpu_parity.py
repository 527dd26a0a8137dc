"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances
  FP64 path : energy <= 1e-10 relative (per term), V <= 1e-9 Ha max abs.
  FP32 path : energy <= 1e-6 Ha/atom; V: ||dV||_2 / ||V||_2 <= 1e-4, at points
              whose kF is not within 1e-5 (relative) of a knot (there FP32 and
              FP64 may legitimately pick neighbouring spline intervals; the
              interval is a floating-point decision taken in each side's own
              precision).
Both sides read the same float32 density (the oracle upcasts it exactly).
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn
from oracle.evaluate import Functional as OFunc, evaluate
from oracle.forces import forces as oforces
from oracle.grid import Grid as OGrid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402

TERM_BITS = {"TF": L.TERM_TF, "VW": L.TERM_VW, "NL": L.TERM_NL, "HARTREE": L.TERM_HARTREE, "PP": L.TERM_PP,
             "XC": L.TERM_XC}
KEYMAP = {"TF": "TF", "VW": "vW", "NL": "NL", "HARTREE": "H", "PP": "PP", "XC": "XC"}


def triclinic():
    return np.array([[9.0, 0.0, 0.0], [1.1, 8.2, 0.0], [-0.6, 0.8, 7.7]])


def small_case(shape, cell=None, natoms=3, seed=0, noise=0.1):
    cell = triclinic() if cell is None else cell
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (natoms, 3)) @ cell
    rho = W.gaussian_density(cell, shape, pos, 2.0, 0.9)
    rho = W.apply_noise(rho + 1e-3, noise, seed + 1)
    rho = W.renormalise(rho, cell, 2.0 * natoms)
    return cell, pos, rho


def run_both(cell, shape, pos, rho64, func_kw, precision, species=None, Z=(2.0,), rc=(0.9,), options=()):
    species = np.zeros(len(pos), np.int32) if species is None else species
    dt = torch.float64 if precision == L.FP64 else torch.float32
    rho_in = rho64 if precision == L.FP64 else rho64.astype(np.float32)
    g = ofd.Grid(cell, shape)
    for opt, val in options:
        g.set_option(opt, val)
    g.set_ions(pos, species, Z, rc)
    f = ofd.Functional(precision=precision, **func_kw)
    E, V = g.energy_potential(torch.from_numpy(np.ascontiguousarray(rho_in)).to("cuda", dt), f)
    og = OGrid(cell, shape)
    Vg = ofn.external_potential_G(og, pos, species, list(Z), list(rc))
    terms = tuple(k for k, b in TERM_BITS.items() if f.terms & b)
    of = OFunc(terms=terms, alpha=f.alpha, beta=f.beta, n_knots=f.n_knots,
               spacing="log" if f.knot_spacing == L.KNOTS_LOG else "arith",
               knots=None if f.knots is None else np.asarray(f.knots),
               potential="exact" if f.nl_potential == L.NLPOT_EXACT else "interpolated",
               kernel="lwt" if f.kernel == L.KERNEL_LWT else "wt_global", mgp_x=f.mgp_x, mgp_y=f.mgp_y)
    Eo, Vo = evaluate(og, rho_in.astype(np.float64), of, Vg)
    return E, V.double().cpu().numpy(), Eo, Vo, og, g


def lattice_positions(cell, counts, seed, jitter=0.1):
    """Atoms on a regular fractional lattice of counts[a] points per axis, each moved by up
    to +-jitter of its lattice spacing: a bulk-like charge balance (random placement along a
    long axis makes long-wavelength charge fluctuations whose Hartree and PP energies per
    atom are tens of Ha, far from any solid)."""
    rng = np.random.default_rng(seed)
    ijk = np.stack(np.meshgrid(*[np.arange(c) for c in counts], indexing="ij"), -1).reshape(-1, 3)
    f = (ijk + 0.5 + rng.uniform(-jitter, jitter, ijk.shape)) / np.asarray(counts)
    return f @ np.asarray(cell)


def knot_mask(rho, n_knots, rtol=1e-5, knots=None):
    k = ofn.make_knots(rho, n_knots) if knots is None else np.asarray(knots)
    kF = ofn.fermi_wavevector(rho)
    d = np.min(np.abs(kF[..., None] / k[None] - 1.0), axis=-1)
    return d > rtol


FP64_CASES = [
    ((12, 10, 15), dict(n_knots=5)),
    ((16, 18, 20), dict(n_knots=6, knot_spacing=L.KNOTS_ARITH)),
    ((30, 24, 27), dict(n_knots=8, nl_potential=L.NLPOT_INTERP)),
    ((20, 20, 20), dict(n_knots=4, kernel=L.KERNEL_WT_GLOBAL)),
    ((25, 32, 18), dict(n_knots=7)),
    ((18, 16, 20), dict(n_knots=6, terms=L.TERMS_VALID)),            # with LDA xc
    # Eq. MGP kernels (tabulated correction on the GPU, quadrature in the oracle)
    ((12, 10, 15), dict(n_knots=5, mgp_x=1.0)),                       # LMGP
    ((16, 18, 20), dict(n_knots=6, mgp_x=0.5)),                       # LMGPA
    ((15, 12, 16), dict(n_knots=5, mgp_x=1.0, mgp_y=5.0 / 3.0)),      # LMGPG
    ((20, 20, 20), dict(n_knots=4, kernel=L.KERNEL_WT_GLOBAL, mgp_x=1.0)),   # MGP (global k_F)
    ((16, 18, 12), dict(n_knots=6, mgp_x=1.0, nl_potential=L.NLPOT_INTERP)),
]


@pytest.mark.parametrize("shape,kw", FP64_CASES)
def test_fp64_energy_potential_matches_oracle(shape, kw):
    cell, pos, rho = small_case(shape)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, kw, L.FP64)
    for k in ("TF", "vW", "NL", "H", "PP", "XC", "total"):
        assert abs(E[k] - Eo[k]) <= 1e-10 * max(1.0, abs(Eo[k])), (k, E[k], Eo[k])
    assert np.max(np.abs(V - Vo)) <= 1e-9 * max(1.0, np.max(np.abs(Vo))), np.max(np.abs(V - Vo))


@pytest.mark.parametrize("term", ["TF", "VW", "NL", "HARTREE", "PP", "XC"])
def test_fp64_single_terms(term):
    shape = (18, 20, 16)
    cell, pos, rho = small_case(shape, seed=3)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(terms=TERM_BITS[term], n_knots=6), L.FP64)
    k = KEYMAP[term]
    assert abs(E[k] - Eo[k]) <= 1e-10 * max(1.0, abs(Eo[k])), (E[k], Eo[k])
    assert np.max(np.abs(V - Vo)) <= 1e-9 * max(1.0, np.max(np.abs(Vo)))


FP32_CASES = [
    ("fcc-al-4/32", dict()),
    ("fcc-al-4/32", dict(nl_potential=L.NLPOT_INTERP)),
    ("fcc-al-4/32", dict(terms=L.TERMS_VALID)),                        # with LDA xc
    ("fcc-al-4/32", dict(mgp_x=1.0)),                                  # LMGP
]


@pytest.mark.parametrize("name,kw", FP32_CASES)
def test_fp32_mixed_workload_matches_oracle(name, kw):
    wl = W.workload(name)
    rho = W.model_density(wl)
    E, V, Eo, Vo, og, _ = run_both(wl["cell"], wl["shape"], wl["positions"], rho,
                                   dict(n_knots=wl["n_knots"], **kw), L.FP32_MIXED, wl["species"],
                                   tuple(wl["Z"]), tuple(wl["rc"]))
    assert abs(E["total"] - Eo["total"]) / wl["n_atoms"] <= 1e-6, (E["total"], Eo["total"])
    for k in ("TF", "vW", "NL", "H", "PP", "XC"):
        assert abs(E[k] - Eo[k]) / wl["n_atoms"] <= 1e-6, (k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), wl["n_knots"])
    rel = np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m])
    assert rel <= 1e-4, rel


def test_fp32_mixed_ragged_triclinic():
    shape = (30, 24, 25)
    cell, pos, rho = small_case(shape, seed=5)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=8), L.FP32_MIXED)
    assert abs(E["total"] - Eo["total"]) <= 1e-6 * 3, (E, Eo)
    m = knot_mask(rho.astype(np.float32).astype(np.float64), 8)
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4


@pytest.mark.parametrize("precision,tol", [(L.FP64, 1e-10), (L.FP32_MIXED, 2e-6)])
def test_forces_match_oracle(precision, tol):
    wl = W.workload("fcc-al-4/32")
    rho = W.model_density(wl)
    rin = rho if precision == L.FP64 else rho.astype(np.float32)
    dt = torch.float64 if precision == L.FP64 else torch.float32
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
    F = g.forces(torch.from_numpy(np.ascontiguousarray(rin)).to("cuda", dt), precision)
    og = OGrid(wl["cell"], wl["shape"])
    Fo = oforces(og, rin.astype(np.float64), wl["positions"], wl["species"], wl["Z"], wl["rc"])
    assert np.max(np.abs(F - Fo)) <= tol * max(1.0, np.max(np.abs(Fo))), np.max(np.abs(F - Fo))


@pytest.mark.parametrize("shape", [(16, 80, 20), (16, 96, 20), (24, 128, 20)])
def test_forces_after_autotuning_match_oracle(shape):
    """The plain one-channel transforms (single-call forces here) use the n1 pencils the
    autotuner picked at the grid's first evaluation, with that pick's tile and block size."""
    cell, pos, rho = _bulk_case(shape)
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, np.zeros(len(pos), np.int32), (3.0,), (0.8,))
    r = torch.from_numpy(rho.astype(np.float32)).cuda()
    g.energy_potential(r, ofd.Functional(n_knots=8))          # tunes
    F = g.forces(r)
    og = OGrid(cell, shape)
    Fo = oforces(og, rho.astype(np.float32).astype(np.float64), pos, np.zeros(len(pos), np.int32), [3.0], [0.8])
    assert np.max(np.abs(F - Fo)) <= 1e-5 * max(1.0, np.max(np.abs(Fo))), (np.max(np.abs(F - Fo)), g.tuning_report())


def test_frozen_knots_fp64():
    shape = (16, 16, 16)
    cell, pos, rho = small_case(shape, seed=9)
    knots = ofn.make_knots(rho, 6) * np.array([0.9, 1, 1, 1, 1, 1.1])
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=6, knots=knots), L.FP64)
    assert abs(E["NL"] - Eo["NL"]) <= 1e-10 * abs(Eo["NL"])
    assert np.max(np.abs(V - Vo)) <= 1e-9


def test_mgp_parameters_out_of_range_are_errors():
    cell, pos, rho = small_case((12, 10, 15))
    g = ofd.Grid(cell, (12, 10, 15))
    g.set_ions(pos, np.zeros(len(pos), np.int32), (2.0,), (0.9,))
    r = torch.from_numpy(rho).cuda()
    for kw in (dict(mgp_x=1.0, mgp_y=0.0), dict(mgp_x=11.0), dict(mgp_x=float("nan")), dict(mgp_x=1.0, mgp_y=12.0)):
        with pytest.raises(ofd.OFDFTError):
            g.energy_potential(r, ofd.Functional(precision=L.FP64, n_knots=5, **kw))


def test_bad_density_and_unsupported_size_are_errors():
    cell = np.eye(3) * 8.0
    with pytest.raises(ofd.OFDFTError) as e:
        ofd.Grid(cell, (14, 16, 16))        # 14 = 2 * 7
    assert e.value.status == -2
    g = ofd.Grid(cell, (16, 16, 16))
    rho = torch.full((16, 16, 16), 0.01, device="cuda")
    rho[3, 4, 5] = float("nan")
    with pytest.raises(ofd.OFDFTError) as e:
        g.energy_potential(rho, ofd.Functional(terms=L.TERM_TF | L.TERM_VW))
    assert e.value.status == -3
    rho[3, 4, 5] = -1.0
    with pytest.raises(ofd.OFDFTError) as e:
        g.energy_potential(rho, ofd.Functional(terms=L.TERM_TF))
    assert e.value.status == -3
    with pytest.raises(ofd.OFDFTError) as e:
        g.energy_potential(rho.abs(), ofd.Functional(terms=L.TERM_PP))   # no ions set
    assert e.value.status == -7


def test_repeated_runs_are_bit_identical():
    wl = W.workload("fcc-al-4/32")
    rho = torch.from_numpy(W.model_density(wl).astype(np.float32)).cuda()
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
    f = ofd.Functional(n_knots=10)
    E0, V0 = g.energy_potential(rho, f)
    for _ in range(5):
        E1, V1 = g.energy_potential(rho, f)
        assert E1 == E0
        assert torch.equal(V0, V1)


# ---------------------------------------------------------------- size-specialised kernels
SPEC_SHAPES = [(128, 96, 64), (80, 120, 32), (192, 64, 96), (64, 192, 120), (30, 36, 80), (32, 40, 192),
               (96, 128, 64)]


@pytest.mark.parametrize("shape", SPEC_SHAPES)
def test_fp32_specialised_sizes_match_oracle(shape):
    """Every axis length here has compile-time kernels for its role (rows: n2,
    pencils: n1, reciprocal pass: n0)."""
    cell = np.diag([0.2 * n for n in shape])
    rng = np.random.default_rng(sum(shape))
    pos = rng.uniform(0, 1, (6, 3)) @ cell
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0) + 2e-3, 0.03, 11), cell, 18.0)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=8), L.FP32_MIXED, Z=(3.0,), rc=(0.8,))
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] - Eo[k]) / 6 <= 1e-6, (k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), 8)
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4


def test_fp64_specialised_128_matches_oracle():
    shape = (128, 32, 128)
    cell = np.diag([0.2 * n for n in shape])
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, 1, (4, 3)) @ cell
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0) + 2e-3, 0.03, 12), cell, 12.0)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=6), L.FP64, Z=(3.0,), rc=(0.8,))
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] - Eo[k]) <= 1e-10 * max(1.0, abs(Eo[k])), (k, E[k], Eo[k])
    assert np.max(np.abs(V - Vo)) <= 1e-9 * max(1.0, np.max(np.abs(Vo)))


@pytest.mark.parametrize("kw", [dict(), dict(nl_potential=L.NLPOT_INTERP), dict(kernel=L.KERNEL_WT_GLOBAL)])
def test_specialised_and_generic_kernels_agree(kw):
    wl = W.workload("fcc-al-256/128")
    rho = torch.from_numpy(W.model_density(wl).astype(np.float32)).cuda()
    f = ofd.Functional(n_knots=16, **kw)
    out = []
    for choice in (L.KERNELS_AUTO, L.KERNELS_GENERIC):
        g = ofd.Grid(wl["cell"], wl["shape"])
        g.set_option(L.OPTION_KERNELS, choice)
        g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
        out.append(g.energy_potential(rho, f))
    (E1, V1), (E2, V2) = out
    # same method; the specialised FP32 plans use radix-16 passes and other
    # reduction blocking, so the two differ by FP32 rounding: bound it by half
    # the oracle tolerance (each side is checked against the oracle elsewhere)
    for k in E1:
        assert abs(E1[k] - E2[k]) / wl["n_atoms"] <= 5e-7, (k, E1[k], E2[k])
    assert float((V1 - V2).norm() / V1.norm()) <= 2.5e-5      # a quarter of the oracle tolerance


@pytest.mark.parametrize("shape", [(1024, 12, 20), (16, 1024, 18), (20, 12, 1024)])
def test_length_1024_axes_match_oracle(shape):
    """1024-point axes in each role, FP32-mixed and FP64, at a bulk-like density: one atom
    (Z = 3) per ~110 bohr^3 on a jittered lattice along the long axis."""
    cell = np.diag([0.25 * n for n in shape])
    vol = float(np.prod(np.diag(cell)))
    counts = [max(1, round(vol / 110.0)) if n == 1024 else 1 for n in shape]
    pos = lattice_positions(cell, counts, shape[0] + 7)
    nat = len(pos)
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0), 0.03, 5), cell, 3.0 * nat)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=6), L.FP64, Z=(3.0,), rc=(0.8,))
    assert abs(E["total"] - Eo["total"]) <= 1e-10 * max(1.0, abs(Eo["total"]))
    assert np.max(np.abs(V - Vo)) <= 1e-9 * max(1.0, np.max(np.abs(Vo)))
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=6), L.FP32_MIXED, Z=(3.0,), rc=(0.8,))
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] - Eo[k]) / nat <= 1e-6, (k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), 6)
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4


@functools.lru_cache(maxsize=None)
def _n_configurations(shape, role):
    """How many configurations the autotuner times for a role at this shape (one evaluation of a
    uniform density on a cubic-ish cell)."""
    g = ofd.Grid(np.diag([0.25 * n for n in shape]), shape)
    g.energy_potential(torch.full(shape, 0.01, dtype=torch.float32, device="cuda"),
                       ofd.Functional(n_knots=6, terms=L.TERMS_ALL & ~L.TERM_PP))
    seg = [x for x in g.tuning_report().split(";") if x.strip().startswith(role)]
    return seg[0].count("[") if seg else 0


@functools.lru_cache(maxsize=None)
def _config_case(shape):
    """A bulk-like density for the shape (built once per shape)."""
    if max(shape) < 1024:
        return _bulk_case(shape)
    cell = np.diag([0.25 * n for n in shape])
    vol = float(np.prod(np.diag(cell)))
    counts = [max(1, round(vol / 110.0)) if n == 1024 else 1 for n in shape]
    pos = lattice_positions(cell, counts, shape[0] + 11)
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0), 0.03, 6), cell, 3.0 * len(pos))
    return cell, pos, rho


def _role_cases(n):
    return [((20, 12, n), L.OPTION_PICK_ROWS), ((16, n, 18), L.OPTION_PICK_PENCIL), ((n, 12, 20), L.OPTION_PICK_RECIP)]


@pytest.mark.parametrize("shape,option", [c for n in (64, 80, 96, 120, 192, 1024) for c in _role_cases(n)])
@pytest.mark.parametrize("pick", range(5))
def test_every_compiled_configuration_matches_oracle(shape, option, pick):
    """Each compiled configuration of the role whose axis is long (the autotuner's candidates for
    the rows, the n1 pencils or the reciprocal-space pass at 64 ... 1024 points, forced one at a
    time; indices past the list are skipped), FP32-mixed, against the oracle."""
    role = {L.OPTION_PICK_ROWS: "rows", L.OPTION_PICK_PENCIL: "pencil", L.OPTION_PICK_RECIP: "recip"}[option]
    if pick >= _n_configurations(shape, role):
        pytest.skip("no such configuration")
    cell, pos, rho = _config_case(shape)
    nat = len(pos)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(n_knots=6), L.FP32_MIXED, Z=(3.0,), rc=(0.8,),
                                   options=((option, pick),))
    for k in ("TF", "vW", "NL", "H", "PP", "total"):
        assert abs(E[k] - Eo[k]) / nat <= 1e-6, (pick, k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), 6)
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4, pick


# ---------------------------------------------------------------- channel-batched row kernels (n2 = 128)
ROW2_MODES = [dict(n_knots=16), dict(n_knots=24), dict(n_knots=16, nl_potential=L.NLPOT_INTERP),
              dict(n_knots=24, nl_potential=L.NLPOT_INTERP), dict(n_knots=5, kernel=L.KERNEL_WT_GLOBAL),
              dict(n_knots=9, knot_spacing=L.KNOTS_ARITH)]


@pytest.mark.parametrize("kw", ROW2_MODES)
def test_fp32_channel_batched_rows_match_oracle(kw):
    """n2 = 128 rows run the channel-batched kernels (all channels of a group in one
    transform): an odd number of rows (the last pair is half empty), 16 knots (one
    group) and 24 knots (two groups, knot pairs split across them), every NL mode."""
    shape = (9, 5, 128)
    cell = np.array([[4.5, 0.0, 0.0], [0.7, 3.0, 0.0], [-0.4, 0.5, 25.6]])
    pos = lattice_positions(cell, (1, 1, 4), 31)          # ~86 bohr^3 per atom
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 0.9), 0.05, 13), cell, 12.0)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, kw, L.FP32_MIXED, Z=(3.0,), rc=(0.8,))
    for k in ("TF", "vW", "NL", "H", "PP", "XC", "total"):
        assert abs(E[k] - Eo[k]) / 4 <= 1e-6, (k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), kw["n_knots"])
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4


@pytest.mark.parametrize("term", ["TF", "VW", "NL", "HARTREE", "PP", "XC"])
def test_fp32_channel_batched_rows_single_terms(term):
    shape = (8, 5, 128)
    cell = np.diag([4.0, 3.0, 25.0])
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 1, (3, 3)) @ cell
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 0.9) + 2e-3, 0.05, 17), cell, 9.0)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, dict(terms=TERM_BITS[term], n_knots=6), L.FP32_MIXED,
                                   Z=(3.0,), rc=(0.8,))
    key = KEYMAP[term]
    assert abs(E[key] - Eo[key]) / 3 <= 1e-6, (term, E[key], Eo[key])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), 6) if term == "NL" else np.ones(shape, bool)
    assert np.linalg.norm((V - Vo)[m]) / max(np.linalg.norm(Vo[m]), 1e-30) <= 1e-4


@pytest.mark.parametrize("kw", [dict(), dict(nl_potential=L.NLPOT_INTERP), dict(kernel=L.KERNEL_WT_GLOBAL)])
def test_channel_batched_and_per_channel_rows_agree(kw):
    wl = W.workload("fcc-al-256/128")
    rho = torch.from_numpy(W.model_density(wl).astype(np.float32)).cuda()
    f = ofd.Functional(n_knots=16, **kw)
    out = []
    for choice in (L.KERNELS_TILE_RECIP, L.KERNELS_PER_CHANNEL_ROWS):
        g = ofd.Grid(wl["cell"], wl["shape"])
        g.set_option(L.OPTION_KERNELS, choice)
        g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
        out.append(g.energy_potential(rho, f))
    (E1, V1), (E2, V2) = out
    # the forward rows do the same arithmetic per sequence in both forms, so every
    # G-space energy agrees to the FP64 rounding of the final sums (whose tree follows
    # the inverse row kernel's block size); the spline blend of the inverse rows groups
    # its products differently, so V (and the real-space E_NL of the interpolated
    # mode) differ by FP32 rounding (each side is checked against the oracle elsewhere)
    for k in E1:
        if kw.get("nl_potential") == L.NLPOT_INTERP and k in ("NL", "total"):
            assert abs(E1[k] - E2[k]) / wl["n_atoms"] <= 5e-7, (k, E1[k], E2[k])
        else:
            assert abs(E1[k] - E2[k]) <= 1e-13 * max(1.0, abs(E1[k])), (k, E1[k], E2[k])
    assert float((V1 - V2).norm() / V1.norm()) <= 2.5e-5


# ---------------------------------------------------------------- persistent reciprocal-space kernel
# n0 in {32, 64, 128, 1024} runs the register-resident, tensor-copy kernel: ragged last column tiles
# (n1 (n2/2+1) not a multiple of 32), every NL mode, the MGP form; n1 (n2/2+1) odd keeps the
# tile kernel (tensor maps need 16-byte row strides)
RECIP_CASES = [((128, 18, 20), dict(n_knots=8)), ((64, 10, 12), dict(n_knots=8)), ((32, 6, 10), dict(n_knots=8)),
               ((128, 5, 8), dict(n_knots=8)), ((128, 18, 20), dict(n_knots=8, nl_potential=L.NLPOT_INTERP)),
               ((64, 10, 12), dict(n_knots=5, kernel=L.KERNEL_WT_GLOBAL)), ((128, 18, 20), dict(n_knots=8, mgp_x=1.0)),
               ((64, 10, 12), dict(n_knots=8, terms=L.TERMS_VALID))]


@functools.lru_cache(maxsize=None)
def _bulk_case(shape):
    cell = np.array([[0.25 * shape[0], 0.0, 0.0], [0.3, 0.45 * shape[1], 0.0], [-0.2, 0.1, 0.4 * shape[2]]])
    vol = abs(np.linalg.det(cell))
    a = vol / max(2, round(vol / 110.0))
    counts = [max(1, round(np.linalg.norm(cell[i]) / a ** (1.0 / 3.0))) for i in range(3)]
    pos = lattice_positions(cell, counts, sum(shape))
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0), 0.05, 3), cell, 3.0 * len(pos))
    return cell, pos, rho


@pytest.mark.parametrize("pick", range(12))
@pytest.mark.parametrize("shape", [(128, 18, 20), (64, 10, 12), (32, 6, 10), (1024, 6, 10)])
def test_every_reciprocal_kernel_configuration_matches_oracle(shape, pick):
    """Each compiled configuration of the reciprocal-space pass for the shape's n0 (the
    autotuner's candidates, forced one at a time; indices past the list are skipped)."""
    cell, pos, rho = _bulk_case(shape)
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, np.zeros(len(pos), np.int32), (3.0,), (0.8,))
    g.energy_potential(torch.from_numpy(rho.astype(np.float32)).cuda(), ofd.Functional(n_knots=8))
    n_cand = g.tuning_report().split(";")[0].count("[")
    if not g.tuning_report().startswith("recip") or pick >= n_cand:
        pytest.skip("no such configuration")
    for kw in (dict(n_knots=8), dict(n_knots=5, kernel=L.KERNEL_WT_GLOBAL), dict(n_knots=8, nl_potential=L.NLPOT_INTERP)):
        E, V, Eo, Vo, og, g2 = run_both(cell, shape, pos, rho, kw, L.FP32_MIXED, Z=(3.0,), rc=(0.8,),
                                        options=((L.OPTION_PICK_RECIP, pick),))
        nat = len(pos)
        for k in ("TF", "vW", "NL", "H", "PP", "total"):
            assert abs(E[k] - Eo[k]) / nat <= 1e-6, (pick, kw, k, E[k], Eo[k])
        m = knot_mask(rho.astype(np.float32).astype(np.float64), kw["n_knots"])
        assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4, (pick, kw)


@pytest.mark.parametrize("pick", range(10))
def test_every_row_kernel_configuration_matches_oracle(pick):
    """Each compiled configuration of the n2 rows for n2 = 128 (channel-batched with groups of
    10 to 20 channels, per-channel; forced one at a time): 11 channels, 23 channels (two groups
    for every channel-batched configuration), the Wang-Teter and interpolated modes."""
    shape = (20, 18, 128)
    cell, pos, rho = _bulk_case(shape)
    g = ofd.Grid(cell, shape)
    g.set_ions(pos, np.zeros(len(pos), np.int32), (3.0,), (0.8,))
    g.energy_potential(torch.from_numpy(rho.astype(np.float32)).cuda(), ofd.Functional(n_knots=8))
    rows = [seg for seg in g.tuning_report().split(";") if seg.strip().startswith("rows")]
    n_cand = rows[0].count("[") if rows else 0
    if pick >= n_cand:
        pytest.skip("no such configuration")
    for kw in (dict(n_knots=8), dict(n_knots=20), dict(n_knots=5, kernel=L.KERNEL_WT_GLOBAL),
               dict(n_knots=8, nl_potential=L.NLPOT_INTERP)):
        E, V, Eo, Vo, og, g2 = run_both(cell, shape, pos, rho, kw, L.FP32_MIXED, Z=(3.0,), rc=(0.8,),
                                        options=((L.OPTION_PICK_ROWS, pick),))
        nat = len(pos)
        for k in ("TF", "vW", "NL", "H", "PP", "total"):
            assert abs(E[k] - Eo[k]) / nat <= 1e-6, (pick, kw, k, E[k], Eo[k])
        m = knot_mask(rho.astype(np.float32).astype(np.float64), kw["n_knots"])
        assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4, (pick, kw)


@pytest.mark.parametrize("shape,kw", RECIP_CASES)
def test_fp32_reciprocal_kernel_shapes_match_oracle(shape, kw):
    cell = np.array([[0.25 * shape[0], 0.0, 0.0], [0.3, 0.45 * shape[1], 0.0], [-0.2, 0.1, 0.4 * shape[2]]])
    # about one atom per 110 bohr^3 on a lattice as even as the cell allows (a bulk-like density:
    # no near-vacuum gaps, where the von Weizsaecker potential divides FP32 noise by a small psi)
    vol = abs(np.linalg.det(cell))
    a = vol / max(2, round(vol / 110.0))
    counts = [max(1, round(np.linalg.norm(cell[i]) / a ** (1.0 / 3.0))) for i in range(3)]
    pos = lattice_positions(cell, counts, sum(shape))
    nat = len(pos)
    rho = W.renormalise(W.apply_noise(W.gaussian_density(cell, shape, pos, 3.0, 1.0), 0.05, 3), cell, 3.0 * nat)
    E, V, Eo, Vo, og, _ = run_both(cell, shape, pos, rho, kw, L.FP32_MIXED, Z=(3.0,), rc=(0.8,))
    for k in ("TF", "vW", "NL", "H", "PP", "XC", "total"):
        assert abs(E[k] - Eo[k]) / nat <= 1e-6, (k, E[k], Eo[k])
    m = knot_mask(rho.astype(np.float32).astype(np.float64), kw["n_knots"])
    assert np.linalg.norm((V - Vo)[m]) / np.linalg.norm(Vo[m]) <= 1e-4
