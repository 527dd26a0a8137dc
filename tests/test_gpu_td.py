"""GPU tests of real-time TD-OFDFT (Sec. "Time-Dependent OFDFT", Eq. cn) through the C ABI.

Closed forms: the Crank-Nicolson phase of a plane wave (v = 0) and of an eigenstate of a
fixed potential (Lanczos), charge conservation (CN is unitary), reversibility (dt, -dt).
Parity: psi(t) and the dipole series against the oracle's propagation (oracle/td.py) on the
same seeded inputs, for TF + vW + Hartree (+ PP + LDA xc, + LWT), FP64 and FP32-mixed.
"""
import ctypes as ct
import math

import numpy as np
import pytest

import workloads as W
from oracle import functionals as ofn
from oracle import td as otd
from oracle.evaluate import Functional as OFunc
from oracle.grid import Grid as OGrid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402

T_ALL = L.TERM_TF | L.TERM_VW | L.TERM_HARTREE


def _box(n, Lb):
    return OGrid(np.diag([Lb, Lb, Lb]), (n, n, n)), np.diag([Lb, Lb, Lb])


def _blob(og, centre=(0.0, 0.0, 0.0), sigma=1.0, ne=2.0):
    r = otd.positions(og) - np.asarray(centre)
    rho = np.exp(-(r ** 2).sum(-1) / (2 * sigma ** 2))
    return rho * ne / (rho.sum() * og.dV)


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt).contiguous()


def _run_gpu(cell, shape, psi0, rho0, func, dt, n, n_corr=1, ions=None, tol=0.0):
    g = ofd.Grid(cell, shape)
    if ions is not None:
        g.set_ions(*ions)
    tdt = torch.float64 if func.precision == L.FP64 else torch.float32
    re, im = _dev(psi0.real, tdt), _dev(psi0.imag, tdt)
    dip, rep = g.td_propagate(re, im, _dev(rho0, tdt), func, dt, n, n_corrector=n_corr, solver_tol=tol)
    return re.double().cpu().numpy() + 1j * im.double().cpu().numpy(), dip, rep, g


@pytest.mark.parametrize("n", [16, 64, 96, 128, 192, 256])     # generic and compile-time n0 transforms
@pytest.mark.parametrize("precision,tol", [(L.FP64, 1e-11), (L.FP32_MIXED, 2e-5)])
def test_plane_wave_takes_the_cn_phase(precision, tol, n):
    og, cell = _box(n, 10.0)
    G = 2 * np.pi * np.array([2.0, -1.0, 3.0]) / 10.0
    psi0 = np.exp(1j * (otd.positions(og) @ G))
    dt, n = 0.3, 7
    psi, dip, rep, _ = _run_gpu(cell, og.shape, psi0, np.abs(psi0) ** 2, ofd.Functional(terms=L.TERM_VW,
                                                                                     precision=precision), dt, n)
    e = 0.5 * G @ G
    phase = ((1 - 0.5j * dt * e) / (1 + 0.5j * dt * e)) ** n
    assert np.max(np.abs(psi - phase * psi0)) < tol
    assert rep["steps"] == n and rep["evaluations"] == 0


def test_eigenstate_of_a_fixed_potential_takes_the_cn_phase():
    import scipy.sparse.linalg as sla
    wl = W.workload("fcc-al-4/32")
    og = OGrid(wl["cell"], (16, 16, 16))
    Vg = ofn.external_potential_G(og, wl["positions"], wl["species"], wl["Z"], wl["rc"])
    v = og.ifft(Vg)

    def mv(x):
        x = x.reshape(og.shape)
        return (0.5 * og.ifft(og.G2 * og.fft(x)) + v * x).reshape(-1)

    w, U = sla.eigsh(sla.LinearOperator((og.N, og.N), matvec=mv, dtype=np.float64), k=1, which="SA", tol=1e-14)
    psi0 = U[:, 0].reshape(og.shape)
    psi0 *= math.sqrt(12.0 / (np.sum(psi0 ** 2) * og.dV))
    dt, n = 0.1, 5
    f = ofd.Functional(terms=L.TERM_VW | L.TERM_PP, precision=L.FP64)
    psi, _, rep, _ = _run_gpu(wl["cell"], og.shape, psi0.astype(complex), psi0 ** 2, f, dt, n,
                              ions=(wl["positions"], wl["species"], wl["Z"], wl["rc"]))
    phase = ((1 - 0.5j * dt * w[0]) / (1 + 0.5j * dt * w[0])) ** n
    assert np.max(np.abs(psi - phase * psi0)) < 1e-8 * np.max(np.abs(psi0))


def test_fixed_potential_propagation_is_reversible():
    wl = W.workload("fcc-al-4/32")
    og = OGrid(wl["cell"], (16, 16, 16))
    rho0 = W.renormalise(W.gaussian_density(wl["cell"], og.shape, wl["positions"], 3.0, 1.2), wl["cell"], 12.0)
    psi0 = otd.kick(og, np.sqrt(rho0), [0.1, 0.0, 0.05])
    f = ofd.Functional(terms=L.TERM_VW | L.TERM_PP, precision=L.FP64)
    ions = (wl["positions"], wl["species"], wl["Z"], wl["rc"])
    fwd, _, _, _ = _run_gpu(wl["cell"], og.shape, psi0, rho0, f, 0.2, 6, ions=ions)
    back, _, _, _ = _run_gpu(wl["cell"], og.shape, fwd, rho0, f, -0.2, 6, ions=ions)
    assert np.max(np.abs(back - psi0)) < 1e-9 * np.max(np.abs(psi0))


def _cluster():
    """Two ions (Z = 2, Mg-like valence) in a 14 bohr box, a Gaussian density around them."""
    og, cell = _box(24, 14.0)
    pos = np.array([[7.0 - 1.3, 7.0, 7.0], [7.0 + 1.3, 7.0, 7.0]])      # Cartesian, cell from its corner
    rho0 = _blob(og, sigma=1.1, ne=4.0)
    return og, cell, pos, rho0


# (oracle terms, library terms, PP, density floor).  The LWT case starts from the blob
# floored at 1e-8 (as the Mg147 workload's density): on the raw blob (rho down to 1e-27,
# knots recomputed from min/max rho at every evaluation) the trajectory amplifies the
# linear solves' residuals about 1e4 times (GPU vs oracle: 9e-8 at solver_tol 1e-11,
# 8e-10 at 1e-13, 4e-11 at 1e-14), which says nothing about either implementation.
CASES = {
    "tf_vw_h": (("TF", "VW", "HARTREE"), T_ALL, False, 0.0),
    "tf_vw_h_pp_xc": (("TF", "VW", "HARTREE", "PP", "XC"), T_ALL | L.TERM_PP | L.TERM_XC, True, 0.0),
    "lwt": (("TF", "VW", "NL", "HARTREE", "PP"), T_ALL | L.TERM_NL | L.TERM_PP, True, 1e-8),
}


def _start(og, rho0, floor):
    if floor > 0.0:
        rho0 = np.maximum(rho0, floor)
        rho0 = rho0 * 4.0 / (rho0.sum() * og.dV)
    return rho0, otd.kick(og, np.sqrt(rho0), [0.05, 0.02, 0.0])


@pytest.fixture(scope="module")
def oracle_runs():
    out = {}
    og, cell, pos, rho_blob = _cluster()
    for name, (oterms, _, pp, floor) in CASES.items():
        rho0, psi0 = _start(og, rho_blob, floor)
        Vg = ofn.external_potential_G(og, pos, [0, 0], [2.0], [1.0]) if pp else None
        psi, dip = otd.propagate(og, psi0, rho0, OFunc(terms=oterms, n_knots=8), Vg, 0.05, 8, n_corrector=1)
        out[name] = (rho0, psi0, psi, dip)
    return og, cell, pos, out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [L.FP64, L.FP32_MIXED])
def test_propagation_matches_the_oracle(oracle_runs, name, precision):
    og, cell, pos, out = oracle_runs
    _, terms, pp, _ = CASES[name]
    rho0, psi0, opsi, odip = out[name]
    f = ofd.Functional(terms=terms, n_knots=8, precision=precision)
    ions = (pos, [0, 0], [2.0], [1.0]) if pp else None
    # FP32-mixed solves to a 1e-7 relative residual: the LWT trajectory amplifies the solves'
    # residuals (at the default 1e-5 its psi moves 5e-4 of max|psi| from the oracle's; at 1e-7,
    # 1e-6), so the bound below tests the evaluations and the propagator, not the stop rule
    tol = 1e-7 if precision == L.FP32_MIXED else 0.0
    psi, dip, rep, g = _run_gpu(cell, og.shape, psi0, rho0, f, 0.05, 8, ions=ions, tol=tol)
    scale = np.max(np.abs(opsi))
    if precision == L.FP64:
        assert np.max(np.abs(psi - opsi)) < 1e-9 * scale, name
        assert np.max(np.abs(dip - odip)) < 1e-10, name
        assert abs(np.sum(np.abs(psi) ** 2) * og.dV - 4.0) < 1e-10
    else:
        # FP32-mixed: v_eff to ~1e-6 relative, solves to 1e-7
        assert np.max(np.abs(psi - opsi)) < 2e-4 * scale, name
        assert np.max(np.abs(dip - odip)) < 2e-4 * np.max(np.abs(odip)), name
    assert dip[-1][0] > 0.0 and rep["steps"] == 8 and rep["evaluations"] == 1 + 8 * 2


def test_kick_and_spectrum_match_the_oracle():
    og, cell = _box(16, 10.0)
    rho0 = _blob(og, sigma=1.0, ne=2.0)
    g = ofd.Grid(cell, og.shape)
    re, im = _dev(np.sqrt(rho0), torch.float64), torch.zeros(og.N, dtype=torch.float64, device="cuda")
    g.td_kick(re, im, [0.3, -0.1, 0.2])
    torch.cuda.synchronize()
    ref = otd.kick(og, np.sqrt(rho0), [0.3, -0.1, 0.2])
    got = re.cpu().numpy().reshape(og.shape) + 1j * im.cpu().numpy().reshape(og.shape)
    assert np.max(np.abs(got - ref)) < 1e-13
    t = np.arange(300) * 0.1
    dmu = 0.4 * np.sin(1.1 * t) * np.exp(-0.01 * t)
    w = np.linspace(0.2, 3.0, 15)
    assert np.max(np.abs(ofd.td_spectrum(dmu, 0.1, w, 0.005) - otd.spectrum(dmu, 0.1, w, 0.005))) < 1e-11


def test_td_options_out_of_range_are_rejected():
    og, cell = _box(16, 10.0)
    g = ofd.Grid(cell, og.shape)
    re = torch.ones(og.N, dtype=torch.float64, device="cuda")
    im = torch.zeros_like(re)
    c, keep = ofd.Functional(terms=T_ALL, precision=L.FP64).to_c()
    rep = L.CTdReport()
    for bad in (L.CTdOptions(0.0, 1, 1, 0.0, 0), L.CTdOptions(0.1, -1, 1, 0.0, 0), L.CTdOptions(0.1, 1, 17, 0.0, 0),
                L.CTdOptions(0.1, 1, 1, -1.0, 0), L.CTdOptions(float("nan"), 1, 1, 0.0, 0)):
        st = g.lib.ofdft_td_propagate(g.h, ct.c_void_p(re.data_ptr()), ct.c_void_p(im.data_ptr()), None, ct.byref(c),
                                      ct.byref(bad), None, ct.byref(rep))
        assert st == L.OFDFT_ERR_INVALID_ARG
    del keep
