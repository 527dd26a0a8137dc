"""The no-allocation Thomas-Fermi entry point against the regular one.

ofdft_tf_energy_potential_noalloc serves callers that cannot let a library
allocate device memory (an application whose own allocator owns all device
memory, or code that must not pay for cudaMalloc's device-wide
synchronisation).  Its reduction partials live in a static device array; these
tests call it through the C ABI twice in a row (the second call reuses the array
left by the first) and compare energy and potential with ofdft_energy_potential
(terms = TF), at a small grid and at the largest size the array allows, and
check that a bad density gives E = NaN.  The file name makes pytest collect it
last.
"""
import ctypes as ct

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402


@pytest.mark.parametrize("precision", [L.FP32_MIXED, L.FP64])
def test_noalloc_tf_matches_regular_entry_point(precision):
    lib = L.load()
    wl = W.workload("fcc-al-4/32")
    dt = torch.float64 if precision == L.FP64 else torch.float32
    rho = torch.from_numpy(W.model_density(wl)).to("cuda", dt).contiguous()
    g = ofd.Grid(wl["cell"], wl["shape"])
    E_ref, V_ref = g.energy_potential(rho, ofd.Functional(terms=L.TERM_TF, precision=precision))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        E_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        V = torch.full_like(rho, -1.0)
        st = lib.ofdft_tf_energy_potential_noalloc(ct.c_void_p(rho.data_ptr()), rho.numel(), g.dV, precision,
                                                   ct.c_void_p(E_dev.data_ptr()), ct.c_void_p(V.data_ptr()),
                                                   ct.c_void_p(stream.cuda_stream))
        assert st == L.OFDFT_OK
        torch.cuda.synchronize()
        # FP64: 1e-10 relative; FP32-mixed: the reductions group points differently
        # (FP32 partials of 4 points in the regular path), so FP32 rounding only
        etol = 1e-10 if precision == L.FP64 else 1e-7
        assert abs(float(E_dev) - E_ref["TF"]) <= etol * abs(E_ref["TF"])
        rtol = 1e-12 if precision == L.FP64 else 1e-6
        assert torch.allclose(V, V_ref, rtol=rtol, atol=0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = L.load()
    rho = torch.ones(16, device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.ofdft_tf_energy_potential_noalloc(ct.c_void_p(rho.data_ptr()), L.NOALLOC_MAX_POINTS + 1, 1.0,
                                               L.FP32_MIXED, ct.c_void_p(E_dev.data_ptr()), None,
                                               ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.OFDFT_ERR_INVALID_ARG


def test_noalloc_at_its_maximum_size_matches_regular_entry_point():
    """n = OFDFT_NOALLOC_MAX_POINTS (a 128 x 256 x 256 grid): every slot of the array in use."""
    lib = L.load()
    shape = (128, 256, 256)
    assert np.prod(shape) == L.NOALLOC_MAX_POINTS
    cell = np.diag([0.25 * n for n in shape])
    rho = torch.from_numpy(W.renormalise(W.apply_noise(np.ones(shape), 0.3, 9), cell, 3000.0).astype(np.float32))
    rho = rho.cuda().contiguous()
    g = ofd.Grid(cell, shape)
    E_ref, V_ref = g.energy_potential(rho, ofd.Functional(terms=L.TERM_TF, precision=L.FP32_MIXED))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        E_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        V = torch.full_like(rho, -1.0)
        st = lib.ofdft_tf_energy_potential_noalloc(ct.c_void_p(rho.data_ptr()), rho.numel(), g.dV, L.FP32_MIXED,
                                                   ct.c_void_p(E_dev.data_ptr()), ct.c_void_p(V.data_ptr()),
                                                   ct.c_void_p(stream.cuda_stream))
        assert st == L.OFDFT_OK
        torch.cuda.synchronize()
        assert abs(float(E_dev) - E_ref["TF"]) <= 1e-7 * abs(E_ref["TF"])
        assert torch.allclose(V, V_ref, rtol=1e-6, atol=0.0)


def test_noalloc_bad_density_gives_nan_energy_then_recovers():
    lib = L.load()
    stream = torch.cuda.current_stream()
    rho = torch.full((4096,), 0.01, device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad in (float("nan"), -1.0, float("inf")):
        rho[1234] = bad
        st = lib.ofdft_tf_energy_potential_noalloc(ct.c_void_p(rho.data_ptr()), rho.numel(), 1.0, L.FP32_MIXED,
                                                   ct.c_void_p(E_dev.data_ptr()), None,
                                                   ct.c_void_p(stream.cuda_stream))
        assert st == L.OFDFT_OK
        torch.cuda.synchronize()
        assert np.isnan(float(E_dev)), bad
    rho[1234] = 0.01
    st = lib.ofdft_tf_energy_potential_noalloc(ct.c_void_p(rho.data_ptr()), rho.numel(), 1.0, L.FP32_MIXED,
                                               ct.c_void_p(E_dev.data_ptr()), None, ct.c_void_p(stream.cuda_stream))
    assert st == L.OFDFT_OK
    torch.cuda.synchronize()
    assert abs(float(E_dev) - 2.871234000188191 * 4096 * 0.01 ** (5.0 / 3.0)) <= 1e-6 * float(E_dev)
