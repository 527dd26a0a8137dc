"""Failure paths of the C ABI, made on the host side (no GPU fault is ever provoked).

- Bounded device waits: with OFDFT_OPTION_WAIT_POLLS = 0 the first wait for the
  inverse rows' bulk copies gives up at once; the kernel lets its copies land with
  a second, longer bounded wait, flags the timeout and returns, so the call
  reports OFDFT_ERR_TIMEOUT and the grid's next call (normal polls) is correct.
- Allocation failure: an allocation cap makes the workspace allocation fail with
  OFDFT_ERR_OOM; lifting the cap makes the same call succeed.
- Optimiser: max_iter = 1 cannot meet the three-iteration stop rule (Sec. 2.4
  convergence reading), so the call reports OFDFT_ERR_NOT_CONVERGED with its
  report filled.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2002_02985_gb300 as ofd  # noqa: E402
from paper_2002_02985_gb300 import _lib as L  # noqa: E402


def _grid(name="fcc-al-4/32"):
    wl = W.workload(name)
    g = ofd.Grid(wl["cell"], wl["shape"])
    g.set_ions(wl["positions"], wl["species"], wl["Z"], wl["rc"])
    rho = torch.from_numpy(W.model_density(wl).astype(np.float32)).cuda()
    return wl, g, rho


def test_expired_bounded_wait_reports_timeout_and_the_grid_recovers():
    wl, g, rho = _grid()
    f = ofd.Functional(n_knots=wl["n_knots"])
    E0, V0 = g.energy_potential(rho, f)
    g.set_option(L.OPTION_WAIT_POLLS, 0)
    with pytest.raises(ofd.OFDFTError) as e:
        g.energy_potential(rho, f)
    assert e.value.status == L.OFDFT_ERR_TIMEOUT
    assert "copies may still" not in str(e.value)          # the copies landed (flag 1, not 2)
    g.set_option(L.OPTION_WAIT_POLLS, 1 << 22)
    E1, V1 = g.energy_potential(rho, f)
    assert E1 == E0
    assert torch.equal(V1, V0)


def test_allocation_cap_reports_oom_then_succeeds_without_it():
    wl, g, rho = _grid()
    f = ofd.Functional(n_knots=wl["n_knots"])
    g.set_option(L.OPTION_ALLOC_CAP, 64 * 1024)             # far below the channel workspace
    with pytest.raises(ofd.OFDFTError) as e:
        g.energy_potential(rho, f)
    assert e.value.status == L.OFDFT_ERR_OOM
    g.set_option(L.OPTION_ALLOC_CAP, 0)
    E, V = g.energy_potential(rho, f)
    assert np.isfinite(E["total"]) and bool(torch.isfinite(V).all())


def test_optimiser_reports_not_converged_with_a_filled_report():
    wl, g, rho = _grid()
    f = ofd.Functional(n_knots=wl["n_knots"])
    psi = rho.sqrt().contiguous()
    rep = g.optimize_density(psi, f, wl["n_electrons"], tol_per_atom=1e-6, max_iter=1, raise_on_not_converged=False)
    assert not rep["converged"]
    assert rep["iterations"] == 1 and rep["evaluations"] >= 2
    assert np.isfinite(rep["energy"])
    with pytest.raises(ofd.OFDFTError) as e:
        g.optimize_density(rho.sqrt().contiguous(), f, wl["n_electrons"], tol_per_atom=1e-6, max_iter=1,
                           raise_on_not_converged=True)
    assert e.value.status == L.OFDFT_ERR_NOT_CONVERGED


def test_unknown_options_are_rejected():
    wl, g, rho = _grid()
    for opt, val in ((99, 0), (L.OPTION_KERNELS, 7), (L.OPTION_WAIT_POLLS, -1), (L.OPTION_ALLOC_CAP, -5),
                     (L.OPTION_BATCH_GROUPED, 2)):
        with pytest.raises(ofd.OFDFTError) as e:
            g.set_option(opt, val)
        assert e.value.status == L.OFDFT_ERR_INVALID_ARG
