"""Plain FP64 CPU oracle of the OFDFT energy/potential path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.
It shares no code with the GPU path: it uses numpy (FP64) and ``numpy.fft``
as its only library primitives and follows the paper's definitions step by
step, without blocking, fusion or reordering.

Modules
-------
grid        reciprocal lattice, half-spectrum FFT conventions (Sec. 2.1 Grid/Field)
lindhard    Lindhard function and the WT kernel G_NL (Eq. WT and the G_NL definition)
functionals Thomas-Fermi, von Weizsaecker (psi form), Hartree, local PP,
            nonlocal LWT KEDF with the s1-s4 spline scheme, global-kF WT
evaluate    total energy and potential E[rho], V = dE/drho (Eqs. efunc, euler)
forces      ionic forces -dE/dR_I of the electron-ion term
optimize    psi = sqrt(rho) conjugate-gradient density optimiser (Eq. euler2)

Parity status: every function is pinned by the `-m "not gpu"` tests in
tests/test_oracle_*.py except the optimiser trajectory (parity unpinned:
the line search is a reading of the paper, only the converged energy is
compared).
"""
