"""ctypes declarations of the C ABI in include/ofdft.h (argument marshalling only).

Loads the in-tree libofdft.so and raises if it is missing: there is no CPU
fallback; every step of the evaluation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libofdft.so")

OFDFT_OK = 0
OFDFT_ERR_INVALID_ARG = -1
STATUS = {0: "OFDFT_OK", -1: "OFDFT_ERR_INVALID_ARG", -2: "OFDFT_ERR_UNSUPPORTED_SIZE",
          -3: "OFDFT_ERR_BAD_DENSITY", -4: "OFDFT_ERR_OOM", -5: "OFDFT_ERR_CUDA",
          -6: "OFDFT_ERR_NOT_CONVERGED", -7: "OFDFT_ERR_NO_IONS", -8: "OFDFT_ERR_TIMEOUT"}

TERM_TF, TERM_VW, TERM_NL, TERM_HARTREE, TERM_PP, TERM_XC = 1, 2, 4, 8, 16, 32
TERMS_ALL = 31          # kinetic + electrostatic functional (the benchmark's)
TERMS_VALID = 63
N_ENERGIES = 7          # total, TF, vW, NL, H, PP, XC
KNOTS_LOG, KNOTS_ARITH = 0, 1
NLPOT_EXACT, NLPOT_INTERP = 0, 1
KERNEL_LWT, KERNEL_WT_GLOBAL = 0, 1
FP64, FP32_MIXED = 0, 1
OPT_CG, OPT_TN, OPT_LBFGS = 0, 1, 2
UPDATE_ROTATE, UPDATE_SCALE = 0, 1
OBJECTIVE_ENERGY, OBJECTIVE_RESIDUAL = 0, 1
OPTION_KERNELS, OPTION_BATCH_GRAPH, OPTION_WAIT_POLLS, OPTION_ALLOC_CAP = 1, 2, 3, 4
OPTION_PICK_ROWS, OPTION_PICK_PENCIL, OPTION_PICK_RECIP, OPTION_EXACT_SUMS = 5, 6, 7, 8
OPTION_BATCH_GROUPED = 9
KERNELS_AUTO, KERNELS_GENERIC, KERNELS_PER_CHANNEL_ROWS, KERNELS_TILE_RECIP = 0, 1, 2, 3
OFDFT_ERR_OOM = -4
OFDFT_ERR_NOT_CONVERGED = -6
OFDFT_ERR_TIMEOUT = -8

# symbols declared in include/ofdft.h (checked by the CPU test suite)
EXPORTS = (
    "ofdft_grid_create", "ofdft_grid_destroy", "ofdft_set_ions", "ofdft_energy_potential",
    "ofdft_energy_potential_async", "ofdft_forces", "ofdft_optimize_density",
    "ofdft_energy_potential_batched", "ofdft_status_string", "ofdft_last_error", "ofdft_version",
    "ofdft_profile_enable", "ofdft_profile_reset", "ofdft_profile_read",
    "ofdft_tf_energy_potential_noalloc", "ofdft_set_ions_pme", "ofdft_ewald", "ofdft_interpolate",
    "ofdft_optimize_density_multistep", "ofdft_optimize_density_ex", "ofdft_td_kick", "ofdft_td_propagate",
    "ofdft_td_spectrum", "ofdft_set_option", "ofdft_tuning_report", "ofdft_fp64_fma_rate", "ofdft_batch_report",
)
NOALLOC_MAX_POINTS = 8388608


class CFunctional(ct.Structure):
    _fields_ = [("terms", ct.c_uint), ("alpha", ct.c_double), ("beta", ct.c_double),
                ("n_knots", ct.c_int), ("knot_spacing", ct.c_int), ("knots", ct.POINTER(ct.c_double)),
                ("nl_potential", ct.c_int), ("kernel", ct.c_int), ("precision", ct.c_int),
                ("rho_floor", ct.c_double), ("mgp_x", ct.c_double), ("mgp_y", ct.c_double)]


class CSpecies(ct.Structure):
    _fields_ = [("n_species", ct.c_int), ("Z", ct.POINTER(ct.c_double)), ("rc", ct.POINTER(ct.c_double))]


class CIons(ct.Structure):
    _fields_ = [("n", ct.c_int), ("pos", ct.POINTER(ct.c_double)), ("species", ct.POINTER(ct.c_int))]


class COptReport(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("evaluations", ct.c_int), ("energy", ct.c_double),
                ("energies", ct.c_double * N_ENERGIES), ("mu", ct.c_double), ("residual", ct.c_double),
                ("last_dE", ct.c_double)]


class COptOptions(ct.Structure):
    _fields_ = [("method", ct.c_int), ("precondition", ct.c_int), ("max_inner", ct.c_int), ("lbfgs_m", ct.c_int),
                ("update", ct.c_int), ("objective", ct.c_int)]


class CTdOptions(ct.Structure):
    _fields_ = [("dt", ct.c_double), ("n_steps", ct.c_int), ("n_corrector", ct.c_int), ("solver_tol", ct.c_double),
                ("max_solver_iter", ct.c_int)]


class CTdReport(ct.Structure):
    _fields_ = [("steps", ct.c_int), ("evaluations", ct.c_int), ("solver_iterations", ct.c_int),
                ("max_residual", ct.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Load libofdft.so (raises OSError with a clear message when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(path)
    P, I, D, V = ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p
    lib.ofdft_grid_create.argtypes = [ct.POINTER(D), ct.POINTER(I), P, ct.POINTER(P)]
    lib.ofdft_grid_destroy.argtypes = [P]
    lib.ofdft_set_ions.argtypes = [P, ct.POINTER(CIons), ct.POINTER(CSpecies)]
    lib.ofdft_set_ions_pme.argtypes = [P, ct.POINTER(CIons), ct.POINTER(CSpecies), I]
    lib.ofdft_energy_potential.argtypes = [P, V, ct.POINTER(CFunctional), ct.POINTER(D), V]
    lib.ofdft_energy_potential_async.argtypes = [P, V, ct.POINTER(CFunctional), V, V]
    lib.ofdft_forces.argtypes = [P, V, I, ct.POINTER(D)]
    lib.ofdft_ewald.argtypes = [P, ct.POINTER(D), ct.POINTER(D)]
    lib.ofdft_interpolate.argtypes = [P, V, P, V, I]
    lib.ofdft_optimize_density_multistep.argtypes = [I, ct.POINTER(P), V, ct.POINTER(CFunctional), D, D, I,
                                                     ct.POINTER(COptReport)]
    lib.ofdft_optimize_density.argtypes = [P, V, ct.POINTER(CFunctional), D, D, I, ct.POINTER(COptReport)]
    lib.ofdft_optimize_density_ex.argtypes = [P, V, ct.POINTER(CFunctional), D, D, I, ct.POINTER(COptOptions),
                                              ct.POINTER(COptReport)]
    lib.ofdft_td_kick.argtypes = [P, V, V, ct.POINTER(D), I]
    lib.ofdft_td_propagate.argtypes = [P, V, V, V, ct.POINTER(CFunctional), ct.POINTER(CTdOptions), ct.POINTER(D),
                                       ct.POINTER(CTdReport)]
    lib.ofdft_td_spectrum.argtypes = [ct.POINTER(D), I, D, D, I, ct.POINTER(D), ct.POINTER(D)]
    lib.ofdft_energy_potential_batched.argtypes = [I, ct.POINTER(P), ct.POINTER(V), ct.POINTER(CFunctional),
                                                   ct.POINTER(D), ct.POINTER(V), ct.POINTER(ct.POINTER(D))]
    lib.ofdft_profile_enable.argtypes = [P, I]
    lib.ofdft_profile_reset.argtypes = [P]
    lib.ofdft_profile_read.argtypes = [P, I, ct.POINTER(ct.c_char_p), ct.POINTER(I), ct.POINTER(D)]
    lib.ofdft_tf_energy_potential_noalloc.argtypes = [V, ct.c_longlong, D, I, V, V, P]
    lib.ofdft_set_option.argtypes = [P, I, ct.c_longlong]
    lib.ofdft_fp64_fma_rate.argtypes = [P, ct.POINTER(D)]
    lib.ofdft_tuning_report.argtypes = [P, I]
    lib.ofdft_tuning_report.restype = ct.c_char_p
    lib.ofdft_batch_report.argtypes = [P]
    lib.ofdft_batch_report.restype = ct.c_char_p
    lib.ofdft_status_string.argtypes = [I]
    lib.ofdft_status_string.restype = ct.c_char_p
    lib.ofdft_last_error.argtypes = [P]
    lib.ofdft_last_error.restype = ct.c_char_p
    lib.ofdft_version.restype = ct.c_char_p
    for name in EXPORTS:
        if name not in ("ofdft_status_string", "ofdft_last_error", "ofdft_version", "ofdft_tuning_report",
                        "ofdft_batch_report"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib
