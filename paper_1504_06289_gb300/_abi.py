"""ctypes prototypes for libcpc.so (declared in include/cpc.h)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpc.so")

CPC_OK = 0
PRECISION = {"fp64": 0, "fp32": 1, "split": 2, "fp64tc": 3}
KIND = {"conv": 0, "master": 1}

vp, sz, i32, f64 = C.c_void_p, C.c_size_t, C.c_int, C.c_double
P_i32, P_f64 = C.POINTER(C.c_int), C.POINTER(C.c_double)

PROTOTYPES = {
    "make_newton_kernel": (i32, [i32, f64, i32, i32, vp, C.POINTER(vp)]),
    "make_newton_kernel_tables": (i32, [i32, f64, i32, i32, vp, vp, vp, P_f64, P_f64]),
    "cpc_kernel_info": (i32, [vp, P_i32, P_f64, P_i32, P_i32, P_i32, P_f64, P_f64]),
    "cpc_kernel_tables": (i32, [vp, vp, vp, vp]),
    "cpc_kernel_free": (i32, [vp]),
    "cpc_kernel_set_conv_paths": (i32, [vp, i32, i32, i32, i32, vp]),
    "cpc_kernel_conv_paths": (i32, [vp, i32, vp, vp]),
    "make_newton_kernel_paths": (i32, [i32, f64, i32, i32, i32, i32, i32, vp, vp, vp]),
    "make_newton_kernel_eh_plan": (i32, [i32, f64, i32, i32, i32, i32, i32, vp]),
    "cp_sample_gaussians": (i32, [i32, f64, i32, vp, vp, vp, vp]),
    "cp_hadamard_pairs": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
    "cp_convolve_workspace": (sz, [vp, i32, i32]),
    "cp_convolve": (i32, [vp, i32, vp, vp, i32, vp, sz, vp]),
    "cp_factor_spectra": (i32, [vp, i32, vp, vp, i32, vp]),
    "cp_convolve_from_spectra": (i32, [vp, i32, vp, vp, i32, vp]),
    "cp_hartree_energy_from_spectra_workspace": (sz, [vp, i32]),
    "cp_hartree_energy_from_spectra": (i32, [vp, i32, vp, vp, vp, vp, i32, vp, sz, vp]),
    "cp_hartree_energy_workspace": (sz, [vp, i32, i32]),
    "cp_hartree_energy": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]),
    "cp_hartree_energy_from_factors_workspace": (sz, [vp, i32, i32]),
    "cp_hartree_energy_from_factors": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]),
    "cp_hartree_energy_noalloc": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp]),
    "cp_hartree_energy_adjoint": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp]),
    "cp_gaussian_param_grad": (i32, [i32, f64, i32, vp, vp, vp, vp, vp, vp, vp]),
    "coulomb_matrix_workspace": (sz, [vp, i32, i32, i32, i32]),
    "coulomb_matrix": (i32, [vp, i32, vp, i32, vp, vp, i32, vp, vp, vp, vp, i32, i32, vp, sz, vp]),
    "coulomb_matrix_tune": (i32, [vp, i32, vp, i32, vp, vp, i32, vp, vp, vp, vp, i32, vp, sz, vp,
                                  C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "lattice_potential_sum": (i32, [vp, vp, vp, vp, i32, vp, vp, i32, vp]),
    "lattice_interaction_energy": (i32, [vp, vp, vp, f64, vp, vp]),
    "nuclear_matrix_workspace": (sz, [vp, i32, i32, i32, i32]),
    "tei_cholesky_workspace": (sz, [vp, i32, i32]),
    "tei_cholesky": (i32, [vp, i32, vp, i32, vp, vp, f64, f64, i32, i32, vp, vp, vp, sz, vp]),
    "tei_coulomb": (i32, [i32, i32, vp, vp, i32, vp, vp, vp, vp, vp, sz, vp]),
    "tei_exchange_workspace": (sz, [i32, i32]),
    "tei_exchange": (i32, [i32, i32, vp, vp, i32, vp, vp, vp, vp, vp, sz, vp]),
    "nuclear_matrix": (i32, [vp, i32, vp, i32, vp, vp, i32, vp, vp, vp, vp, i32, vp, sz, vp]),
    "cpc_kernel_timing": (i32, [i32]),
    "cpc_kernel_timing_read": (i32, [C.c_char_p, P_f64, P_i32]),
    "cpc_status_string": (C.c_char_p, [i32]),
    "cpc_last_error": (C.c_char_p, []),
}

_lib = None


class CpcError(RuntimeError):
    pass


def load() -> C.CDLL:
    """Load libcpc.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CpcError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1504_06289_gb300.build` (nvcc, sm_103a)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, what: str) -> None:
    if status != CPC_OK:
        lib = load()
        msg = lib.cpc_last_error().decode()
        raise CpcError(f"{what}: {lib.cpc_status_string(status).decode()} ({status}): {msg}")
