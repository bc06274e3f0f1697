"""ctypes declarations of the C ABI in include/stokes_mf.h (argument marshalling only).

Loading fails loudly when libstokes_mf.so is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstokes_mf.so")

STATUS = {0: "STOKES_OK", 1: "STOKES_EINVAL", 2: "STOKES_ENOMEM", 3: "STOKES_ECUDA", 4: "STOKES_ENOTCONV",
          5: "STOKES_EBREAKDOWN", 6: "STOKES_ETIMEOUT"}


class StokesMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("n_levels", C.c_int), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("vertices", C.POINTER(C.c_double)), ("dirichlet_faces", C.c_uint)]


class StokesOpts(C.Structure):
    _fields_ = [("kA", C.c_int), ("kS", C.c_int), ("m", C.c_int), ("cycle", C.c_int), ("schur_diag", C.c_int),
                ("vcycle_fp32", C.c_int), ("gmres_restart", C.c_int), ("eig_iters", C.c_int),
                ("eig_safety", C.c_double), ("seed", C.c_ulonglong), ("c_mass", C.c_double),
                ("c_grad", C.c_double), ("sym_grad", C.c_int), ("rho_cell", C.POINTER(C.c_double)),
                ("deterministic", C.c_int), ("wait_cycles", C.c_uint)]


# name -> (restype, argtypes)
P = C.c_void_p
SIGNATURES = {
    "stokes_default_opts": (None, [C.POINTER(StokesOpts)]),
    "stokes_setup": (C.c_int, [C.POINTER(StokesMesh), C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double),
                               C.POINTER(StokesOpts), P, C.POINTER(P)]),
    "stokes_sizes": (C.c_int, [P, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "stokes_vmult": (C.c_int, [P, C.c_int, C.c_int, P, P, P]),
    "stokes_apply_blocks": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, P, P, P]),
    "stokes_mass_rhs": (C.c_int, [P, C.c_int, C.c_int, P, P, P]),
    "stokes_smooth": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, P]),
    "stokes_smooth_noalloc": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, P]),
    "stokes_transfer": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, P]),
    "stokes_coarse_solve": (C.c_int, [P, C.c_int, P, P, P]),
    "mg_vcycle": (C.c_int, [P, C.c_int, P, P, P]),
    "stokes_solve": (C.c_int, [P, P, P, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), P]),
    "stokes_solve_host": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double), P]),
    "stokes_get_level_params": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "stokes_get_diagonals": (C.c_int, [P, C.c_int, P, P, P]),
    "stokes_cell_grad": (C.c_int, [P, P, P, P, P]),
    "stokes_set_viscosity": (C.c_int, [P, C.POINTER(C.c_double), P]),
    "stokes_velocity_nodes": (C.c_int, [P, C.c_int, P, P]),
    "stokes_lift_rhs": (C.c_int, [P, P, P, P]),
    "stokes_mg_iterate": (C.c_int, [P, P, P, C.c_int, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), P]),
    "stokes_time_apply": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), P]),
    "stokes_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), P]),
    "stokes_get_launch_shape": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "stokes_get_smoother_fusion": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "stokes_setup_batch": (C.c_int, [C.c_int, C.POINTER(StokesMesh), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(StokesOpts), P, C.POINTER(P)]),
    "stokes_batch_context": (C.c_int, [P, C.c_int, C.POINTER(P)]),
    "stokes_solve_batch": (C.c_int, [P, C.POINTER(P), C.POINTER(P), C.c_double, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_double), P]),
    "stokes_batch_last_error": (C.c_char_p, [P]),
    "stokes_destroy_batch": (None, [P]),
    "stokes_set_launch_shape": (C.c_int, [P, C.c_int, C.c_int, C.c_int]),
    "stokes_get_geometry_stored": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "stokes_launch_count": (C.c_longlong, [P]),
    "stokes_krylov_mode": (C.c_int, [P]),
    "stokes_set_wait_cycles": (C.c_int, [P, C.c_uint]),
    "stokes_batch_krylov_mode": (C.c_int, [P]),
    "stokes_batch_set_wait_cycles": (C.c_int, [P, C.c_uint]),
    "stokes_batch_vcycle": (C.c_int, [P, C.POINTER(P), C.POINTER(P), P]),
    "stokes_last_error": (C.c_char_p, [P]),
    "stokes_global_last_error": (C.c_char_p, []),
    "stokes_destroy": (None, [P]),
}

_lib = None


def load(path=None):
    """Load (once) and declare the library.  Raises OSError if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} is not built; run `python -m paper_2205_15770_gb300.build` "
                      "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
