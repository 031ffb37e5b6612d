"""ctypes binding of libibmschur (include/ibm_schur.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names; pointers are passed as integers (device
addresses, e.g. ``tensor.data_ptr()``).  Loading fails loudly when the shared
library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libibmschur.so"

IBM_OK = 0
IBM_ERR_ARG = 1
IBM_ERR_CUDA = 2
IBM_ERR_NOMEM = 3
IBM_ERR_NOT_CONVERGED = 4
IBM_ERR_BREAKDOWN = 5
IBM_ERR_NAN = 6
IBM_ERR_MARKER_DOMAIN = 7
IBM_ERR_STATE = 8
IBM_PREC_FP64 = 0
IBM_PREC_FP32 = 1
IBM_ARNOLDI_FP64 = 0
IBM_ARNOLDI_DS = 1
IBM_ARNOLDI_FP32 = 2
IBM_FSI_CRIT_LAGRANGIAN = 0
IBM_FSI_CRIT_EULERIAN = 1
IBM_CMODE_SCALAR = 0
IBM_CMODE_EXACT = 1
IBM_CMODE_CONSISTENT = 2
HIST_MAX = 256

STATUS_NAMES = {0: "IBM_OK", 1: "IBM_ERR_ARG", 2: "IBM_ERR_CUDA", 3: "IBM_ERR_NOMEM",
                4: "IBM_ERR_NOT_CONVERGED", 5: "IBM_ERR_BREAKDOWN", 6: "IBM_ERR_NAN",
                7: "IBM_ERR_MARKER_DOMAIN", 8: "IBM_ERR_STATE"}


class ibm_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("h", C.c_double), ("Re", C.c_double), ("dt", C.c_double)]


class ibm_solve_opts(C.Structure):
    _fields_ = [("precond_prec", C.c_int32), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("restart", C.c_int32), ("mg_pre", C.c_int32), ("mg_post", C.c_int32),
                ("reorth", C.c_int32), ("helm_rtol", C.c_double), ("helm_maxit", C.c_int32),
                ("with_advection", C.c_int32), ("arnoldi", C.c_int32), ("c_mode", C.c_int32),
                ("c_rtol", C.c_double), ("c_maxit", C.c_int32), ("cycle_graphs", C.c_int32)]


class ibm_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("relres_true", C.c_double),
                ("relres_hist", C.c_double * HIST_MAX), ("helm_iters", C.c_int32),
                ("helm_relres", C.c_double), ("div_l2", C.c_double), ("slip_l2", C.c_double),
                ("c_iters", C.c_int64), ("graph_cycles", C.c_int32)]


class ibm_rigid_sphere(C.Structure):
    _fields_ = [("radius", C.c_double), ("theta", C.c_double),
                ("xc", C.c_double * 3), ("xc_prev", C.c_double * 3),
                ("us", C.c_double * 3), ("us_prev", C.c_double * 3),
                ("om", C.c_double * 3), ("om_prev", C.c_double * 3),
                ("om_cs", C.c_double * 3), ("om_cs_prev", C.c_double * 3),
                ("rot", C.c_double * 9),
                ("mom", C.c_double * 3), ("mom_prev", C.c_double * 3),
                ("amom", C.c_double * 3), ("amom_prev", C.c_double * 3),
                ("free_motion", C.c_int32)]


class ibm_fsi_opts(C.Structure):
    _fields_ = [("gravity", C.c_double * 3), ("xi", C.c_double), ("tol", C.c_double),
                ("max_inner", C.c_int32), ("criterion", C.c_int32)]


class ibm_fsi_stats(C.Structure):
    _fields_ = [("inner", C.c_int32), ("fgmres_iters", C.c_int32), ("ratio", C.c_double),
                ("helm_iters", C.c_int32), ("helm_relres", C.c_double)]


PROF_NCLASS = 16
PROF_NAMES = ["laplacian_f64", "schur_markers", "vcycle", "multidot", "axpy_norm", "predictor",
              "solve", "step", "marker_build", "mg_smooth_fine", "helm_sweep", "adjoint", "fsi"]


class ibm_profile(C.Structure):
    _fields_ = [("ms", C.c_double * PROF_NCLASS), ("launches", C.c_int64 * PROF_NCLASS),
                ("bytes", C.c_double * PROF_NCLASS)]


_P = C.c_void_p
# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("ibm_default_opts", None, [C.POINTER(ibm_solve_opts)]),
    ("ibm_create", C.c_int, [C.POINTER(ibm_grid_desc), _P, C.POINTER(_P)]),
    ("ibm_destroy", None, [_P]),
    ("ibm_last_error", C.c_char_p, [_P]),
    ("ibm_num_cells", C.c_int64, [_P]),
    ("ibm_num_faces", C.c_int64, [_P]),
    ("ibm_set_markers", C.c_int, [_P, C.c_int64, _P]),
    ("ibm_apply_laplacian", C.c_int, [_P, _P, _P]),
    ("ibm_apply_schur", C.c_int, [_P, _P, _P]),
    ("ibm_apply_laplacian_precond", C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32]),
    ("ibm_interp", C.c_int, [_P, _P, _P]),
    ("ibm_spread", C.c_int, [_P, _P, _P]),
    ("ibm_gradient", C.c_int, [_P, _P, _P]),
    ("ibm_gradient_t", C.c_int, [_P, _P, _P]),
    ("ibm_solve_schur", C.c_int, [_P, _P, _P, C.POINTER(ibm_solve_opts),
                                  C.POINTER(ibm_solve_stats)]),
    ("ibm_force_correction", C.c_int, [_P, _P, _P, _P]),
    ("ibm_step", C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                           C.POINTER(ibm_solve_opts), C.POINTER(ibm_solve_stats)]),
    ("ibm_body_forces_noalloc", C.c_int, [_P, _P, _P, C.c_int64, C.c_int32,
                                          C.POINTER(C.c_double), C.c_double, _P,
                                          C.POINTER(C.c_double)]),
    ("ibm_profile_enable", C.c_int, [_P, C.c_int32]),
    ("ibm_kernel_launches", C.c_int64, []),
    ("ibm_profile_read", C.c_int, [_P, C.POINTER(ibm_profile)]),
    ("ibm_body_forces", C.c_int, [_P, _P, _P, _P, C.c_int32, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    ("ibm_apply_schur_opts", C.c_int, [_P, _P, _P, C.POINTER(ibm_solve_opts),
                                       C.POINTER(C.c_int64)]),
    ("ibm_apply_c_inverse", C.c_int, [_P, _P, _P, C.c_double, C.c_int32,
                                      C.POINTER(C.c_int32)]),
    ("ibm_default_fsi_opts", None, [C.POINTER(ibm_fsi_opts)]),
    ("ibm_fsi_step", C.c_int, [_P, C.c_int32, C.POINTER(ibm_rigid_sphere), C.c_int64, _P, _P,
                               _P, _P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(ibm_solve_opts),
                               C.POINTER(ibm_fsi_opts), C.POINTER(ibm_fsi_stats)]),
    ("ibm_adjoint_step", C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.POINTER(ibm_solve_opts),
                                   C.POINTER(ibm_solve_stats)]),
    ("ibm_body_forces_adjoint", C.c_int, [_P, _P, _P, _P, C.c_int32, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double), _P, _P,
                                          C.POINTER(C.c_double)]),
]

_lib = None


def load(path: str | Path | None = None):
    """Loads the shared library (once) and declares every signature."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(
            f"{p.name} is not built; run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = C.CDLL(str(p))
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx=None):
    if status != IBM_OK:
        msg = load().ibm_last_error(ctx).decode() if ctx else ""
        raise IBMError(status, msg)


def default_opts() -> ibm_solve_opts:
    o = ibm_solve_opts()
    load().ibm_default_opts(C.byref(o))
    return o
