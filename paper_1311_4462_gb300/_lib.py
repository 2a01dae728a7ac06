"""ctypes declarations for libtm.so (the C ABI in include/tm.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtm.so")

TM_OK, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_NOCONV, TM_ERR_NAN, TM_ERR_TIMEOUT, TM_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "TM_OK", -1: "TM_ERR_ARG", -2: "TM_ERR_CUDA", -3: "TM_ERR_NOCONV", -4: "TM_ERR_NAN",
                -5: "TM_ERR_TIMEOUT", -6: "TM_ERR_NOMEM"}
TM_TWIST_PLUS, TM_TWIST_MINUS, TM_NDEG_DOUBLET = 1, -1, 2
TM_PREC_F64, TM_PREC_F32, TM_PREC_F16, TM_PREC_DF64 = 8, 4, 2, 16
TM_PC_ASYM, TM_PC_SYM = 0, 1
TM_C128, TM_C64 = 0, 1
TM_EPI_NONE, TM_EPI_TWINV, TM_EPI_TWXPAY_ASYM, TM_EPI_TWXPAY_SYM, TM_EPI_XPAY, TM_EPI_TWINV_XPAY, TM_EPI_XMAY_K2 = range(7)
TM_SOLVER_CG, TM_SOLVER_MIXED = 0, 1
TM_SOLUTION_MAT, TM_SOLUTION_MATDAG_MAT = 0, 1
TM_DD_ALL, TM_DD_INTERIOR, TM_DD_BOUNDARY = 0, 1, 2
TM_GAUGE_F64_FULL_LINKS = 16


class tm_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("mu", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("flavor", ctypes.c_int), ("t_antiperiodic", ctypes.c_int),
                ("recon", ctypes.c_int)]


class tm_field(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("norm", ctypes.c_void_p), ("prec", ctypes.c_int), ("nrhs", ctypes.c_int)]


class tm_solver_params(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("solution", ctypes.c_int), ("pc", ctypes.c_int), ("dagger", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("delta", ctypes.c_double),
                ("sloppy_prec", ctypes.c_int), ("use_x0", ctypes.c_int), ("want_pc_residual", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("true_prec", ctypes.c_int)]


class tm_solver_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_residual", ctypes.c_double),
                ("pc_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


class TMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
vp = ctypes.c_void_p
FP = ctypes.POINTER(tm_field)

# name -> argtypes (restype is tm_status = int unless noted)
_SIGS = {
    "tm_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    "tm_gauge_create": [ctypes.POINTER(tm_params), vp, vp, ctypes.POINTER(vp)],
    "tm_gauge_create_ex": [ctypes.POINTER(tm_params), vp, ctypes.c_int, vp, ctypes.POINTER(vp)],
    "tm_gauge_destroy": [vp],
    "tm_field_bytes": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                       ctypes.POINTER(ctypes.c_size_t)],
    "tm_field_upload": [vp, FP, vp, vp, vp],
    "tm_field_download": [vp, vp, vp, FP, vp],
    "tm_pack": [vp, FP, vp, ctypes.c_int, ctypes.c_int, vp],
    "tm_unpack": [vp, vp, ctypes.c_int, FP, ctypes.c_int, vp],
    "tm_dslash": [vp, FP, FP, ctypes.c_int, ctypes.c_int, FP, vp],
    "tm_dslash_dagger": [vp, FP, FP, ctypes.c_int, ctypes.c_int, FP, vp],
    "tm_precond_op": [vp, FP, FP, FP, ctypes.c_int, ctypes.c_int, vp],
    "tm_mat": [vp, FP, FP, FP, FP, ctypes.c_int, vp],
    "tm_normal_op": [vp, FP, FP, FP, FP, ctypes.c_int, ctypes.c_int, vp],
    "tm_prepare_rhs": [vp, FP, FP, FP, ctypes.c_int, ctypes.c_int, vp],
    "tm_reconstruct_odd": [vp, FP, FP, FP, ctypes.c_int, vp],
    "tm_twist": [vp, FP, FP, ctypes.c_int, ctypes.c_int, vp],
    "tm_solve_workspace_bytes": [vp, ctypes.POINTER(tm_solver_params), ctypes.POINTER(ctypes.c_size_t)],
    "tm_solve": [vp, FP, FP, ctypes.POINTER(tm_solver_params), ctypes.POINTER(tm_solver_stats), vp, ctypes.c_size_t,
                 vp],
    "tm_norm2": [vp, FP, ctypes.POINTER(ctypes.c_double), vp],
    "tm_dot": [vp, FP, FP, ctypes.POINTER(ctypes.c_double), vp],
    "tm_axpby": [vp, FP, ctypes.c_double, FP, ctypes.c_double, FP, vp],
    "tm_force": [vp, vp, ctypes.c_int, FP, FP, FP, FP, ctypes.c_double, ctypes.c_int, vp],
    "tm_norm2_noalloc": [FP, ctypes.c_int, ctypes.c_int, vp, vp],
    "tm_autotune": [vp, vp],
    "tm_precond_op_active": [vp, FP, FP, FP, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp],
    "tm_solve_multi_workspace_bytes": [vp, ctypes.POINTER(tm_solver_params), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_size_t)],
    "tm_solve_multi": [vp, FP, FP, ctypes.POINTER(tm_solver_params), ctypes.POINTER(tm_solver_stats), vp,
                       ctypes.c_size_t, vp],
    "tm_noise_z2": [vp, FP, ctypes.c_int, ctypes.c_ulonglong, vp],
    "tm_g5dot": [vp, FP, FP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp],
    "tm_tune_export": [vp, ctypes.c_char_p, ctypes.c_size_t],
    "tm_tune_import": [vp, ctypes.c_char_p],
    "tm_gauge_set_clover": [vp, ctypes.c_double, vp],
    "tm_local_op": [vp, FP, FP, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp],
    "tm_device_status": [vp, vp],
    "tm_fused_work_list": [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int],
    "tm_fused_set_work_list": [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_ulonglong, vp],
    "tm_gauge_set_partition": [vp, ctypes.c_int, ctypes.c_int],
    "tm_dd_face_bytes": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
    "tm_dd_pack_faces": [vp, vp, vp, FP, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp],
    "tm_dd_dslash": [vp, FP, FP, ctypes.c_int, ctypes.c_int, FP, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp],
}


def load():
    """Load libtm.so.  There is no fallback: a missing or stale library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtm.so is not built ({LIB_PATH}); run paper_1311_4462_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    lib.tm_version.restype = ctypes.c_char_p
    lib.tm_version.argtypes = []
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().tm_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int):
    if status != TM_OK:
        raise TMError(status, last_error())
    return status


def exported_names():
    return ["tm_version"] + list(_SIGS)
