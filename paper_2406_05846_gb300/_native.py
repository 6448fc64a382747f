"""ctypes declarations of the C ABI in include/strom.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstrom.so")

STROM_OK, STROM_MAXITER, STROM_PENDING = 0, 1, 2
STROM_ERR_INVALID, STROM_ERR_OOM, STROM_ERR_NOT_PD, STROM_ERR_NUMERICAL, STROM_ERR_TIMEOUT, STROM_ERR_CUDA = (
    -1, -2, -3, -4, -5, -6)
STROM_PREC_FP64, STROM_PREC_FP32, STROM_PREC_MIXED = 0, 1, 2
STROM_FACTOR_AUTO, STROM_FACTOR_DENSE, STROM_FACTOR_SPARSE = 0, 1, 2
STROM_WARM_MAX_KEY = 8


class strom_poly(C.Structure):
    _fields_ = [("nterms", C.c_int32), ("coef", C.POINTER(C.c_double)), ("expo", C.POINTER(C.c_uint8))]


class strom_clique(C.Structure):
    _fields_ = [("f", strom_poly), ("ng", C.c_int32), ("g", C.POINTER(strom_poly)),
                ("nh", C.c_int32), ("h", C.POINTER(strom_poly))]


class strom_problem_desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("dx", C.c_int32), ("du", C.c_int32), ("kappa", C.c_int32),
                ("R", C.c_double), ("cliques", C.POINTER(strom_clique))]


class strom_sdp_info(C.Structure):
    _fields_ = [("N", C.c_int32), ("nv", C.c_int32), ("nblocks", C.c_int32), ("nsvec", C.c_int64),
                ("m", C.c_int64), ("nnz", C.c_int64), ("rows_by_kind", C.c_int64 * 5)]


class strom_sdp_desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("dx", C.c_int32), ("du", C.c_int32), ("nblocks", C.c_int32),
                ("block_n", C.POINTER(C.c_int32)), ("block_kind", C.POINTER(C.c_int8)),
                ("block_clique", C.POINTER(C.c_int32)), ("block_index", C.POINTER(C.c_int32)),
                ("C", C.POINTER(C.c_double)), ("m", C.c_int64), ("rowptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("row_kind", C.POINTER(C.c_int8)), ("row_clique", C.POINTER(C.c_int32))]


class strom_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int32), ("sigma0", C.c_double), ("tau", C.c_double),
                ("sigma_every", C.c_int32), ("sigma_ratio", C.c_double), ("sigma_factor", C.c_double),
                ("sigma_min", C.c_double), ("sigma_max", C.c_double), ("rank_tol", C.c_double),
                ("precision", C.c_int32), ("polish_eta", C.c_double), ("check_every", C.c_int32),
                ("time_budget_s", C.c_double), ("eig_warm_period", C.c_int32),
                ("share_tail", C.c_int32), ("factor", C.c_int32), ("eig_reorth", C.c_int32)]


class strom_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("pobj", C.c_double), ("dobj", C.c_double),
                ("eta_p", C.c_double), ("eta_d", C.c_double), ("eta_g", C.c_double), ("sigma", C.c_double),
                ("m_kept", C.c_int64)]


class strom_certificate(C.Structure):
    _fields_ = [("max_ratio", C.c_double), ("lower_bound", C.c_double), ("phat", C.c_double), ("xi", C.c_double),
                ("hmax", C.c_double), ("gmin", C.c_double), ("feasible", C.c_int32), ("rank_one", C.c_int32),
                ("certified", C.c_int32)]


class strom_factor_info(C.Structure):
    _fields_ = [("n_other", C.c_int64), ("n_tail", C.c_int64), ("nnz_S", C.c_int64), ("nnz_L", C.c_int64),
                ("dense_entries", C.c_int64), ("levels_fwd", C.c_int32), ("levels_bwd", C.c_int32),
                ("max_group", C.c_int32), ("max_col", C.c_int32), ("max_span", C.c_int32)]


class strom_rank_test(C.Structure):
    _fields_ = [("n", C.c_int32), ("rank", C.c_int32), ("rank_low", C.c_int32), ("flat", C.c_int32),
                ("n_sub", C.c_int32), ("ratio_sub", C.c_double), ("lambda_max", C.c_double)]


P = C.c_void_p
PD = C.POINTER(C.c_double)
PI32 = C.POINTER(C.c_int32)
PI64 = C.POINTER(C.c_int64)
PI8 = C.POINTER(C.c_int8)
PU8 = C.POINTER(C.c_uint8)

# name: (restype, argtypes)
class strom_server_class(C.Structure):
    _fields_ = [("N", C.c_int32), ("shared_tail", C.c_int32), ("nsvec", C.c_int64), ("m", C.c_int64),
                ("slots", C.c_int32), ("running", C.c_int32), ("queued", C.c_int32), ("waiting", C.c_int32),
                ("batches_created", C.c_int32), ("pad", C.c_int32), ("slot_bytes", C.c_int64),
                ("reserved_bytes", C.c_int64)]


class strom_tune_report(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("tile", C.c_int32 * 4), ("ms", C.c_double * 4), ("chosen", C.c_int32),
                ("eig_threads", (C.c_int32 * 4) * 2), ("eig_ms", (C.c_double * 4) * 2)]


SIGNATURES = {
    "strom_last_error": (C.c_char_p, []),
    "strom_version": (C.c_char_p, []),
    "strom_problem_create": (C.c_int, [C.POINTER(strom_problem_desc), C.POINTER(P)]),
    "strom_problem_destroy": (None, [P]),
    "strom_relax": (C.c_int, [P, C.POINTER(P)]),
    "strom_sdp_info_get": (C.c_int, [P, C.POINTER(strom_sdp_info)]),
    "strom_sdp_export": (C.c_int, [P, PI32, PI64, PI8, PI32, PD, PI64, PI32, PD, PD, PI8, PI32]),
    "strom_sdp_destroy": (None, [P]),
    "strom_sdp_import": (C.c_int, [C.POINTER(strom_sdp_desc), C.POINTER(P)]),
    "strom_sdp_factor_info": (C.c_int, [P, C.POINTER(strom_factor_info)]),
    "strom_sdp_star_export": (C.c_int, [P, PI64, PI64, PI64, PD, PD, PI32, PI64, PD, PD, PD]),
    "strom_options_default": (None, [C.POINTER(strom_options)]),
    "strom_solver_create": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(strom_options), C.POINTER(P)]),
    "strom_solver_destroy": (None, [P]),
    "strom_solver_count": (C.c_int32, [P]),
    "strom_solve": (C.c_int, [P, P]),
    "strom_solver_factor": (C.c_int, [P, P]),
    "strom_certify_batch": (C.c_int, [P, C.POINTER(P), C.c_double, C.c_double, C.POINTER(strom_certificate)]),
    "strom_moment_rank_test": (C.c_int, [PD, C.c_int32, PU8, C.c_double, C.POINTER(strom_rank_test), PD]),
    "strom_launch_count": (C.c_uint64, []),
    "strom_transfer_bytes": (None, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "strom_solver_step": (C.c_int, [P, C.c_int32, P, PI32]),
    "strom_solver_reset": (C.c_int, [P, C.c_int32, PD, PD, C.c_double]),
    "strom_get_result": (C.c_int, [P, C.c_int32, C.POINTER(strom_result)]),
    "strom_get_state": (C.c_int, [P, C.c_int32, PD, PD, PD]),
    "strom_get_moment": (C.c_int, [P, C.c_int32, C.c_int32, PD]),
    "strom_get_kept_rows": (C.c_int, [P, C.c_int32, PU8]),
    "strom_certify": (C.c_int, [P, C.c_int32, P, C.c_double, C.c_double, C.POINTER(strom_certificate), PD, PD]),
    "strom_certify_host": (C.c_int, [P, C.c_int32, PI32, C.POINTER(C.c_int8), PI32, PD, PD, PD, C.c_double,
                                     C.c_double, C.c_double, C.POINTER(strom_certificate), PD, PD]),
    "strom_solver_nsvec_total": (C.c_int64, [P]),
    "strom_solver_m_total": (C.c_int64, [P]),
    "strom_solver_offsets": (C.c_int, [P, C.c_int32, PI64, PI64]),
    "strom_kernel_A": (C.c_int, [P, P, P, P]),
    "strom_kernel_At": (C.c_int, [P, P, P, P]),
    "strom_kernel_solve": (C.c_int, [P, P, P, P]),
    "strom_solver_tune": (C.c_int, [P, C.c_int32, P, C.POINTER(strom_tune_report)]),
    "strom_batch_create": (C.c_int, [P, C.c_int32, C.POINTER(strom_options), C.POINTER(P)]),
    "strom_solver_factor_kind": (C.c_int32, [P]),
    "strom_kernel_spmv_csr": (C.c_int, [P, P, P, C.c_int64, P, P, P]),
    "strom_batch_slot_bytes": (C.c_int, [P, C.POINTER(strom_options), PI64, PI64, PI64]),
    "strom_server_create": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(strom_options), C.POINTER(P)]),
    "strom_server_destroy": (None, [P]),
    "strom_server_submit": (C.c_int, [P, P, P, C.POINTER(C.c_uint64)]),
    "strom_server_step": (C.c_int, [P, C.c_int32, P, PI32, PI32]),
    "strom_server_poll": (C.c_int, [P, C.c_uint64, C.POINTER(strom_result), C.POINTER(strom_certificate),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "strom_server_info": (C.c_int, [P, C.c_int32, C.POINTER(strom_server_class), PI32, PI64]),
    "strom_batch_create_budget": (C.c_int, [P, C.c_int64, C.POINTER(strom_options), C.POINTER(P), PI32]),
    "strom_batch_destroy": (None, [P]),
    "strom_batch_submit": (C.c_int, [P, P, P, PD, PD, C.POINTER(C.c_uint64)]),
    "strom_batch_step": (C.c_int, [P, C.c_int32, P, PI32, PI32]),
    "strom_batch_poll": (C.c_int, [P, C.c_uint64, C.POINTER(strom_result), C.POINTER(strom_certificate),
                                   PD, PD]),
    "strom_warm_select": (C.c_int, [PD, C.c_int32, C.c_int32, PD, PI32, PD, PI32]),
    "strom_warm_create": (C.c_int, [C.c_int32, C.c_int64, C.c_int32, C.POINTER(P)]),
    "strom_warm_destroy": (None, [P]),
    "strom_warm_count": (C.c_int32, [P]),
    "strom_warm_add": (C.c_int, [P, PD, PD, PD, C.c_double, PI32]),
    "strom_warm_add_from_solver": (C.c_int, [P, P, C.c_int32, PD, PI32]),
    "strom_warm_query": (C.c_int, [P, PD, PI32, PD, PI32]),
    "strom_warm_get": (C.c_int, [P, C.c_int32, PD, PD, PD, PD]),
    "strom_solver_warm_start": (C.c_int, [P, C.c_int32, P, PD]),
    "strom_batch_set_warm": (C.c_int, [P, P, C.c_int32]),
    "strom_batch_submit_keyed": (C.c_int, [P, P, P, PD, C.POINTER(C.c_uint64)]),
    "strom_psd_plan_create": (C.c_int, [PI64, PI32, C.c_int32, C.c_int32, C.POINTER(P)]),
    "strom_psd_plan_destroy": (None, [P]),
    "strom_psd_execute": (C.c_int, [P, P, P, P, P]),
    "strom_kernel_psd_project": (C.c_int, [P, PI64, PI32, C.c_int32, C.c_int32, P, P]),
    "strom_kernel_psd_project_noalloc": (C.c_int, [P, PI64, PI32, C.c_int32, C.c_int32, P, P]),
}

_lib = None


def lib():
    """Load libstrom.so (built in-tree). Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libstrom.so is not built; run paper_2406_05846_gb300.build.build() "
                               "(the CUDA library is required, there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class StromError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().strom_last_error().decode(errors="replace")
        super().__init__("%s failed with status %d: %s" % (where, status, msg))
        self.status = status


def check(status, where):
    if status < 0:
        raise StromError(status, where)
    return status
