"""ctypes declarations of the C ABI in include/tt_sdp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libttsdp.so")

c_int32 = ctypes.c_int32
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p
P_int32 = ctypes.POINTER(c_int32)
P_double = ctypes.POINTER(c_double)


class ContractDims(ctypes.Structure):
    _fields_ = [("rw", c_int32), ("rw2", c_int32), ("R", c_int32), ("R2", c_int32),
                ("rv", c_int32), ("rv2", c_int32), ("m", c_int32), ("n", c_int32)]


class TTDesc(ctypes.Structure):
    _fields_ = [("d", c_int32), ("ranks", P_int32), ("m", c_int32), ("n", c_int32), ("cores", c_void_p)]


class Problem(ctypes.Structure):
    _fields_ = [("C", TTDesc), ("A_eq", TTDesc), ("B_eq", TTDesc), ("K_y", TTDesc),
                ("A_ineq", TTDesc), ("B_ineq", TTDesc), ("K_t", TTDesc), ("ones_t", TTDesc),
                ("ineq_sign", c_int32), ("q", ctypes.c_int64), ("lam0", c_double), ("lam0_ineq", c_double)]


class Options(ctypes.Structure):
    _fields_ = [("eps_gap", c_double), ("rank_cap", c_int32), ("xz_warmup", c_int32),
                ("eta0", c_double), ("eta_floor", c_double), ("eta_C", c_double), ("damping", c_double),
                ("precision", c_int32), ("max_iters", c_int32), ("max_sweeps", c_int32), ("kick", c_int32),
                ("eig_rank", c_int32), ("eig_sweeps", c_int32), ("seed", ctypes.c_uint64),
                ("local_dense_max", c_int32), ("gmres_restart", c_int32), ("gmres_max_iters", c_int32),
                ("eig_two_site", c_int32), ("time_limit", c_double), ("combined_multipliers", c_int32),
                ("finish_tol", c_double), ("nu0", c_double), ("nu_max", c_double), ("refine_sweeps", c_int32),
                ("fp32_factors", c_int32)]


class IterInfo(ctypes.Structure):
    _fields_ = [("iter", c_int32), ("converged", c_int32), ("mu", c_double), ("rel_p", c_double),
                ("rel_d", c_double), ("rel_gap", c_double), ("pobj", c_double), ("dobj", c_double),
                ("alpha_p", c_double), ("alpha_d", c_double), ("max_rank_X", c_int32), ("max_rank_Z", c_int32),
                ("max_rank_W", c_int32), ("sweeps", c_int32), ("direction", c_int32), ("seconds", c_double),
                ("gmres_iters", ctypes.c_int64), ("pred_used", ctypes.c_int64), ("pred_fallbacks", ctypes.c_int64),
                ("forcing", c_double), ("forcing_corrections", ctypes.c_int64), ("damped_retries", ctypes.c_int64),
                ("xz_fallbacks", ctypes.c_int64), ("finishing", c_int32), ("accepted", c_int32), ("nu", c_double),
                ("merit", c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("iters", c_int32), ("pobj", c_double), ("dobj", c_double),
                ("rel_gap", c_double), ("rel_p", c_double), ("rel_d", c_double), ("seconds", c_double)]


# name -> (restype, argtypes); every symbol declared in include/tt_sdp.h
SIGNATURES = {
    "tt_env_left_step": (c_int32, [ctypes.POINTER(ContractDims), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_int32, c_void_p]),
    "tt_env_right_step": (c_int32, [ctypes.POINTER(ContractDims), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_int32, c_void_p]),
    "tt_env_left_step_noalloc": (c_int32, [ctypes.POINTER(ContractDims), c_void_p, c_void_p, c_void_p, c_void_p,
                                           c_void_p, c_void_p]),
    "tt_local_apply": (c_int32, [ctypes.POINTER(ContractDims), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_int32, c_void_p]),
    "tt_local_matrix": (c_int32, [ctypes.POINTER(ContractDims), c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                  c_void_p]),
    "tt_core_count": (c_size_t, [c_int32, P_int32, c_int32, c_int32]),
    "tt_hadamard": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc), c_void_p, c_void_p]),
    "tt_matvec": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc), c_void_p, c_void_p]),
    "tt_inner": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc), P_double, c_void_p]),
    "tt_min_gen_eig": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc), c_int32, c_int32, c_int32,
                                 ctypes.c_uint64, P_double, c_void_p]),
    "tt_round": (c_int32, [ctypes.POINTER(TTDesc), c_double, c_int32, P_int32, c_void_p, c_size_t, P_double,
                           c_int32, c_void_p]),
    "tt_from_dense": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_int32, P_int32, c_void_p,
                                ctypes.POINTER(c_size_t), c_void_p]),
    "tt_sdp_default_options": (None, [ctypes.POINTER(Options)]),
    "tt_sdp_create": (c_int32, [ctypes.POINTER(Problem), ctypes.POINTER(Options), ctypes.POINTER(Allocator), c_void_p,
                                ctypes.POINTER(c_void_p)]),
    "tt_sdp_create_batch": (c_int32, [c_int32, ctypes.POINTER(Problem), ctypes.POINTER(Options),
                                      ctypes.POINTER(Allocator), c_void_p, ctypes.POINTER(c_void_p)]),
    "tt_sdp_batch_size": (c_int32, [c_void_p]),
    "tt_sdp_batch_member": (c_void_p, [c_void_p, c_int32]),
    "tt_lu_solve": (c_int32, [c_int32, c_void_p, c_void_p, c_int32, P_double, c_void_p]),
    "tt_kkt_solve": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_int32, P_double, c_void_p]),
    "tt_kkt_stats": (None, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), c_int32]),
    "tt_sdp_round": (c_int32, [ctypes.POINTER(TTDesc), c_double, c_int32, c_int32, ctypes.POINTER(TTDesc), P_double,
                               c_void_p]),
    "tt_sdp_create_maxcut": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(Options), c_void_p,
                                       ctypes.POINTER(c_void_p)]),
    "tt_sdp_create_theta": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(Options), c_void_p,
                                      ctypes.POINTER(c_void_p)]),
    "tt_sdp_create_cc": (c_int32, [ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc), ctypes.POINTER(TTDesc),
                                   ctypes.POINTER(Options), c_void_p, ctypes.POINTER(c_void_p)]),
    "tt_sdp_newton_step": (c_int32, [c_void_p, ctypes.POINTER(IterInfo)]),
    "tt_sdp_solve": (c_int32, [c_void_p, ctypes.POINTER(Result)]),
    "tt_sdp_redo_update": (c_int32, [c_void_p, c_double, c_double]),
    "tt_sdp_solve_batch": (c_int32, [c_int32, ctypes.POINTER(c_void_p), c_int32, ctypes.POINTER(Result)]),
    "tt_sdp_get_iterate": (c_int32, [c_void_p, c_int32, P_int32, c_void_p, ctypes.POINTER(c_size_t)]),
    "tt_sdp_order": (c_int32, [c_void_p]),
    "tt_sdp_destroy": (None, [c_void_p]),
    "tt_sdp_status_string": (ctypes.c_char_p, [c_int32]),
    "tt_last_error": (ctypes.c_char_p, []),
    "tt_launch_count": (ctypes.c_uint64, []),
    "tt_contraction_stats": (None, [P_double, P_double]),
    "tt_contraction_stats_reset": (None, []),
    "tt_profile_report": (c_size_t, [ctypes.c_char_p, c_size_t]),
    "tt_rankpred_param_count": (c_int32, []),
    "tt_rankpred_create": (c_int32, [ctypes.c_uint64, ctypes.POINTER(c_void_p)]),
    "tt_rankpred_destroy": (None, [c_void_p]),
    "tt_rankpred_get_params": (c_int32, [c_void_p, c_void_p]),
    "tt_rankpred_set_params": (c_int32, [c_void_p, c_void_p]),
    "tt_rankpred_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "tt_rankpred_train": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, ctypes.c_float,
                                    ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]),
    "tt_rankpred_predict": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "tt_sdp_set_rank_predictor": (c_int32, [c_void_p, c_void_p]),
    "tt_sdp_set_trace": (c_int32, [c_void_p, c_int32]),
    "tt_sdp_get_trace": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_size_t)]),
    "tt_tc_stats": (None, [P_double, P_double, ctypes.POINTER(ctypes.c_uint64)]),
    "tt_lu_stats": (None, [P_double, P_double, ctypes.POINTER(ctypes.c_uint64)]),
    "tt_gemm64_stats": (None, [P_double, P_double, ctypes.POINTER(ctypes.c_uint64)]),
}

_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the compiled library; raises if it is missing (there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
