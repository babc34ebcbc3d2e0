"""ctypes declarations of the C ABI in include/pn_batch.h (argument marshalling only).

Every struct here mirrors the header field for field.  Loading fails loudly if
the CUDA library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
RELEASE_LIB_PATH = os.path.join(HERE, "libpn_b300.so")
# The debug build (device bounds checks that report PN_E_CHECK; every call waits for its work).
DEBUG_LIB_PATH = os.path.join(HERE, "libpn_b300_debug.so")
# PN_B300_DEBUG=1 in the environment selects the debug build for the whole process.
LIB_PATH = DEBUG_LIB_PATH if os.environ.get("PN_B300_DEBUG") == "1" else RELEASE_LIB_PATH

PN_OK, PN_E_ARG, PN_E_CUDA, PN_E_NOMEM, PN_E_UNIMPLEMENTED, PN_E_CHECK = 0, -1, -2, -3, -4, -5
PN_ST_OK, PN_ST_MAX_STEPS, PN_ST_H_UNDERFLOW, PN_ST_NONFINITE, PN_ST_BAD_INPUT, PN_ST_LAND_MAXIT, PN_ST_RUNNING = range(7)
PN_FP64, PN_MIXED, PN_MIXED_DS = 0, 1, 2
PN_STOP_LAND, PN_STOP_FIRST_CROSS = 0, 1
PN_THETA_BCV2, PN_THETA_AS_PRINTED = 0, 1
PN_SCHED_AUTO, PN_SCHED_PLAIN, PN_SCHED_PERSISTENT = 0, 1, 2
PN_ORDER_INPUT, PN_ORDER_LENGTH = 0, 1
ABI_VERSION = 3  # PN_ABI_VERSION of the header these declarations follow
(PN_TERM_1PN, PN_TERM_SO, PN_TERM_TAIL, PN_TERM_2PN, PN_TERM_SS, PN_TERM_25PN, PN_TERM_3PN, PN_TERM_35PN,
 PN_TERM_PREC) = (1 << i for i in range(9))
PN_TERM_ALL = 0x1FF

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)


class pn_params(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double), ("safety", C.c_double),
                ("fac_min", C.c_double), ("fac_max", C.c_double), ("h_min", C.c_double),
                ("land_tol", C.c_double), ("max_steps", C.c_int64), ("land_max_iter", C.c_int32),
                ("stop_mode", C.c_int32), ("term_mask", C.c_uint32), ("theta_mode", C.c_int32),
                ("fixed_step", C.c_int32), ("precision", C.c_int32), ("schedule", C.c_int32),
                ("block", C.c_int32), ("bpt", C.c_int32), ("ckpt_every", C.c_int32), ("order", C.c_int32)]


INPUT_FIELDS = ("m1", "m2", "chi1", "chi2", "s1x", "s1y", "s1z", "s2x", "s2y", "s2z", "lx", "ly", "lz",
                "omega0", "omega_f")
OUTPUT_DFIELDS = ("S1x", "S1y", "S1z", "S2x", "S2y", "S2z", "Lx", "Ly", "Lz", "omega", "t")
OUTPUT_IFIELDS = ("n_acc", "n_rej", "n_land", "status")
OUTPUT_DOTS = ("dot_s1s2", "dot_ls1", "dot_ls2")
COT_FIELDS = ("dot_s1s2", "dot_ls1", "dot_ls2", "Lx", "Ly", "Lz", "S1x", "S1y", "S1z", "S2x", "S2y", "S2z", "t")
GRAD_FIELDS = ("s1x", "s1y", "s1z", "s2x", "s2y", "s2z", "q")
GRAD_TAN_FIELDS = ("s1x_tan", "s1y_tan", "s1z_tan", "s2x_tan", "s2y_tan", "s2z_tan")  # optional
GRAD_ANGLE_FIELDS = ("s1_dtheta", "s1_dphi", "s2_dtheta", "s2_dphi")  # optional


class pn_inputs(C.Structure):
    _fields_ = [(f, _D) for f in INPUT_FIELDS]


class pn_outputs(C.Structure):
    _fields_ = [(f, _D) for f in OUTPUT_DFIELDS] + [(f, _I) for f in OUTPUT_IFIELDS] + [(f, _D) for f in OUTPUT_DOTS]


class pn_dist(C.Structure):
    _fields_ = [("q_mode", C.c_int32), ("chi_mode", C.c_int32), ("q_lo", C.c_double), ("q_hi", C.c_double),
                ("chi_lo", C.c_double), ("chi_hi", C.c_double), ("omega0_lo", C.c_double),
                ("omega0_hi", C.c_double), ("omega_f", C.c_double)]


class pn_cotangents(C.Structure):
    _fields_ = [(f, _D) for f in COT_FIELDS]


class pn_grads(C.Structure):
    _fields_ = [(f, _D) for f in GRAD_FIELDS + GRAD_TAN_FIELDS + GRAD_ANGLE_FIELDS]


class pn_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("count_by_status", C.c_int64 * 8), ("acc_total", C.c_int64),
                ("rej_total", C.c_int64), ("land_total", C.c_int64), ("acc_min", C.c_int32),
                ("acc_max", C.c_int32), ("attempts_min", C.c_int32), ("attempts_max", C.c_int32),
                ("pearson_s1s2", C.c_double), ("pearson_ls1", C.c_double), ("pearson_ls2", C.c_double),
                ("pearson_count", C.c_int64), ("mean_final_s1s2", C.c_double), ("std_final_s1s2", C.c_double),
                ("ms_last_integrate", C.c_double), ("ms_last_adjoint", C.c_double)]


class pn_hist_spec(C.Structure):
    _fields_ = [("quantity_x", C.c_int32), ("quantity_y", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("x_lo", C.c_double), ("x_hi", C.c_double), ("y_lo", C.c_double), ("y_hi", C.c_double)]


class pn_ks_result(C.Structure):
    _fields_ = [("n", C.c_int64), ("d_lo", C.c_double), ("d_hi", C.c_double), ("p_at_d_lo", C.c_double),
                ("p_at_d_hi", C.c_double)]


PN_Q_FINAL_S1S2, PN_Q_FINAL_LS1, PN_Q_FINAL_LS2, PN_Q_INIT_S1S2, PN_Q_INIT_LS1, PN_Q_INIT_LS2 = range(6)


class pn_tune_result(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("block", C.c_int32), ("bpt", C.c_int32), ("n_candidates", C.c_int32),
                ("best_ms", C.c_double), ("n_tuned", C.c_int64)]


# Every exported symbol and its signature (restype, argtypes).
SIGNATURES = {
    "pn_abi_version": (C.c_int, []),
    "pn_params_default": (None, [C.POINTER(pn_params)]),
    "pn_batch_init": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.POINTER(pn_params), C.c_void_p]),
    "pn_batch_set_params": (C.c_int, [C.c_void_p, C.POINTER(pn_params)]),
    "pn_batch_sample": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(pn_dist), C.c_int64, C.POINTER(pn_inputs)]),
    "pn_batch_integrate": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs)]),
    "pn_batch_integrate_host": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs)]),
    "pn_batch_integrate_host_async": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs)]),
    "pn_batch_host_wait": (C.c_int, [C.c_void_p]),
    "pn_batch_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pn_batch_integrate_budget": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs),
                                            C.c_int32]),
    "pn_batch_resume": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs), C.c_int32]),
    "pn_batch_eval_rhs": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pn_batch_autotune": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs),
                                    C.POINTER(pn_tune_result)]),
    "pn_batch_adjoint": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_cotangents),
                                   C.POINTER(pn_grads), C.POINTER(pn_outputs)]),
    "pn_batch_masses": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "pn_batch_stats": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs),
                                 C.POINTER(pn_stats)]),
    "pn_batch_stats_segments": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(pn_inputs),
                                          C.POINTER(pn_outputs), C.POINTER(pn_stats)]),
    "pn_batch_histogram": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs),
                                     C.POINTER(pn_hist_spec), C.POINTER(C.c_int64)]),
    "pn_batch_kde": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(pn_inputs), C.POINTER(pn_outputs), C.c_int32,
                               C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pn_ks_uniform": (C.c_int, [C.POINTER(C.c_int64), C.c_int32, C.c_double, C.c_double,
                                C.POINTER(pn_ks_result)]),
    "pn_batch_destroy": (None, [C.c_void_p]),
    "pn_integrate_noalloc": (C.c_int, [C.c_int64, C.POINTER(pn_params), C.POINTER(pn_inputs), C.POINTER(pn_outputs),
                                       C.c_void_p]),
    "pn_debug_selftest": (C.c_int, []),
    "pn_last_error": (C.c_char_p, [C.c_void_p]),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libpn_b300.so (raises if it is missing; build it with paper_0908_3889_b300.build.build())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_0908_3889_b300.build.build())")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.pn_abi_version() != ABI_VERSION:
        raise RuntimeError("libpn_b300.so ABI version mismatch")
    if path is None:
        _lib = lib
    return lib
