"""ctypes declarations of the C ABI in include/qfactor.h.

The shared library libqfactor.so is built in-tree (``_build.build()``).  If
it is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

from . import _build

QF_OK = 0
QF_EINVAL = -1
QF_ENOMEM = -2
QF_ECUDA = -3
QF_ENONFINITE = -4
QF_ETIMEOUT = -5

QF_C128 = 0
QF_C64 = 1
QF_C64_REFINE64 = 2
QF_DF64 = 3
QF_C64_REFINE_DF = 4

QF_NOALLOC_SCRATCH_BYTES = 64 * 1024
QF_BATCH_MAX_QUBITS = 6

QF_STOP_CONVERGED = 1
QF_STOP_PLATEAU = 2
QF_STOP_MAX_SWEEPS = 3

REASONS = {QF_STOP_CONVERGED: "converged", QF_STOP_PLATEAU: "plateau",
           QF_STOP_MAX_SWEEPS: "max_sweeps"}


class qf_options(ct.Structure):
    _fields_ = [
        ("dist_tol", ct.c_double),
        ("max_sweeps", ct.c_int32),
        ("min_sweeps", ct.c_int32),
        ("reset_iter", ct.c_int32),
        ("long_diff_count", ct.c_int32),
        ("diff_tol_a", ct.c_double),
        ("diff_tol_r", ct.c_double),
        ("long_diff_r", ct.c_double),
        ("beta", ct.c_double),
        ("precision", ct.c_int32),
        ("max_c64_sweeps", ct.c_int32),
        ("switch_tol", ct.c_double),
        ("cost_history", ct.c_void_p),
    ]


class qf_result(ct.Structure):
    _fields_ = [
        ("best_start", ct.c_int32),
        ("sweeps", ct.c_int32),
        ("c64_sweeps", ct.c_int32),
        ("reason", ct.c_int32),
        ("best_cost", ct.c_double),
    ]


class qf_gate_loc(ct.Structure):
    _fields_ = [("k", ct.c_int32), ("q", ct.c_int32 * 4)]


class qf_gate_spec(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("q", ct.c_int32 * 3)]


QF_GATE_U4 = 0
QF_GATE_U8 = 1
QF_GATE_RZ = 2
QF_GATE_GPI = 3
QF_GATE_MS = 4


class qf_batch_stats(ct.Structure):
    _fields_ = [
        ("warps_per_cta", ct.c_int32),
        ("ctas", ct.c_int32),
        ("kernel_ms", ct.c_double),
        ("total_sweeps", ct.c_int64),
        ("total_c64_sweeps", ct.c_int64),
    ]


P = ct.c_void_p
I = ct.c_int
D = ct.c_double
DP = ct.POINTER(ct.c_double)
I64P = ct.POINTER(ct.c_int64)
IP = ct.POINTER(ct.c_int)

# name -> (restype, argtypes)
SIGNATURES = {
    "qf_last_error": (ct.c_char_p, []),
    "qf_version": (I, []),
    "qf_options_default": (I, [ct.POINTER(qf_options)]),
    "qf_instantiate": (I, [P, I, I, P, P, D, I, P, DP, ct.POINTER(I), P]),
    "qf_instantiate_ex": (I, [P, I, I, P, I, P, ct.POINTER(qf_options), P, DP,
                              ct.POINTER(qf_result), P]),
    "qf_cost_and_env": (I, [P, I, I, P, I, P, DP, P, P, P]),
    "qf_cost_grad": (I, [P, I, I, P, I, P, DP, P, P]),
    "qf_cost_and_env_k": (I, [P, I, I, P, I, P, DP, P, P, P]),
    "qf_cost_grad_k": (I, [P, I, I, P, I, P, DP, P, P]),
    "qf_instantiate_batched": (I, [I, P, P, P, P, I, P, ct.POINTER(qf_options), P, DP, P, P,
                                   ct.POINTER(qf_batch_stats), P]),
    "qf_instantiate_batched_k": (I, [I, P, P, P, P, I, P, ct.POINTER(qf_options), P, DP, P, P,
                                     ct.POINTER(qf_batch_stats), P]),
    "qf_plan_create": (I, [I, I, P, I, I, ct.POINTER(P)]),
    "qf_plan_destroy": (I, [P]),
    "qf_plan_load": (I, [P, P, P, P]),
    "qf_plan_sweep": (I, [P, I, I, D]),
    "qf_plan_rebuild": (I, [P, I]),
    "qf_plan_costs": (I, [P, DP, P]),
    "qf_plan_get_gates": (I, [P, P]),
    "qf_plan_enable_pass_timing": (I, [P, I]),
    "qf_plan_pass_stats": (I, [P, DP, I64P, I64P, DP]),
    "qf_plan_set_lookahead": (I, [P, I]),
    "qf_plan_lookahead_windows": (I, [P, IP]),
    "qf_plan_status": (I, [P]),
    "qf_init_tensor": (I, [P, I, I, P, I, P, P, I, P]),
    "qf_apply_pair": (I, [P, I, I, I, I, P, P, I, P]),
    "qf_partial_trace": (I, [P, I, I, I, I, P, I, P]),
    "qf_apply_two_pairs": (I, [P, I, I, I, I, P, P, I, I, P, P, I, P]),
    "qf_convert_tensor": (I, [P, I, P, I, ct.c_int64, P]),
    "qf_partial_trace_after": (I, [P, I, I, I, I, P, P, I, I, P, I, P]),
    "qf_partial_trace_noalloc": (I, [P, I, I, I, I, P, I, P]),
    "qf_optimize_gates": (I, [P, P, D, I, P, P, P]),
    "qf_trace": (I, [P, I, I, P, I, P]),
    "qf_reunitarize_gates": (I, [P, I, P]),
    "qf_circuit_unitary": (I, [I, I, P, P, P, P]),
    "qf_instantiate_k": (I, [P, I, I, P, I, P, ct.POINTER(qf_options), P, DP,
                             ct.POINTER(qf_result), P]),
    "qf_plan_create_k": (I, [I, I, P, I, I, ct.POINTER(P)]),
    "qf_plan_gate_entries": (I, [P, I64P]),
    "qf_plan_create_spec": (I, [I, I, P, I, I, ct.POINTER(P)]),
    "qf_instantiate_spec": (I, [P, I, I, P, I, P, P, ct.POINTER(qf_options), P, P, DP,
                                ct.POINTER(qf_result), P]),
    "qf_plan_load_spec": (I, [P, P, P, P, P]),
    "qf_plan_get_params": (I, [P, P]),
    "qf_apply_gate_k": (I, [P, I, I, P, P, P, I, P]),
    "qf_partial_trace_k": (I, [P, I, I, P, P, I, P]),
    "qf_optimize_gates_k": (I, [P, I, P, D, I, P, P, P]),
    "qf_init_tensor_k": (I, [P, I, I, P, I, P, P, I, P]),
    "qf_circuit_unitary_k": (I, [I, I, P, P, P, P]),
    "qf_set_tc_wait_limit": (I, [I]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libqfactor.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(
                f"QFactor CUDA library not found at {path}; build it with "
                "paper_2306_08152_gb300._build.build() (there is no CPU fallback)")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class QFactorError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"QFactor error {code}: {msg}")
        self.code = code


def check(rc: int):
    if rc != QF_OK:
        msg = load().qf_last_error()
        raise QFactorError(rc, msg.decode() if msg else "")
    return rc
