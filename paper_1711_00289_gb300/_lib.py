"""ctypes binding of include/conv.h (argument marshalling only).

The structures mirror the C declarations field for field; every function of the
header is bound here with the same name.  Loading fails loudly if the shared
library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

CONV_OK, CONV_ERR_ARG, CONV_ERR_CUDA, CONV_ERR_WORKSPACE, CONV_ERR_UNSUPPORTED, \
    CONV_ERR_TIMEOUT = range(6)
CONV_FP64, CONV_MIXED = 0, 1
CONV_PATH_AUTO, CONV_PATH_PLAIN, CONV_PATH_COMPACT = 0, 1, 2
CONV_MAP_DEFAULT, CONV_MAP_THREAD, CONV_MAP_WARP = 0, 1, 2
FLAG_TRIGGERED, FLAG_ACTIVE, FLAG_LIMITED, FLAG_NEWTON, FLAG_BADINPUT = 1, 2, 4, 8, 16
EXIT_SHIFT = 8
MAX_LEVELS = 32
NOALLOC_MAX_COLS = 65536


class ConvError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("pver", C.c_int32), ("n_cols", C.c_int32), ("ld", C.c_int32),
                ("reserved", C.c_int32), ("hyai", C.POINTER(C.c_double)),
                ("hybi", C.POINTER(C.c_double)), ("p0", C.c_double)]


class DeepParams(C.Structure):
    _fields_ = [("capelmt", C.c_double), ("lambda_default", C.c_double),
                ("tau_default", C.c_double), ("c0", C.c_double), ("alpha_dd", C.c_double),
                ("p_launch_min", C.c_double), ("p_top_lim", C.c_double), ("q_min", C.c_double),
                ("ent_zscale", C.c_double), ("n_newton_lcl", C.c_int32),
                ("n_newton_h", C.c_int32), ("n_plumes", C.c_int32), ("reserved", C.c_int32),
                ("plume_spread", C.c_double)]


class ShallowParams(C.Structure):
    _fields_ = [("eps_s", C.c_double), ("tke", C.c_double), ("c_m", C.c_double),
                ("cin_scale", C.c_double), ("cin_max", C.c_double), ("a_w", C.c_double),
                ("b_w", C.c_double), ("ql_crit", C.c_double), ("p_lcl_min", C.c_double),
                ("p_lfc_min", C.c_double), ("p_top_lim", C.c_double),
                ("n_newton_lcl", C.c_int32), ("n_newton_h", C.c_int32), ("evap_k", C.c_double)]


class In(C.Structure):
    _fields_ = [("T", C.c_void_p), ("q", C.c_void_p), ("ps", C.c_void_p),
                ("lam", C.c_void_p), ("tau", C.c_void_p)]


class Out(C.Structure):
    _fields_ = [("dTdt", C.c_void_p), ("dqdt", C.c_void_p), ("prec", C.c_void_p),
                ("flags", C.c_void_p), ("kb", C.c_void_p), ("klcl", C.c_void_p),
                ("ktop", C.c_void_p), ("kaux", C.c_void_p), ("cape", C.c_void_p),
                ("mb", C.c_void_p), ("cons_err", C.c_void_p), ("mu", C.c_void_p),
                ("du", C.c_void_p), ("md", C.c_void_p)]


class Launch(C.Structure):
    _fields_ = [("path", C.c_int32), ("block_threads", C.c_int32), ("mapping", C.c_int32),
                ("reserved1", C.c_int32), ("stage_events", C.POINTER(C.c_void_p))]


class Member(C.Structure):
    _fields_ = [("grid", Grid), ("in_", In), ("deep_out", Out), ("shallow_out", Out),
                ("deep", DeepParams), ("shallow", ShallowParams), ("dt", C.c_double)]


_lib = None


def lib(build: bool = True):
    """Load libconvgb.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libconvgb.so not built ({path}); run paper_1711_00289_gb300.build")
    L = C.CDLL(path)
    P = C.POINTER
    vp, st, d = C.c_void_p, C.c_int, C.c_double
    L.conv_deep_defaults.argtypes = [P(DeepParams)]
    L.conv_deep_defaults.restype = None
    L.conv_shallow_defaults.argtypes = [P(ShallowParams)]
    L.conv_shallow_defaults.restype = None
    L.conv_status_str.argtypes = [st]
    L.conv_status_str.restype = C.c_char_p
    L.conv_workspace_bytes.argtypes = [P(Grid), st, P(Launch)]
    L.conv_workspace_bytes.restype = C.c_size_t
    L.conv_deep_run.argtypes = [P(Grid), P(In), P(DeepParams), d, st, P(Out), P(Launch), vp,
                                C.c_size_t, vp]
    L.conv_deep_run.restype = st
    L.conv_shallow_run.argtypes = [P(Grid), P(In), P(ShallowParams), st, P(Out), P(Launch), vp,
                                   C.c_size_t, vp]
    L.conv_shallow_run.restype = st
    L.conv_deep_shallow_run.argtypes = [P(Grid), P(In), P(DeepParams), P(ShallowParams), d, st,
                                        P(Out), P(Out), P(Launch), vp, C.c_size_t, vp]
    L.conv_deep_shallow_run.restype = st
    L.conv_bench_op_rate.argtypes = [st, st, st, P(C.c_double)]
    L.conv_bench_op_rate.restype = st
    L.conv_bench_f32_quotient.argtypes = [vp, vp, vp, C.c_int64, vp]
    L.conv_bench_f32_quotient.restype = st
    L.conv_bench_lcl.argtypes = [vp, vp, vp, vp, vp, C.c_int64, st, vp]
    L.conv_bench_lcl.restype = st
    L.conv_deep_shallow_run_noalloc.argtypes = [P(Grid), P(In), P(DeepParams),
                                                P(ShallowParams), d, st, P(Out), P(Out), vp]
    L.conv_deep_shallow_run_noalloc.restype = st
    L.conv_batch_plan.argtypes = [P(Member), st, st, P(vp)]
    L.conv_batch_plan.restype = st
    L.conv_batch_workspace_bytes.argtypes = [vp]
    L.conv_batch_workspace_bytes.restype = C.c_size_t
    L.conv_batch_run.argtypes = [vp, vp, C.c_size_t, vp, P(vp)]
    L.conv_batch_run.restype = st
    L.conv_batch_autotune.argtypes = [vp, vp, C.c_size_t, vp, st]
    L.conv_batch_autotune.restype = st
    L.conv_batch_config.argtypes = [vp, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_int32)]
    L.conv_batch_config.restype = st
    L.conv_batch_free.argtypes = [vp]
    L.conv_batch_free.restype = None
    L.conv_deep_adjoint.argtypes = [P(Grid), P(In), P(DeepParams), d, st, vp, vp,
                                    P(C.c_double), vp, vp, vp, vp, vp, vp, vp]
    L.conv_deep_adjoint.restype = st
    L.conv_deep_shallow_adjoint.argtypes = [P(Grid), P(In), P(DeepParams), P(ShallowParams), d,
                                            st, vp, vp, vp, vp, P(C.c_double), vp, vp, vp, vp,
                                            vp, st, vp]
    L.conv_deep_shallow_adjoint.restype = st
    L.conv_advance.argtypes = [P(Grid), vp, vp, vp, vp, d, P(Out), P(Out), d, st, vp]
    L.conv_advance.restype = st
    L.conv_tracer_transport.argtypes = [P(Grid), vp, P(Out), P(Out), d, st, vp, vp, vp, st, vp]
    L.conv_tracer_transport.restype = st
    L.conv_momentum_transport.argtypes = [P(Grid), vp, P(Out), P(Out), d, d, d, vp, vp, vp, st,
                                          vp]
    L.conv_momentum_transport.restype = st
    L.conv_pipeline_plan.argtypes = [P(Grid), st, st, P(vp)]
    L.conv_pipeline_plan.restype = st
    L.conv_pipeline_run.argtypes = [vp, P(In), P(DeepParams), P(ShallowParams), d, P(Out),
                                    P(Out), vp]
    L.conv_pipeline_run.restype = st
    L.conv_pipeline_free.argtypes = [vp]
    L.conv_batch_set_config.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
    L.conv_batch_set_config.restype = st
    L.conv_batch_tune_record.argtypes = [vp, vp]
    L.conv_batch_tune_record.restype = st
    L.conv_count_triggered.argtypes = [vp, C.c_int32, C.c_int32, vp, vp]
    L.conv_count_triggered.restype = st
    L.conv_partition_columns.argtypes = [C.c_int32, C.c_int32, vp, d, d, C.c_int32, vp]
    L.conv_partition_columns.restype = st
    L.conv_pipeline_free.restype = None
    _lib = L
    return L


CONV_OP_FMA, CONV_OP_EXP, CONV_OP_LOG, CONV_OP_DIV, CONV_OP_POW, CONV_OP_SQRT = range(6)
CONV_ARITH_FP64, CONV_ARITH_FP32, CONV_ARITH_FP32_FAST = range(3)


def op_rate(op: int, arith: int, iters: int = 2000) -> float:
    """Measured evaluations per second of one operation on the current device."""
    r = C.c_double()
    check(lib().conv_bench_op_rate(op, arith, iters, C.byref(r)), "conv_bench_op_rate")
    return r.value


def f32_quotient(a: int, b: int, q: int, n: int, stream: int = 0) -> None:
    """q[i] = a[i] / b[i] with the mixed path's FP32 division (device pointers)."""
    check(lib().conv_bench_f32_quotient(a, b, q, n, stream), "conv_bench_f32_quotient")


def lcl_pressures(T: int, q: int, p: int, pL32: int, pL64: int, n: int, n_newton: int = 6,
                  stream: int = 0) -> None:
    """FP32 and FP64 LCL pressures of n parcels (device pointers)."""
    check(lib().conv_bench_lcl(T, q, p, pL32, pL64, n, n_newton, stream), "conv_bench_lcl")


def status_str(s: int) -> str:
    return lib().conv_status_str(int(s)).decode()


def check(status: int, what: str):
    if status != CONV_OK:
        raise ConvError(status, what)


def deep_defaults(**kw) -> DeepParams:
    p = DeepParams()
    lib().conv_deep_defaults(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown deep parameter {k}")
        setattr(p, k, v)
    return p


def shallow_defaults(**kw) -> ShallowParams:
    p = ShallowParams()
    lib().conv_shallow_defaults(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown shallow parameter {k}")
        setattr(p, k, v)
    return p
