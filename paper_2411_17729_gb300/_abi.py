"""ctypes binding of the cascade C ABI (include/cascade.h), same names.

Argument marshalling only: every computation happens in libcascade.so.  If
the library has not been built, importing this module raises ImportError;
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcascade.so")

CASCADE_OK = 0
CASCADE_ERR_INVALID_ARG = 1
CASCADE_ERR_UNSUPPORTED = 2
CASCADE_ERR_OOM = 3
CASCADE_ERR_CUDA = 4
CASCADE_ERR_TIMEOUT = 5
CASCADE_ERR_STATE = 6

CASCADE_FP64 = 0
CASCADE_FP32 = 1
CASCADE_BF16_SPLIT = 2

CASCADE_FLAG_SAVE_STATES = 1
CASCADE_FLAG_RECOMPUTE = 2
CASCADE_FLAG_NO_FUSED_OUTPUT = 4
CASCADE_FLAG_GRAPH = 8
CASCADE_FLAG_SCAN = 16
CASCADE_FLAG_ZOH = 32
CASCADE_FLAG_NO_FUSED_FIRST = 64
CASCADE_FLAG_DENSE_SETUP = 128
CASCADE_FLAG_FUSE_WIDE_OUTPUT = 256
CASCADE_FLAG_NO_FUSED_STAGES = 512

PRECISIONS = {"fp64": CASCADE_FP64, "fp32": CASCADE_FP32, "bf16_split": CASCADE_BF16_SPLIT}


class cascade_desc_t(C.Structure):
    _fields_ = [("m", C.c_int32), ("p", C.c_int32), ("q", C.c_int32), ("nsys", C.c_int32),
                ("N", C.c_int32), ("precision", C.c_int32), ("max_len", C.c_int32),
                ("flags", C.c_int32), ("max_rows", C.c_int64), ("eps", C.c_double)]


cascade_plan_t = C.c_void_p
_P = C.c_void_p
_D = C.POINTER(C.c_double)

# (name, restype, argtypes) for every function of include/cascade.h
SIGNATURES = [
    ("cascade_status_string", C.c_char_p, [C.c_int]),
    ("cascade_last_error", C.c_char_p, [cascade_plan_t]),
    ("cascade_plan_create", C.c_int, [C.POINTER(cascade_plan_t), C.POINTER(cascade_desc_t)]),
    ("cascade_plan_destroy", None, [cascade_plan_t]),
    ("cascade_set_system_continuous", C.c_int, [cascade_plan_t, _P, _P, _P, _P, _P, _P, _P]),
    ("cascade_set_system_discrete", C.c_int, [cascade_plan_t, _P, _P, _P, _P, _P]),
    ("cascade_get_N", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_get_powers", C.c_int, [cascade_plan_t, C.c_int32, C.c_int32, _P, _P]),
    ("cascade_set_batch", C.c_int, [cascade_plan_t, C.POINTER(C.c_int64), C.c_int32,
                                    C.POINTER(C.c_int32)]),
    ("cascade_get_seq_N", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_get_matvec_count", C.c_int, [cascade_plan_t, C.POINTER(C.c_int64)]),
    ("cascade_get_output_fused", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_get_first_fused", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_get_fused_stages", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_get_stage_shapes", C.c_int,
     [cascade_plan_t, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("cascade_set_stage_shapes", C.c_int, [cascade_plan_t, C.c_int32, C.POINTER(C.c_int32)]),
    ("cascade_workspace_size", C.c_int, [cascade_plan_t, C.POINTER(C.c_size_t)]),
    ("cascade_forward", C.c_int, [cascade_plan_t, _P, _P, _P, C.c_size_t, _P]),
    ("cascade_forward_host", C.c_int, [cascade_plan_t, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    ("cascade_forward_fixed_scratch", C.c_int, [cascade_plan_t, _P, _P, _P]),
    ("cascade_backward", C.c_int, [cascade_plan_t, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                   C.c_size_t, _P]),
    ("cascade_recursion_forward", C.c_int, [cascade_plan_t, _P, _P, _P]),
    ("cascade_get_device_error", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_selftest_timeout", C.c_int, [C.c_int32]),
    ("cascade_launch_count", C.c_int64, []),
    ("cascade_autotune", C.c_int, [cascade_plan_t, _P, _P, _P, C.c_size_t, _P, C.c_int32,
                                   C.POINTER(C.c_int32)]),
    ("cascade_set_kernel_shape", C.c_int, [cascade_plan_t, C.POINTER(C.c_int32)]),
    ("cascade_enable_stage_timing", C.c_int, [cascade_plan_t, C.c_int32]),
    ("cascade_get_stage_times", C.c_int, [cascade_plan_t, C.c_int32, C.POINTER(C.c_int32),
                                          C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2411_17729_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class CascadeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status: int, plan=None) -> None:
    if status != CASCADE_OK:
        l = lib()
        msg = (l.cascade_last_error(plan) or b"").decode() or \
            (l.cascade_status_string(status) or b"").decode()
        raise CascadeError(status, msg)


def __getattr__(name):
    # module-level access to the C functions under their C names
    if name.startswith("cascade_"):
        return getattr(lib(), name)
    raise AttributeError(name)
