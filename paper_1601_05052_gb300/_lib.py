"""ctypes declarations of libdd.so's C ABI (include/dd.h).

Loading fails loudly: there is no fallback. If the shared library is missing
it is built in-tree with nvcc first (see _build.py); if that is impossible an
ImportError names the reason.
"""
import ctypes
import os

from . import _build

DD_F32, DD_F16, DD_BF16, DD_U8 = 0, 1, 2, 3
DTYPES = {"f32": DD_F32, "f16": DD_F16, "bf16": DD_BF16, "u8": DD_U8}
STATUS = ["DD_OK", "DD_ERR_ARG", "DD_ERR_CUDA", "DD_ERR_NOMEM", "DD_ERR_UNSUPPORTED",
          "DD_ERR_TIMEOUT", "DD_ERR_NOT_TUNED", "DD_ERR_DEVICE"]


class Variant(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32),
                ("dm_per_thread", ctypes.c_int32), ("samples_per_thread", ctypes.c_int32),
                ("warps_dm", ctypes.c_int32), ("warps_time", ctypes.c_int32),
                ("chans_per_stage", ctypes.c_int32), ("stages", ctypes.c_int32)]

    def as_tuple(self):
        return tuple(getattr(self, f) for f, _ in self._fields_)

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneReport(ctypes.Structure):
    _fields_ = [("n_tried", ctypes.c_int32), ("best", Variant), ("best_ms", ctypes.c_double),
                ("best_gflops", ctypes.c_double), ("mean_gflops", ctypes.c_double),
                ("std_gflops", ctypes.c_double), ("snr", ctypes.c_double),
                ("chebyshev", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "best"}
        d["best"] = self.best.as_dict()
        return d


class DDError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__("%s: %s" % (name, msg))


P = ctypes.c_void_p
i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

# (name, restype, argtypes) for every function declared in include/dd.h
SIGNATURES = [
    ("dd_compute_shifts", i32, [i32, P, f64, f64, i32, P, P]),
    ("dd_plan_create", i32, [ctypes.POINTER(P), i32, P, f64, f64, i32, P, i64, i32, i32]),
    ("dd_plan_create_from_shifts", i32, [ctypes.POINTER(P), i32, i32, P, i64, i32, i32]),
    ("dd_plan_destroy", None, [P]),
    ("dd_plan_input_len", i64, [P]),
    ("dd_plan_input_stride", i64, [P]),
    ("dd_plan_max_shift", i32, [P]),
    ("dd_plan_shifts", i32, [P, P]),
    ("dd_plan_get_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_plan_set_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_plan_get_launch_order", i32, [P, ctypes.POINTER(i32)]),
    ("dd_plan_set_launch_order", i32, [P, i32]),
    ("dd_variant_count", i32, []),
    ("dd_variant_get", i32, [i32, ctypes.POINTER(Variant)]),
    ("dd_execute", i32, [P, P, P, P, P]),
    ("dd_execute_host", i32, [P, P, P, P, P]),
    ("dd_adjoint", i32, [P, P, P, P, P, P, P]),
    ("dd_grad_w_noalloc", i32, [P, P, P, P, P]),
    ("dd_tune", i32, [P, i32, ctypes.POINTER(TuneReport)]),
    ("dd_tune_adjoint", i32, [P, i32, ctypes.POINTER(TuneReport)]),
    ("dd_adjoint_get_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_adjoint_set_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_debug_wait_timeout", i32, [P, i32, P]),
    ("dd_batch_create", i32, [ctypes.POINTER(P), i32, PP]),
    ("dd_batch_execute", i32, [P, PP, PP, PP, P]),
    ("dd_batch_get_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_batch_set_variant", i32, [P, ctypes.POINTER(Variant)]),
    ("dd_batch_get_plan_variant", i32, [P, i32, ctypes.POINTER(Variant)]),
    ("dd_batch_set_plan_variant", i32, [P, i32, ctypes.POINTER(Variant)]),
    ("dd_batch_tune", i32, [P, i32, ctypes.POINTER(TuneReport)]),
    ("dd_batch_destroy", None, [P]),
    ("dd_stream_create", i32, [ctypes.POINTER(P), P]),
    ("dd_stream_push", i32, [P, P, P, P, P]),
    ("dd_stream_reset", i32, [P, P]),
    ("dd_stream_latency", i64, [P]),
    ("dd_stream_destroy", None, [P]),
    ("dd_plan_check_device", i32, [P]),
    ("dd_status_str", ctypes.c_char_p, [i32]),
    ("dd_get_last_error", i32, []),
    ("dd_last_error_message", ctypes.c_char_p, []),
    ("dd_version", i32, []),
]

_lib = None


def load():
    """Returns the loaded libdd.so, building it first if needed."""
    global _lib
    if _lib is not None:
        return _lib
    try:
        path = _build.build()
    except Exception as e:  # no nvcc, compile error, ...
        if os.path.exists(_build.LIB):
            path = _build.LIB
        else:
            raise ImportError("libdd.so is not built and cannot be built: %s" % e) from e
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != 0:
        msg = load().dd_last_error_message()
        raise DDError(status, msg.decode() if msg else "")
