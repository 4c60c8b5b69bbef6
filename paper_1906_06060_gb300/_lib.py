"""ctypes declarations of the C ABI in include/hotrg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhotrg.so")

HOTRG_OK, HOTRG_EINVAL, HOTRG_ENOMEM, HOTRG_ENUMERIC = 0, -1, -2, -3
HOTRG_ENOCONV, HOTRG_ETIMEOUT, HOTRG_EDEVICE, HOTRG_ESTATE, HOTRG_ENOTSUP = -4, -5, -6, -7, -8
HOTRG_FP64, HOTRG_BF16X3, HOTRG_BF16X6, HOTRG_BF16X4, HOTRG_FP16X3, HOTRG_FP16X4 = 0, 1, 2, 3, 4, 5


class Opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("fp64_steps", c_int), ("x6_steps", c_int), ("batch", c_int),
                ("beta", POINTER(c_double)), ("h", POINTER(c_double)), ("stream", c_void_p),
                ("workspace", c_void_p), ("workspace_bytes", c_size_t), ("max_steps", c_int),
                ("kblock", c_int), ("fold_group", c_int), ("derivatives", c_int), ("impurities", c_int),
                ("z2", c_int), ("graphs", c_int),
                ("wait_timeout_s", c_double), ("max_sweeps", c_int), ("group", c_int),
                ("cta_group", c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("steps", c_int), ("last_axis", c_int), ("lnz_per_site", c_double),
                ("last_ln_c", c_double), ("x_indicator", c_double), ("dlnz_dbeta", c_double),
                ("dlnz_dh", c_double), ("internal_energy", c_double), ("magnetization", c_double),
                ("nn_correlation", c_double), ("spin", c_double)]


class Timing(ctypes.Structure):
    _fields_ = [("ms_step", c_double), ("ms_isometry", c_double), ("ms_operands", c_double),
                ("ms_gemm", c_double), ("ms_epilogue", c_double), ("ms_norm", c_double),
                ("steps", c_longlong), ("gemm_launches", c_longlong), ("kernel_launches", c_longlong),
                ("gemm_flops", c_double), ("gemm_tensor_flops", c_double), ("step_flops", c_double),
                ("dense_step_flops", c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("kblock", c_int), ("group_m", c_int), ("fold_group", c_int), ("ms", c_double),
                ("cta_group", c_int)]


_SIGS = {
    "hotrg_opts_default": (None, [POINTER(Opts)]),
    "hotrg_workspace_size": (c_int, [c_int, c_int, POINTER(Opts), POINTER(c_size_t)]),
    "hotrg_init": (c_int, [POINTER(c_void_p), c_int, c_double, c_double, c_int, POINTER(Opts)]),
    "hotrg_step": (c_int, [c_void_p, c_int]),
    "hotrg_free_energy": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    "hotrg_observables": (c_int, [c_void_p, c_int, POINTER(Obs)]),
    "hotrg_spectra": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_double), c_int, POINTER(c_int)]),
    "hotrg_ln_norms": (c_int, [c_void_p, c_int, POINTER(c_double), c_int, POINTER(c_int)]),
    "hotrg_get_tensor": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_double), c_size_t]),
    "hotrg_set_tensor": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_double)]),
    "hotrg_set_tensor_z2": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_double)]),
    "hotrg_state_size": (c_int, [c_void_p, POINTER(c_size_t)]),
    "hotrg_state_save": (c_int, [c_void_p, c_void_p, c_size_t]),
    "hotrg_state_load": (c_int, [c_void_p, c_void_p, c_size_t]),
    "hotrg_autotune": (c_int, [c_void_p, POINTER(Tuning)]),
    "hotrg_timing_start": (c_int, [c_void_p]),
    "hotrg_timing_stop": (c_int, [c_void_p, POINTER(Timing)]),
    "hotrg_destroy": (None, [c_void_p]),
    "hotrg_strerror": (c_char_p, [c_int]),
    "hotrg_gemm_scratch_bytes": (c_size_t, [c_longlong, c_longlong, c_longlong]),
    "hotrg_gemm_split": (c_int, [c_void_p, c_longlong, c_void_p, c_longlong, c_void_p, c_longlong,
                                 c_longlong, c_longlong, c_longlong, c_int, c_int, c_int, c_void_p, c_size_t,
                                 c_void_p]),
    "hotrg_gemm_split_f16": (c_int, [c_void_p, c_longlong, c_void_p, c_longlong, c_void_p, c_longlong,
                                     c_longlong, c_longlong, c_longlong, c_int, c_int, c_int, c_void_p, c_size_t,
                                     c_void_p]),
    "hotrg_gemm_status": (c_int, [c_void_p, c_void_p]),
    "hotrg_gemm_wait_probe_bytes": (c_size_t, []),
    "hotrg_gemm_wait_probe": (c_int, [c_double, c_void_p, c_size_t, c_void_p]),
    "hotrg_gemm_split_noalloc": (c_int, [c_void_p, c_longlong, c_void_p, c_longlong, c_void_p, c_longlong,
                                         c_longlong, c_longlong, c_longlong, c_int, c_void_p]),
    "hotrg_bench_fp64_fma": (c_int, [c_longlong, c_void_p, POINTER(c_double), c_void_p]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libhotrg.so from the package directory. Raises if it has not been built: there is
    no fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhotrg.so not built ({LIB_PATH}); run "
                              "`python -m paper_1906_06060_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HotrgError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().hotrg_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != HOTRG_OK:
        raise HotrgError(code, where)
