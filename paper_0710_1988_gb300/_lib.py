"""ctypes declarations of libwd.so (the C ABI in include/wd.h).

The library must have been built (``python -m paper_0710_1988_gb300.build``);
importing this module without it raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwd.so")

WD_OK = 0
WD_BAD_ARG = 1
WD_NOT_CONVERGED = 2
WD_BREAKDOWN = 3
WD_SINGULAR_PROJECTION = 4
WD_TIMEOUT = 5
WD_CUDA_ERROR = 6
WD_OUT_OF_MEMORY = 7


class WdStats(ctypes.Structure):
    _fields_ = [
        ("mvp", ctypes.c_longlong),
        ("mvp_extra", ctypes.c_longlong),
        ("iters", ctypes.c_int),
        ("cycles", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("breakdown", ctypes.c_int),
        ("rel_res", ctypes.c_double),
        ("true_rel_res", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class WdProfile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_longlong * 6),
        ("ms", ctypes.c_double * 6),
        ("dslash_site_updates", ctypes.c_longlong),
        ("dslash_low_site_updates", ctypes.c_longlong),
    ]

    CATEGORIES = ("dslash", "stream", "tall_skinny", "dense", "dslash_low", "stream_low")

    def as_dict(self):
        return {c: {"launches": int(self.launches[i]), "ms": float(self.ms[i])}
                for i, c in enumerate(self.CATEGORIES)} | {
            "dslash_site_updates": int(self.dslash_site_updates),
            "dslash_low_site_updates": int(self.dslash_low_site_updates)}


P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double

# name -> (restype, argtypes); every symbol include/wd.h declares
SIGNATURES = {
    "wd_create": (I, [ctypes.POINTER(I), P, D, D, ctypes.POINTER(P)]),
    "wd_set_params": (I, [P, D, D]),
    "wd_set_operator": (I, [P, I]),
    "wd_eo_prepare": (I, [P, P, P, I, P]),
    "wd_eo_reconstruct": (I, [P, P, P, P, I, P]),
    "wd_apply": (I, [P, P, P, I, I, P]),
    "gmresdr_solve": (I, [P, P, P, I, I, D, I, P, P, P, ctypes.POINTER(WdStats), P]),
    "gmresdr_history": (I, [P, P, I]),
    "wd_probe_fp64_peak": (I, [I, I, P, P, P]),
    "wd_probe_bf16_mma_peak": (I, [I, I, P, P, P]),
    "wd_set_contraction": (I, [P, I]),
    "wd_set_eigen_estimates": (I, [P, I]),
    "wd_tsgemm": (I, [P, I, P, I, I, P, P, I, D, ctypes.c_longlong, I, P]),
    "wd_deflation_create": (I, [P, P, P, I, ctypes.POINTER(P), P]),
    "wd_deflation_destroy": (None, [P]),
    "dbicgstab_solve_deflated": (I, [P, P, P, P, I, D, I, ctypes.POINTER(WdStats), P]),
    "dbicgstab_solve": (I, [P, P, P, I, P, P, I, D, I, ctypes.POINTER(WdStats), P]),
    "dbicgstab_solve_adjoint": (I, [P, P, P, P, I, D, I, ctypes.POINTER(WdStats), P]),
    "dbicgstab_solve_adjoint_mixed": (I, [P, P, P, P, I, D, I, I, ctypes.POINTER(WdStats), P]),
    "wd_gradients": (I, [P, P, P, P, ctypes.POINTER(D), P]),
    "tm_multishift_solve": (I, [P, P, P, I, ctypes.POINTER(D), I, D, I, I, I, ctypes.POINTER(WdStats), P]),
    "dbicgstab_solve_mixed": (I, [P, P, P, P, I, D, I, I, ctypes.POINTER(WdStats), P]),
    "wd_apply_f32": (I, [P, P, P, I, I, P]),
    "wd_apply_f32_noalloc": (I, [P, P, P, I, I, P]),
    "wd_autotune_f32": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float), P]),
    "wd_set_f32_shape": (I, [P, I, I, I]),
    "wd_set_mixed_storage": (I, [P, I]),
    "wd_set_mixed_restart": (I, [P, D, I]),
    "wd_apply_f16": (I, [P, P, P, I, I, P]),
    "wd_autotune_f16": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float), P]),
    "wd_set_f16_shape": (I, [P, I, I, I]),
    "wd_profile_enable": (I, [P, ctypes.c_uint]),
    "wd_profile_read": (I, [P, ctypes.POINTER(WdProfile)]),
    "wd_destroy": (None, [P]),
    "wd_error_string": (ctypes.c_char_p, [I]),
    "wd_last_error_detail": (I, [ctypes.c_char_p, ctypes.c_size_t]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_0710_1988_gb300.build` "
            "(the solvers have no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class WdError(RuntimeError):
    def __init__(self, status: int, detail: str):
        self.status = status
        super().__init__(f"wd status {status}: {detail}")


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().wd_last_error_detail(buf, len(buf))
    return buf.value.decode(errors="replace")


def check(status: int, allow=(WD_OK,)) -> int:
    if status not in allow:
        raise WdError(status, last_error() or lib().wd_error_string(status).decode())
    return status
