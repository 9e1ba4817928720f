"""ctypes binding of the C ABI in include/cheb_expmv.h (argument marshalling only).

The library is loaded from this package directory. If it is missing it is built
with nvcc; if that fails, loading raises - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class TuneResult(ctypes.Structure):
    _fields_ = [
        ("path", ctypes.c_int),
        ("l", ctypes.c_int),
        ("h", ctypes.c_int),
        ("blocking", ctypes.c_int),
        ("candidates", ctypes.c_int),
        ("best_ms_per_step", ctypes.c_double),
        ("default_ms_per_step", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int),
        ("time_splits", ctypes.c_int),
        ("matvecs", ctypes.c_int64),
        ("emin", c_double),
        ("emax", c_double),
        ("center", c_double),
        ("radius", c_double),
        ("a", c_double),
        ("trunc_bound", c_double),
        ("norm", c_double),
        ("energy", c_double),
        ("eval_bound", c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes); mirrors include/cheb_expmv.h
SIGNATURES = {
    "cheb_status_string": (ctypes.c_char_p, [c_int]),
    "cheb_version": (ctypes.c_char_p, []),
    "cheb_coefficients": (c_int, [c_double, c_double, c_double, c_double, c_int, c_int, _dp, _ip, _dp]),
    "cheb_workspace_bytes": (c_size_t, [c_int, c_int]),
    "cheb_ising_bounds": (c_int, [c_int, _dp, _dp, c_void_p, c_size_t, c_void_p, _dp, _dp]),
    "cheb_expmv": (c_int, [c_int, _dp, _dp, c_double, c_double, c_void_p, c_int, c_double, c_int, c_int,
                           c_void_p, c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_expmv_path": (c_int, [c_int, _dp, _dp, c_double, c_double, c_void_p, c_int, c_double, c_int, c_int,
                                c_int, c_void_p, c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_poly_apply": (c_int, [c_int, _dp, _dp, c_double, c_double, c_double, c_int, _dp, c_void_p, c_int,
                                c_int, c_void_p, c_size_t, c_void_p]),
    "cheb_monomial_to_chebyshev": (c_int, [c_int, _dp, _dp]),
    "cheb_energy": (c_int, [c_int, _dp, _dp, c_void_p, c_int, c_void_p, c_size_t, c_void_p, _dp, _dp]),
    "cheb_set_fused_split": (c_int, [c_int, c_int, c_int]),
    "cheb_get_fused_split": (c_int, [c_int, _ip, _ip]),
    "cheb_set_fused_split_fp64": (c_int, [c_int, c_int, c_int]),
    "cheb_get_fused_split_fp64": (c_int, [c_int, _ip, _ip]),
    "cheb_set_fused_blocking": (c_int, [c_int]),
    "cheb_get_fused_blocking": (c_int, []),
    "cheb_set_fused_compensated": (c_int, [c_int]),
    "cheb_get_fused_compensated": (c_int, []),
    "cheb_expmv_noalloc": (c_int, [c_int, _dp, _dp, c_double, c_double, c_void_p, c_int, c_double, c_int, c_int,
                                   c_void_p, ctypes.POINTER(Info)]),
    "cheb_anneal": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, c_void_p, c_int, c_double, c_int, c_void_p,
                            c_void_p, c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_anneal_general": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, _dp, c_void_p, c_int, c_double, c_int,
                                    c_void_p, c_void_p, c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_magnus4": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, c_void_p, c_int, c_double, c_int, c_void_p, c_void_p,
                             c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_magnus4_nodes": (c_int, [c_double, c_int, ctypes.c_void_p, c_void_p, _dp, _dp]),
    "cheb_magnus4_adjoint": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, c_void_p, c_void_p, c_void_p, c_int, c_double,
                                     c_int, _dp, _dp, _dp, _dp, c_void_p, c_size_t, c_void_p]),
    "cheb_magnus4_adaptive_workspace_bytes": (c_size_t, [c_int, c_int]),
    "cheb_magnus4_adaptive": (c_int, [c_int, _dp, _dp, c_double, ctypes.c_void_p, c_void_p, c_int, c_double, c_void_p,
                                      c_int, c_int, c_void_p, c_size_t, c_void_p, _ip, _dp]),
    "cheb_batched_workspace_bytes": (c_size_t, [c_int, _ip, c_int]),
    "cheb_set_batch_persistent": (c_int, [c_int]),
    "cheb_get_batch_persistent": (c_int, []),
    "cheb_expmv_batched": (c_int, [c_int, _ip, ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp, _dp, c_void_p, c_int,
                                   c_double, c_int, c_void_p, c_size_t, c_void_p, ctypes.POINTER(Info)]),
    "cheb_adjoint_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "cheb_anneal_adjoint": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, c_void_p, c_void_p, c_void_p, c_int, c_double,
                                    c_int, _dp, _dp, _dp, _dp, c_void_p, c_size_t, c_void_p]),
    "cheb_anneal_general_adjoint": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, _dp, c_void_p, c_void_p, c_void_p, c_int,
                                            c_double, c_int, _dp, _dp, _dp, _dp, _dp, c_void_p, c_size_t, c_void_p]),
    "cheb_anneal_graph_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "cheb_anneal_graph_create": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, _dp, c_void_p, c_int, c_double, c_int,
                                         c_void_p, c_void_p, c_size_t, c_void_p, ctypes.POINTER(c_void_p)]),
    "cheb_anneal_graph_launch": (c_int, [c_void_p, c_void_p]),
    "cheb_anneal_graph_destroy": (None, [c_void_p]),
    "cheb_anneal_checkpointed": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, c_void_p, c_int, c_double, c_int,
                                         c_void_p, c_void_p, c_size_t, c_void_p]),
    "cheb_anneal_general_checkpointed": (c_int, [c_int, _dp, _dp, c_int, _dp, _dp, _dp, c_void_p, c_int, c_double,
                                                 c_int, c_void_p, c_void_p, c_size_t, c_void_p]),
    "cheb_energy_grad": (c_int, [c_int, _dp, _dp, c_void_p, c_void_p, c_int, _dp, _dp, _dp, c_void_p, c_size_t,
                                 c_void_p]),
    "cheb_wait_selftest": (c_int, [c_void_p, c_size_t, c_void_p]),
    "cheb_pair_schedule_check": (c_int, [c_int, c_int, c_int, c_int, ctypes.POINTER(ctypes.c_longlong)]),
    "cheb_workspace_status": (c_int, [c_void_p, c_size_t, c_void_p]),
    "cheb_autotune_workspace_bytes": (c_size_t, [c_int, c_int]),
    "cheb_autotune": (c_int, [c_int, c_int, c_int, c_void_p, c_size_t, c_void_p, ctypes.POINTER(TuneResult)]),
    "cheb_autotune_load": (c_int, [ctypes.c_char_p, ctypes.c_char_p, _ip]),
    "cheb_autotune_reset": (c_int, []),
    "cheb_set_programmatic_launch": (c_int, [c_int]),
    "cheb_launch_count": (ctypes.c_longlong, []),
    "cheb_profile_enable": (c_int, [c_int]),
    "cheb_profile_reset": (c_int, []),
    "cheb_profile_read": (c_int, [c_int, ctypes.POINTER(ctypes.c_longlong), _dp]),
}

STATUS = {0: "CHEB_OK", 1: "CHEB_ERR_INVALID_ARG", 2: "CHEB_ERR_WORKSPACE", 3: "CHEB_ERR_CUDA",
          4: "CHEB_ERR_TIMEOUT", 5: "CHEB_ERR_NONFINITE", 6: "CHEB_ERR_UNSUPPORTED"}


# cheb_schedule_fn: int (*)(double t, double* A, double* B, void* user)
ScheduleFn = ctypes.CFUNCTYPE(c_int, c_double, _dp, _dp, c_void_p)


def schedule_callback(A, B):
    """Wrap two Python callables A(t), B(t) as a cheb_schedule_fn (keep the returned
    object alive for the duration of the call)."""

    def fn(t, pa, pb, user):
        try:
            pa[0] = float(A(t))
            pb[0] = float(B(t))
            return 0
        except Exception:  # any failure aborts the library call with INVALID_ARG
            return 1

    return ScheduleFn(fn)


class ChebError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


def lib_path() -> str:
    return _build.LIB_PATH


def lib():
    """Load (building first if needed) the CUDA library; raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            if _build.needs_build():
                _build.build()
            L = ctypes.CDLL(_build.LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(code: int, where: str):
    if code != 0:
        raise ChebError(code, where)
