"""ctypes view of the C ABI in include/tsspgemm.h (argument marshalling only).

The shared library is built in-tree by :mod:`paper_2408_11988_gb300.build`.
If it is missing, every entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

c_int32, c_int64, c_void_p, c_size_t = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t

TS_OK = 0
TS_ERR_INVALID_ARG = -1
TS_ERR_BAD_CSR = -2
TS_ERR_UNSUPPORTED = -3
TS_ERR_WORKSPACE_TOO_SMALL = -4
TS_ERR_CAPACITY = -5
TS_ERR_OVERFLOW = -6
TS_ERR_CUDA = -7
TS_ERR_STATE = -8

PLUS_TIMES = 0
OR_SELECT2ND = 1

ACC_AUTO = 0
ACC_DENSE = 1
ACC_HASH = 2
ACC_COPIES = 3
ACC_DENSE_B = 4


class CsrDesc(ctypes.Structure):
    _fields_ = [("nrows", c_int64), ("ncols", c_int64), ("nnz", c_int64),
                ("rowptr", c_void_p), ("col", c_void_p), ("val", c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("accum", c_int32), ("col_tile", c_int32), ("cta_min_flops", c_int64),
                ("warps_per_cta", c_int32), ("hash_slots", c_int32), ("group", c_int32),
                ("pack_b", c_int32), ("stage", c_int32), ("sym_group", c_int32), ("bwd_group", c_int32),
                ("row_lanes", c_int32), ("dB_mode", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for k, v in (d or {}).items():
            setattr(t, k, int(v))
        return t


class TSError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {status_string(status)}: {msg}")
        self.status = status


P = ctypes.POINTER
_SIGS = {
    "ts_last_error": (ctypes.c_char_p, []),
    "ts_status_string": (ctypes.c_char_p, [c_int32]),
    "ts_version": (c_int32, []),
    "ts_kernel_launches": (c_int64, []),
    "ts_validate_workspace_size": (c_size_t, []),
    "ts_csr_validate": (c_int32, [P(CsrDesc), P(c_int64), c_void_p, c_size_t, c_void_p]),
    "ts_plan_create": (c_int32, [P(CsrDesc), P(CsrDesc), c_int32, P(Tuning), P(c_void_p)]),
    "ts_plan_destroy": (c_int32, [c_void_p]),
    "ts_plan_get_tuning": (c_int32, [c_void_p, P(Tuning)]),
    "ts_plan_set_tuning": (c_int32, [c_void_p, P(Tuning)]),
    "ts_workspace_size": (c_int32, [c_void_p, P(c_size_t)]),
    "ts_workspace_check": (c_int32, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_spgemm_symbolic": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), c_void_p, P(c_int64),
                                     c_void_p, c_size_t, c_void_p]),
    "ts_spgemm_numeric": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p,
                                    c_size_t, c_void_p]),
    "ts_spgemm_backward": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_spgemm_backward_dA": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p,
                                        c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_spgemm_backward_dB": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p,
                                        c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_plan_autotune": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p, c_void_p,
                                   c_void_p, c_int32, P(Tuning), c_void_p, c_size_t, c_void_p]),
    "msbfs_workspace_size": (c_int32, [c_int64, c_int64, c_int64, P(c_size_t)]),
    "msbfs_init": (c_int32, [c_int64, c_int64, c_void_p, c_void_p, c_void_p, P(CsrDesc), c_void_p]),
    "msbfs_step": (c_int32, [P(CsrDesc), P(CsrDesc), c_void_p, c_void_p, c_int32, P(CsrDesc),
                             c_int64, P(c_int64), c_void_p, c_size_t, c_void_p]),
    "msbfs_emit": (c_int32, [P(CsrDesc), c_int64, c_void_p, c_size_t, c_void_p]),
    "msbfs_step_parents": (c_int32, [P(CsrDesc), P(CsrDesc), c_void_p, c_void_p, c_void_p, c_int32, P(CsrDesc),
                                     c_int64, P(c_int64), c_void_p, c_size_t, c_void_p]),
    "msbfs_init_parents": (c_int32, [c_int64, c_int64, c_void_p, c_void_p, c_void_p]),
    "f2v_workspace_size": (c_int32, [c_int64, c_int64, c_int64, c_int64, c_int32, c_int32, P(c_size_t)]),
    "f2v_step": (c_int32, [P(CsrDesc), P(CsrDesc), c_int64, c_int64, c_void_p, c_int32, ctypes.c_float, c_int32,
                           c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_batched_plan_create": (c_int32, [c_int32, P(CsrDesc), P(CsrDesc), c_int32, P(Tuning),
                                         P(c_void_p)]),
    "ts_batched_plan_destroy": (c_int32, [c_void_p]),
    "ts_batched_workspace_size": (c_int32, [c_void_p, P(c_size_t)]),
    "ts_batched_bounds": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(c_int64), c_void_p,
                                    c_size_t, c_void_p]),
    "ts_batched_bind": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), c_void_p,
                                  c_size_t, c_void_p]),
    "ts_spgemm_batched": (c_int32, [c_void_p, c_int32, P(CsrDesc), P(CsrDesc), P(CsrDesc),
                                    c_void_p, c_size_t, c_void_p]),
    "ts_spgemm_batched_backward": (c_int32, [c_void_p, c_int32, P(c_void_p), P(c_void_p),
                                             P(c_void_p), c_void_p, c_size_t, c_void_p]),
    "ts_batched_bind_grads": (c_int32, [c_void_p, c_int32, P(c_void_p), P(c_void_p), P(c_void_p), c_void_p,
                                        c_size_t, c_void_p]),
    "ts_batched_check": (c_int32, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "ts_batched_autotune": (c_int32, [c_void_p, c_int32, P(Tuning), c_void_p, c_size_t, c_void_p]),
    "ts_batched_get_tuning": (c_int32, [c_void_p, c_int32, P(Tuning)]),
    "ts_noalloc_scratch_bytes": (c_size_t, []),
    "ts_spgemm_forward_noalloc": (c_int32, [c_void_p, P(CsrDesc), P(CsrDesc), P(CsrDesc), P(c_int64),
                                            c_void_p]),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libtsspgemm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            handle = ctypes.CDLL(LIB, mode=ctypes.RTLD_LOCAL)
            for name, (res, args) in _SIGS.items():
                f = getattr(handle, name)
                f.restype = res
                f.argtypes = args
            _lib = handle
    return _lib


def status_string(s: int) -> str:
    return lib().ts_status_string(s).decode()


def last_error() -> str:
    return lib().ts_last_error().decode()


def check(status: int, fn: str) -> int:
    if status != TS_OK:
        raise TSError(status, fn, last_error())
    return status


def call(fn: str, *args) -> None:
    """Call fn and raise TSError on a non-zero status."""
    check(getattr(lib(), fn)(*args), fn)
