"""Multi-threaded CPU baseline of the product (not used by the library).

``spgemm_omp.c`` states the paper's local kernel (Sec. III-C) for the host's
cores: rows of A over OpenMP threads, a dense sparse accumulator (SPA) of d
floats per thread, counts then values, FP32.  ``bench.py`` reports its
forward throughput beside the GPU numbers as ``cpu_plain``; it is a plain
baseline written for the same hardware box, distinct from the FP64
single-threaded oracle (``oracle/``) that checks results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_omp.c")
_LIB = os.path.join(_HERE, "libcpuplain.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile spgemm_omp.c into libcpuplain.so (gcc -O3 -fopenmp)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            lib.cpu_plain_count.restype = i64
            lib.cpu_plain_count.argtypes = [i64, i32, p, p, p, p, p, i32]
            lib.cpu_plain_numeric.restype = ctypes.c_int
            lib.cpu_plain_numeric.argtypes = [i64, i32, p, p, p, p, p, p, p, p, p, i32]
            lib.cpu_plain_max_threads.restype = i32
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_L().cpu_plain_max_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def spgemm(A, B, threads: int = 0):
    """C = A * B (plus-times, FP32) on the host: returns (rowptr, col, val).
    A and B are host CSR matrices (rowptr int64, col int32, val float32)."""
    lib = _L()
    t = threads if threads > 0 else max_threads()
    n, d = int(A.nrows), int(B.ncols)
    Ap = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    Ai = np.ascontiguousarray(A.col, dtype=np.int32)
    Ax = None if A.val is None else np.ascontiguousarray(A.val, dtype=np.float32)
    Bp = np.ascontiguousarray(B.rowptr, dtype=np.int64)
    Bi = np.ascontiguousarray(B.col, dtype=np.int32)
    Bx = None if B.val is None else np.ascontiguousarray(B.val, dtype=np.float32)
    Cp = np.zeros(n + 1, dtype=np.int64)
    nnz = lib.cpu_plain_count(n, d, _p(Ap), _p(Ai), _p(Bp), _p(Bi), _p(Cp), t)
    if nnz < 0:
        raise ValueError("cpu_plain: a column index out of range (or out of memory)")
    Ci = np.empty(max(nnz, 1), dtype=np.int32)
    Cx = np.empty(max(nnz, 1), dtype=np.float32)
    if lib.cpu_plain_numeric(n, d, _p(Ap), _p(Ai), _p(Ax), _p(Bp), _p(Bi), _p(Bx), _p(Cp), _p(Ci), _p(Cx), t):
        raise ValueError("cpu_plain: a column index out of range (or out of memory)")
    return Cp, Ci[:nnz], Cx[:nnz]
