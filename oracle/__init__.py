"""ORACLE -- test infrastructure only.

A plain, slow, single-threaded CPU statement of the TS-SpGEMM hot path in
double precision (``oracle.c``), with a thin ctypes wrapper.  It is used by
``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``; nothing in the product package imports it, and it shares no
code with the CUDA path.  Inputs come from ``synth`` (seeded generators).

What each function follows:
  spgemm      -- paper Sec. II-A (semiring product, flops = multiplications)
                 and Sec. III-A, Eq. 1 (row-wise Gustavson).
  spgemm_count -- the row counts of that product's pattern (its first half).
  msbfs       -- paper Alg. 3 (multi-source BFS over the boolean semiring).
  bfs_levels  -- textbook FIFO-queue BFS (hop distance), one source.
  backward*   -- gradients of <dC, A*B> w.r.t. the stored values of A and B
                 (the product is bilinear, so these are exact sums).
Every function is pinned by tests/test_oracle.py against something other than
itself: dense brute force, scipy's sparse product, identities, a textbook
queue BFS and exact finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PLUS_TIMES = 0
OR_SELECT2ND = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, single-threaded, -O2)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            sig = {
                "oracle_spgemm_count": (i64, [i64, p, p, p, p, p, i64, p]),
                "oracle_spgemm": (ci, [i64, ci, p, p, p, p, p, p, p, i64, p, p, p, p]),
                "oracle_msbfs": (i64, [i64, p, p, i64, p, p, p, i64]),
                "oracle_msbfs_parents": (i64, [i64, p, p, i64, p, p, p, p, i64]),
                "oracle_backward": (ci, [i64, i64, p, p, p, i64, p, p, p, p, p, p, p, p, p, p]),
                "oracle_backward_dA_rows": (ci, [i64, p, p, p, p, p, p, p, p, p, i64, p, p]),
                "oracle_backward_dB_rows": (ci, [i64, p, p, p, p, p, p, p, p, p, i64, p, p]),
                "oracle_bfs_levels": (i64, [i64, p, p, ctypes.c_int32, p]),
                "oracle_f2v_topk": (ci, [i64, i64, i64, p, p, p]),
                "oracle_f2v_step": (ci, [i64, p, p, i64, i64, p, p, i64, i64, p, i64, ctypes.c_double,
                                         p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def spgemm(A, B, semiring: int = PLUS_TIMES, rows: Optional[np.ndarray] = None):
    """C = A*B (Eq. 1) for all rows, or for the selected rows of A.

    A and B are objects with nrows/ncols/rowptr/col/val (``synth.CSR``).
    Returns (rowptr int64[nsel+1], col int32[nnz], val float64[nnz] | None,
    bound float64[nnz] | None); bound[e] = sum of |A(i,k)|*|B(k,j)| for the
    entry.  Values are None for the boolean semiring.
    """
    d = B.ncols
    Ap, Ai = _i64(A.rowptr), _i32(A.col)
    Bp, Bi = _i64(B.rowptr), _i32(B.col)
    sel = None if rows is None else _i64(rows)
    nsel = A.nrows if rows is None else len(sel)
    cnt = np.zeros(max(nsel, 1), dtype=np.int64)
    tot = _L().oracle_spgemm_count(d, _p(Ap), _p(Ai), _p(Bp), _p(Bi), _p(sel), nsel, _p(cnt))
    if tot < 0:
        raise MemoryError("oracle_spgemm_count")
    Cp = np.zeros(nsel + 1, dtype=np.int64)
    np.cumsum(cnt[:nsel], out=Cp[1:])
    Ci = np.empty(max(tot, 1), dtype=np.int32)
    if semiring == PLUS_TIMES:
        Ax, Bx = _f64(A.val), _f64(B.val)
        Cx = np.empty(max(tot, 1), dtype=np.float64)
        Cb = np.empty(max(tot, 1), dtype=np.float64)
    else:
        Ax = Bx = Cx = Cb = None
    st = _L().oracle_spgemm(d, semiring, _p(Ap), _p(Ai), _p(Ax), _p(Bp), _p(Bi), _p(Bx), _p(sel),
                            nsel, _p(Cp), _p(Ci), _p(Cx), _p(Cb))
    if st != 0:
        raise RuntimeError(f"oracle_spgemm failed ({st})")
    if semiring == PLUS_TIMES:
        return Cp, Ci[:tot], Cx[:tot], Cb[:tot]
    return Cp, Ci[:tot], None, None


def spgemm_count(A, B) -> np.ndarray:
    """Row pointers of C = A*B (int64[n+1]): nnz(C_i) is the number of distinct
    columns over the rows of B that row i of A selects (Eq. 1's pattern)."""
    Ap, Ai = _i64(A.rowptr), _i32(A.col)
    Bp, Bi = _i64(B.rowptr), _i32(B.col)
    n = A.nrows
    cnt = np.zeros(max(n, 1), dtype=np.int64)
    tot = _L().oracle_spgemm_count(B.ncols, _p(Ap), _p(Ai), _p(Bp), _p(Bi), None, n, _p(cnt))
    if tot < 0:
        raise MemoryError("oracle_spgemm_count")
    Cp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt[:n], out=Cp[1:])
    return Cp


def msbfs(A, sources: np.ndarray, maxlev: int = 4096):
    """Alg. 3 from the given sources.  Returns (levels int32[n, d], number of
    products computed, frontier nnz per level (index 0 = initial frontier))."""
    n = A.nrows
    src = _i32(sources)
    d = len(src)
    levels = np.empty((n, d), dtype=np.int32)
    fnnz = np.zeros(maxlev, dtype=np.int64)
    prods = _L().oracle_msbfs(n, _p(_i64(A.rowptr)), _p(_i32(A.col)), d, _p(src), _p(levels),
                              _p(fnnz), maxlev)
    if prods < 0:
        raise RuntimeError(f"oracle_msbfs failed ({prods})")
    return levels, int(prods), fnnz[: prods + 1].copy()


def msbfs_parents(A, sources: np.ndarray, maxlev: int = 4096):
    """Alg. 3 with the (sel2nd, min) semiring (BFS-tree variant, Sec. IV):
    returns (levels int32[n, d], parents int32[n, d], products, frontier nnz
    per level).  Dense n x d working arrays: small inputs only."""
    n = A.nrows
    src = _i32(sources)
    d = len(src)
    levels = np.empty((n, d), dtype=np.int32)
    parents = np.empty((n, d), dtype=np.int32)
    fnnz = np.zeros(maxlev, dtype=np.int64)
    prods = _L().oracle_msbfs_parents(n, _p(_i64(A.rowptr)), _p(_i32(A.col)), d, _p(src), _p(levels),
                                      _p(parents), _p(fnnz), maxlev)
    if prods < 0:
        raise RuntimeError(f"oracle_msbfs_parents failed ({prods})")
    return levels, parents, int(prods), fnnz[: prods + 1].copy()


def f2v_step(A, Z, r0: int, b: int, neg: np.ndarray, s: int, lr: float, k: int):
    """Sparse Force2Vec step on rows [r0, r0+b) (paper Sec. IV, sparse
    embedding; readings in oracle.c).  Z: CSR with exactly k entries per row.
    Returns (U[b, d] float64, Ubound[b, d], Ncol[b, k], Nval[b, k])."""
    d = Z.ncols
    U = np.empty((max(b, 1), d), dtype=np.float64)
    Ub = np.empty_like(U)
    Ncol = np.empty((max(b, 1), k), dtype=np.int32)
    Nval = np.empty((max(b, 1), k), dtype=np.float64)
    st = _L().oracle_f2v_step(A.nrows, _p(_i64(A.rowptr)), _p(_i32(A.col)), d, k, _p(_i32(Z.col)),
                              _p(_f64(Z.val)), r0, b, _p(_i32(neg)), s, float(lr), _p(U), _p(Ub),
                              _p(Ncol), _p(Nval))
    if st != 0:
        raise RuntimeError("oracle_f2v_step failed")
    return U[:b], Ub[:b], Ncol[:b], Nval[:b]


def f2v_topk(U: np.ndarray, k: int):
    """The k entries of largest magnitude of each row of U (ties: smaller
    column), ascending columns: (Ncol[rows, k], Nval[rows, k])."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    rows, d = U.shape
    Ncol = np.empty((max(rows, 1), k), dtype=np.int32)
    Nval = np.empty((max(rows, 1), k), dtype=np.float64)
    if _L().oracle_f2v_topk(rows, d, k, _p(U), _p(Ncol), _p(Nval)) != 0:
        raise MemoryError("oracle_f2v_topk")
    return Ncol[:rows], Nval[:rows]


def bfs_levels(A, source: int) -> np.ndarray:
    """Hop distances from one source by a FIFO-queue BFS (-1 = unreachable)."""
    out = np.empty(A.nrows, dtype=np.int32)
    r = _L().oracle_bfs_levels(A.nrows, _p(_i64(A.rowptr)), _p(_i32(A.col)), int(source), _p(out))
    if r < 0:
        raise MemoryError("oracle_bfs_levels")
    return out


def backward(A, B, C_rowptr, C_col, dC):
    """(dA, dA_bound, dB, dB_bound) of L = <dC, A*B> for plus-times."""
    n, d = A.nrows, B.ncols
    dA = np.empty(max(A.nnz, 1), dtype=np.float64)
    dAb = np.empty_like(dA)
    dB = np.empty(max(B.nnz, 1), dtype=np.float64)
    dBb = np.empty_like(dB)
    st = _L().oracle_backward(n, d, _p(_i64(A.rowptr)), _p(_i32(A.col)), _p(_f64(A.val)),
                              B.nrows, _p(_i64(B.rowptr)), _p(_i32(B.col)), _p(_f64(B.val)),
                              _p(_i64(C_rowptr)), _p(_i32(C_col)), _p(_f64(dC)),
                              _p(dA), _p(dAb), _p(dB), _p(dBb))
    if st != 0:
        raise RuntimeError(f"oracle_backward failed ({st})")
    return dA[: A.nnz], dAb[: A.nnz], dB[: B.nnz], dBb[: B.nnz]


def backward_dA_rows(A, B, C_rowptr, C_col, dC, rows):
    """dA restricted to the entries of the selected rows of A (row after row)."""
    rows = _i64(rows)
    m = int(sum(int(A.rowptr[r + 1] - A.rowptr[r]) for r in rows))
    out = np.empty(max(m, 1), dtype=np.float64)
    bnd = np.empty_like(out)
    st = _L().oracle_backward_dA_rows(B.ncols, _p(_i64(A.rowptr)), _p(_i32(A.col)),
                                      _p(_i64(B.rowptr)), _p(_i32(B.col)), _p(_f64(B.val)),
                                      _p(_i64(C_rowptr)), _p(_i32(C_col)), _p(_f64(dC)),
                                      _p(rows), len(rows), _p(out), _p(bnd))
    if st != 0:
        raise RuntimeError(f"oracle_backward_dA_rows failed ({st})")
    return out[:m], bnd[:m]


def backward_dB_rows(A, B, C_rowptr, C_col, dC, krows):
    """dB restricted to the entries of the selected rows of B (row after row)."""
    krows = _i64(krows)
    m = int(sum(int(B.rowptr[k + 1] - B.rowptr[k]) for k in krows))
    out = np.empty(max(m, 1), dtype=np.float64)
    bnd = np.empty_like(out)
    st = _L().oracle_backward_dB_rows(A.nrows, _p(_i64(A.rowptr)), _p(_i32(A.col)), _p(_f64(A.val)),
                                      _p(_i64(B.rowptr)), _p(_i32(B.col)),
                                      _p(_i64(C_rowptr)), _p(_i32(C_col)), _p(_f64(dC)),
                                      _p(krows), len(krows), _p(out), _p(bnd))
    if st != 0:
        raise RuntimeError(f"oracle_backward_dB_rows failed ({st})")
    return out[:m], bnd[:m]
