"""Seeded synthetic inputs for TS-SpGEMM (generator only: no product arithmetic).

Both sides of every parity check draw their inputs from this module: the CUDA
path (through ``paper_2408_11988_gb300``) and the CPU oracle (``oracle``).  It
holds the input recipe of the paper's workload classes (Sec. V-A: Erdos-Renyi
graphs of average degree 8, scale-free web graphs, B with d columns and a
given per-row sparsity) as R-MAT / ER stand-ins; see ``synth.c`` for the
conventions.  Matrices are returned as :class:`CSR` with int64 row pointers,
int32 column indices (ascending, distinct per row) and optional float32 values.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

# seed of workload k is BASE_SEED + k (one seed per configuration)
BASE_SEED = 240811988


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
            dbl = ctypes.c_double
            sig = {
                "synth_er": (None, [i64, i64, i64, u64, p, p]),
                "synth_ts_rowptr": (None, [i64, i64, dbl, u64, p]),
                "synth_ts_cols": (None, [i64, i64, u64, p, p]),
                "synth_uniform_f32": (None, [i64, u64, p]),
                "synth_normal_f32": (None, [i64, u64, p]),
                "synth_permutation": (None, [i64, u64, p]),
                "synth_sources": (i64, [i64, p, i64, u64, p]),
                "synth_rmat_edges": (None, [i64, i64, dbl, dbl, dbl, i64, u64, p, p, p]),
                "synth_csr_from_edges": (i64, [i64, i64, p, p, ctypes.c_int, ctypes.c_int, p, p]),
                "synth_num_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class CSR:
    """Host CSR matrix: rowptr int64[nrows+1], col int32[nnz], val float32[nnz] or None."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def with_values(self, val: Optional[np.ndarray]) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rowptr, self.col, val)


def threads() -> int:
    return int(_L().synth_num_threads())


def uniform(m: int, seed: int) -> np.ndarray:
    """m float32 values, uniform on [0,1), 24 random bits each."""
    out = np.empty(m, dtype=np.float32)
    if m:
        _L().synth_uniform_f32(m, seed, _ptr(out))
    return out


def normal(m: int, seed: int) -> np.ndarray:
    """m float32 values, standard normal (Box-Muller)."""
    out = np.empty(m, dtype=np.float32)
    if m:
        _L().synth_normal_f32(m, seed, _ptr(out))
    return out


def er(n: int, k: int, seed: int, ncols: Optional[int] = None) -> CSR:
    """Erdos-Renyi pattern with exactly k distinct uniform columns per row."""
    ncols = n if ncols is None else ncols
    k = min(k, ncols)
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(n * k, dtype=np.int32)
    _L().synth_er(n, ncols, k, seed, _ptr(rowptr), _ptr(col))
    return CSR(n, ncols, rowptr, col)


def tall_skinny(n: int, d: int, density: float, seed: int) -> CSR:
    """n x d pattern whose rows hold density*d distinct uniform columns
    (stochastically rounded per row)."""
    rowptr = np.empty(n + 1, dtype=np.int64)
    _L().synth_ts_rowptr(n, d, float(density), seed, _ptr(rowptr))
    col = np.empty(int(rowptr[-1]), dtype=np.int32)
    if col.size:
        _L().synth_ts_cols(n, d, seed, _ptr(rowptr), _ptr(col))
    return CSR(n, d, rowptr, col)


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _L().synth_permutation(n, seed, _ptr(out))
    return out


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, symmetrize: bool = False, n: Optional[int] = None,
         permute: bool = True) -> CSR:
    """R-MAT pattern: edge_factor*n edges, self-loops and duplicates removed,
    vertices relabelled by a seeded permutation; n defaults to 2**scale and
    smaller n redraws edges with an endpoint >= n."""
    n = (1 << scale) if n is None else int(n)
    assert 0 < n <= (1 << scale) < (1 << 31)
    m = edge_factor * n
    perm = permutation(n, seed) if permute else None
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    _L().synth_rmat_edges(scale, m, a, b, c, n, seed, _ptr(perm), _ptr(src), _ptr(dst))
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(m * (2 if symmetrize else 1), dtype=np.int32)
    nnz = _L().synth_csr_from_edges(n, m, _ptr(src), _ptr(dst), int(symmetrize), 1,
                                    _ptr(rowptr), _ptr(col))
    if nnz < 0:
        raise MemoryError("synth_csr_from_edges: allocation failed")
    del src, dst
    return CSR(n, n, rowptr, col[:nnz].copy())


def sources(A: CSR, count: int, seed: int) -> np.ndarray:
    """count distinct vertices of nonzero out-degree (BFS sources)."""
    out = np.empty(count, dtype=np.int32)
    got = _L().synth_sources(A.nrows, _ptr(A.rowptr), count, seed, _ptr(out))
    return out[:got].copy()


# ---------------------------------------------------------------------------
# Workloads.  Each returns host matrices; sizes are parameters so that tests can
# run the same recipe at small scale.
# ---------------------------------------------------------------------------

def er_product(n: int = 16384, k: int = 8, d: int = 64, density: float = 0.10,
               seed: int = BASE_SEED + 1):
    """Erdos-Renyi A (k per row, U(0,1) values) times B (n x d, density, U(0,1))."""
    A = er(n, k, seed)
    A.val = uniform(A.nnz, seed + 101)
    B = tall_skinny(n, d, density, seed + 202)
    B.val = uniform(B.nnz, seed + 303)
    return A, B


def rmat_embedding(scale: int = 22, edge_factor: int = 16, d: int = 256, density: float = 0.05,
                   seed: int = BASE_SEED + 3, b_values: str = "normal"):
    """Directed R-MAT A with U(0,1) values times B (n x d, density) with N(0,1)
    (or U(0,1)) values: the sparse-embedding product shape."""
    A = rmat(scale, edge_factor, seed)
    A.val = uniform(A.nnz, seed + 101)
    B = tall_skinny(A.nrows, d, density, seed + 202)
    B.val = normal(B.nnz, seed + 303) if b_values == "normal" else uniform(B.nnz, seed + 303)
    return A, B


def grad_output(nnz_c: int, seed: int) -> np.ndarray:
    """dC values on C's pattern, N(0,1)."""
    return normal(nnz_c, seed + 404)


def msbfs_graph(scale: int = 20, edge_factor: int = 16, nsources: int = 128,
                seed: int = BASE_SEED + 2):
    """Symmetrised pattern-only R-MAT graph and distinct BFS sources of nonzero degree."""
    A = rmat(scale, edge_factor, seed, symmetrize=True)
    src = sources(A, nsources, seed + 505)
    return A, src


def batched_instances(count: int = 64, seed: int = BASE_SEED + 4, log2n_lo: float = 12.0,
                      log2n_hi: float = 18.0, ds=(32, 64, 128, 256)):
    """Uneven batch: n log-uniform in [2^lo, 2^hi], edge factor U{8..32},
    d from ds, density log-uniform in [1%, 50%]; U(0,1) values."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for b in range(count):
        n = int(math.floor(2.0 ** rng.uniform(log2n_lo, log2n_hi)))
        n = max(n, 2)
        scale = max(1, int(math.ceil(math.log2(n))))
        ef = int(rng.integers(8, 33))
        d = int(ds[int(rng.integers(0, len(ds)))])
        dens = float(math.exp(rng.uniform(math.log(0.01), math.log(0.50))))
        s = seed * 1000 + 17 * b
        A = rmat(scale, ef, s, n=n)
        A.val = uniform(A.nnz, s + 101)
        B = tall_skinny(n, d, dens, s + 202)
        B.val = uniform(B.nnz, s + 303)
        out.append((A, B))
    return out


def sparse_embedding(n: int, d: int, k: int, seed: int, scale: float = 0.1) -> CSR:
    """n x d embedding with exactly k distinct uniform columns per row and
    values scale * N(0,1) (a sparse Force2Vec starting point)."""
    Z = er(n, k, seed, ncols=d)
    Z.val = (normal(Z.nnz, seed + 1) * np.float32(scale)).astype(np.float32)
    return Z


def negatives(b: int, s: int, n: int, seed: int) -> np.ndarray:
    """b*s negative-sample vertex ids, uniform on [0, n) (24-bit draws)."""
    u = uniform(b * s, seed).astype(np.float64)
    return np.minimum((u * n).astype(np.int64), n - 1).astype(np.int32)


def force2vec_inputs(scale: int = 20, edge_factor: int = 16, d: int = 128, k: int = 26,
                     seed: int = BASE_SEED + 6):
    """Symmetrised pattern-only R-MAT graph and its sparse starting embedding
    (d = 128, 80 % sparse: k = 26 entries per row)."""
    A = rmat(scale, edge_factor, seed, symmetrize=True)
    Z = sparse_embedding(A.nrows, d, k, seed + 11)
    return A, Z
