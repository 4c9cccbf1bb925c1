"""The seeded input generators: recipe properties and determinism."""
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rows_sorted_distinct(M):
    for i in range(M.nrows):
        r = M.col[M.rowptr[i]:M.rowptr[i + 1]]
        assert np.all(np.diff(r) > 0)
        if r.size:
            assert 0 <= r[0] and r[-1] < M.ncols


def test_er_recipe():
    A = synth.er(500, 8, 1)
    assert A.nnz == 4000 and np.all(np.diff(A.rowptr) == 8)
    _rows_sorted_distinct(A)


def test_tall_skinny_recipe():
    B = synth.tall_skinny(4000, 64, 0.10, 2)
    cnt = np.diff(B.rowptr)
    assert set(np.unique(cnt)) <= {6, 7}            # 6.4 stochastically rounded
    assert abs(cnt.mean() - 6.4) < 0.1
    _rows_sorted_distinct(B)
    D = synth.tall_skinny(300, 256, 0.5, 3)          # dense rows use selection sampling
    assert np.all(np.diff(D.rowptr) == 128)
    _rows_sorted_distinct(D)
    hist = np.bincount(D.col, minlength=256)
    assert hist.min() > 100                          # roughly uniform columns


def test_rmat_recipe():
    A = synth.rmat(10, 16, 4)
    _rows_sorted_distinct(A)
    for i in range(A.nrows):
        assert not np.any(A.col[A.rowptr[i]:A.rowptr[i + 1]] == i)  # no self loops
    deg = np.diff(A.rowptr)
    assert deg.max() > 8 * deg.mean()                # skewed degrees
    S = synth.rmat(9, 8, 5, symmetrize=True)
    M = set()
    for i in range(S.nrows):
        for j in S.col[S.rowptr[i]:S.rowptr[i + 1]]:
            M.add((i, int(j)))
    assert all((j, i) in M for (i, j) in M)
    Q = synth.rmat(10, 8, 6, n=700)                  # n < 2^scale redraws endpoints
    assert Q.nrows == 700 and Q.col.max() < 700


def test_values():
    u = synth.uniform(100000, 9)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.01
    assert np.all(u * 2**24 == np.floor(u * 2**24))
    z = synth.normal(200000, 9)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_deterministic_across_thread_counts():
    code = ("import sys; sys.path.insert(0, %r); import synth, hashlib;"
            "A = synth.rmat(11, 16, 77);"
            "B = synth.tall_skinny(A.nrows, 128, 0.05, 78);"
            "v = synth.normal(B.nnz, 79);"
            "h = hashlib.sha1(); [h.update(x.tobytes()) for x in (A.rowptr, A.col, B.rowptr, B.col, v)];"
            "print(h.hexdigest())") % ROOT
    outs = []
    for t in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                                   capture_output=True, text=True).stdout.strip())
    assert outs[0] == outs[1]
