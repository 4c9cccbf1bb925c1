"""Pins of the CPU oracle against things other than itself (no GPU needed).

- dense brute force (numpy float64 matmul of the expanded matrices) and the
  integer product of the patterns, on tiny inputs with empty/full rows;
- scipy's sparse product (an independent SpGEMM) on a mid-size ER case;
- identities A = I, B = I, A = 0, B = 0;
- invariants: nnz(C_i) <= min(d, flops_i), plus-times pattern equals the
  boolean pattern, FP64 row sums;
- hand-worked fixtures in tests/golden (Eq. 1 and Alg. 3);
- a textbook queue BFS for Alg. 3;
- exact central differences (the product is bilinear) and the dense
  formulas dA = (dC B^T) on A's pattern, dB = (A^T dC) on B's pattern.
"""
import json
import os
from collections import deque

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from synth import CSR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_csr(rng, nrows, ncols, density, full_rows=(), empty_rows=(), vals="uniform"):
    mask = rng.random((nrows, ncols)) < density
    for r in full_rows:
        mask[r, :] = True
    for r in empty_rows:
        mask[r, :] = False
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(mask.sum(axis=1))
    col = np.nonzero(mask)[1].astype(np.int32)
    if vals == "uniform":
        val = rng.random(col.size)
    else:
        val = rng.standard_normal(col.size)
    return CSR(nrows, ncols, rowptr, col, val.astype(np.float64))


def dense(M):
    out = np.zeros((M.nrows, M.ncols), dtype=np.float64)
    for i in range(M.nrows):
        s, e = M.rowptr[i], M.rowptr[i + 1]
        out[i, M.col[s:e]] = M.val[s:e] if M.val is not None else 1.0
    return out


def pattern(M):
    out = np.zeros((M.nrows, M.ncols), dtype=np.int64)
    for i in range(M.nrows):
        out[i, M.col[M.rowptr[i]:M.rowptr[i + 1]]] = 1
    return out


def csr_from_result(n, d, res):
    Cp, Ci, Cx, _ = res
    return CSR(n, d, Cp, Ci, Cx)


@pytest.mark.parametrize("n,d,da,db", [(1, 1, 1.0, 1.0), (5, 3, 0.4, 0.5), (17, 32, 0.2, 0.1),
                                       (64, 64, 0.05, 0.3), (40, 7, 0.0, 0.5), (40, 7, 0.3, 0.0),
                                       (33, 64, 0.1, 1.0)])
def test_spgemm_matches_dense_bruteforce(n, d, da, db):
    rng = np.random.default_rng(1000 * n + d)
    full = (0,) if n > 2 else ()
    empty = (n - 1,) if n > 2 else ()
    A = random_csr(rng, n, n, da, full_rows=full, empty_rows=empty, vals="normal")
    B = random_csr(rng, n, d, db, full_rows=(1,) if n > 2 else (), empty_rows=(2,) if n > 3 else ())
    C = csr_from_result(n, d, oracle.spgemm(A, B))
    Pdense = pattern(A) @ pattern(B)
    np.testing.assert_array_equal(pattern(C), (Pdense > 0).astype(np.int64))
    ref = dense(A) @ dense(B)
    absref = np.abs(dense(A)) @ np.abs(dense(B))
    np.testing.assert_allclose(dense(C), ref, rtol=0, atol=1e-12 * max(1.0, absref.max()))
    # boolean semiring: same pattern, no values
    Cb = oracle.spgemm(A, B, semiring=oracle.OR_SELECT2ND)
    np.testing.assert_array_equal(Cb[0], C.rowptr)
    np.testing.assert_array_equal(Cb[1], C.col)
    assert Cb[2] is None


def test_spgemm_matches_scipy():
    A, B = synth.er_product(n=2000, k=8, d=64, density=0.10, seed=7)
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B)
    As = sp.csr_matrix((A.val.astype(np.float64), A.col, A.rowptr), shape=(A.nrows, A.ncols))
    Bs = sp.csr_matrix((B.val.astype(np.float64), B.col, B.rowptr), shape=(B.nrows, B.ncols))
    Cs = (As @ Bs).tocsr()
    Cs.sort_indices()
    np.testing.assert_array_equal(Cp, Cs.indptr)
    np.testing.assert_array_equal(Ci, Cs.indices)
    np.testing.assert_allclose(Cx, Cs.data, rtol=1e-13)
    assert np.all(Cb >= np.abs(Cx) * (1 - 1e-15))


def test_spgemm_count_matches_scipy_pattern():
    # row counts of the pattern alone: the distinct columns per row of the
    # structural product (scipy's product of 0/1 matrices counts products,
    # its nonzeros are the distinct columns since all terms are positive)
    A, B = synth.er_product(n=700, k=5, d=96, density=0.08, seed=17)
    Cp = oracle.spgemm_count(A, B)
    Sa = sp.csr_matrix((np.ones(A.nnz), A.col, A.rowptr), shape=(A.nrows, A.ncols))
    Sb = sp.csr_matrix((np.ones(B.nnz), B.col, B.rowptr), shape=(B.nrows, B.ncols))
    S = (Sa @ Sb).tocsr()
    S.sort_indices()
    np.testing.assert_array_equal(Cp, S.indptr)
    np.testing.assert_array_equal(Cp, oracle.spgemm(A, B)[0])


def test_spgemm_golden_eq1():
    g = json.load(open(os.path.join(GOLDEN, "eq1_small.json")))
    n, d = g["n"], g["d"]
    A = CSR(n, n, np.array(g["A"]["rowptr"]), np.array(g["A"]["col"], dtype=np.int32),
            np.array(g["A"]["val"]))
    B = CSR(n, d, np.array(g["B"]["rowptr"]), np.array(g["B"]["col"], dtype=np.int32),
            np.array(g["B"]["val"]))
    Cp, Ci, Cx, _ = oracle.spgemm(A, B)
    np.testing.assert_array_equal(Cp, g["C"]["rowptr"])
    np.testing.assert_array_equal(Ci, g["C"]["col"])
    np.testing.assert_array_equal(Cx, g["C"]["val"])


def test_identities():
    rng = np.random.default_rng(3)
    n, d = 50, 24
    B = random_csr(rng, n, d, 0.3, empty_rows=(4,), vals="normal")
    B.val = B.val.astype(np.float32).astype(np.float64)
    I = CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    Cp, Ci, Cx, _ = oracle.spgemm(I, B)            # A = I: C = B exactly
    np.testing.assert_array_equal(Cp, B.rowptr)
    np.testing.assert_array_equal(Ci, B.col)
    assert np.array_equal(Cx, B.val)
    A = random_csr(rng, n, n, 0.1, vals="normal")
    Cp, Ci, Cx, _ = oracle.spgemm(A, I)            # B = I (d = n): C = A exactly
    np.testing.assert_array_equal(Cp, A.rowptr)
    np.testing.assert_array_equal(Ci, A.col)
    assert np.array_equal(Cx, A.val)
    Z = CSR(n, n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    Cp, Ci, _, _ = oracle.spgemm(Z, B)             # A = 0
    assert Cp[-1] == 0 and np.all(Cp == 0) and Ci.size == 0
    Zb = CSR(n, d, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    Cp, Ci, _, _ = oracle.spgemm(A, Zb)            # B = 0
    assert np.all(Cp == 0) and Ci.size == 0


def test_invariants_rmat():
    A, B = synth.rmat_embedding(scale=10, edge_factor=16, d=64, density=0.2, seed=11)
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B)
    blen = np.diff(B.rowptr)
    flops = np.array([blen[A.col[A.rowptr[i]:A.rowptr[i + 1]]].sum() for i in range(A.nrows)])
    cnt = np.diff(Cp)
    assert np.all(cnt <= np.minimum(B.ncols, flops))
    assert np.all((cnt == 0) == (flops == 0))
    # row sums in FP64: sum_j C(i,j) = sum_k A(i,k) * rowsum(B_k)
    bsum = np.add.reduceat(B.val.astype(np.float64), B.rowptr[:-1]) * (blen > 0)
    lhs = np.add.reduceat(Cx, Cp[:-1]) * (cnt > 0) if Cx.size else np.zeros(A.nrows)
    rhs = np.array([np.dot(A.val[A.rowptr[i]:A.rowptr[i + 1]].astype(np.float64),
                           bsum[A.col[A.rowptr[i]:A.rowptr[i + 1]]]) for i in range(A.nrows)])
    scale = np.add.reduceat(Cb, Cp[:-1]) * (cnt > 0)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * np.maximum(scale, 1.0))
    # selected rows equal the same rows of the full product
    rows = np.array([5, 0, A.nrows - 1, 17, 17], dtype=np.int64)
    Sp, Si, Sx, _ = oracle.spgemm(A, B, rows=rows)
    for q, r in enumerate(rows):
        np.testing.assert_array_equal(Si[Sp[q]:Sp[q + 1]], Ci[Cp[r]:Cp[r + 1]])
        np.testing.assert_array_equal(Sx[Sp[q]:Sp[q + 1]], Cx[Cp[r]:Cp[r + 1]])


def queue_bfs(A, s):
    lev = np.full(A.nrows, -1, dtype=np.int64)
    lev[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for v in A.col[A.rowptr[u]:A.rowptr[u + 1]]:
            if lev[v] < 0:
                lev[v] = lev[u] + 1
                q.append(v)
    return lev


def undirected(n, edges):
    src = np.array([u for u, v in edges] + [v for u, v in edges], dtype=np.int64)
    dst = np.array([v for u, v in edges] + [u for u, v in edges], dtype=np.int64)
    M = sp.csr_matrix((np.ones(src.size), (src, dst)), shape=(n, n))
    M.sum_duplicates()
    M.sort_indices()
    return CSR(n, n, M.indptr.astype(np.int64), M.indices.astype(np.int32))


def test_msbfs_golden_alg3():
    g = json.load(open(os.path.join(GOLDEN, "alg3_small.json")))
    A = undirected(g["n"], g["edges_undirected"])
    levels, prods, fnnz = oracle.msbfs(A, np.array(g["sources"]))
    np.testing.assert_array_equal(levels, np.array(g["levels"]))
    assert prods == g["products"]
    assert fnnz[0] == len(g["sources"]) and fnnz[-1] == 0


@pytest.mark.parametrize("kind", ["rmat", "er", "chain"])
def test_msbfs_matches_queue_bfs(kind):
    if kind == "rmat":
        A = synth.rmat(9, 8, 21, symmetrize=True)
    elif kind == "er":
        A0 = synth.er(300, 2, 22)
        src, dst = np.repeat(np.arange(300), 2), A0.col
        A = undirected(300, list(zip(src.tolist(), dst.tolist())))
    else:
        A = undirected(40, [(i, i + 1) for i in range(39)])
    srcs = synth.sources(A, 24, 5)
    levels, prods, fnnz = oracle.msbfs(A, srcs)
    maxlev = -1
    for s_idx, s in enumerate(srcs):
        ref = queue_bfs(A, int(s))
        np.testing.assert_array_equal(levels[:, s_idx], ref)
        np.testing.assert_array_equal(oracle.bfs_levels(A, int(s)), ref)
        maxlev = max(maxlev, int(ref.max()))
    assert prods == maxlev + 1
    assert fnnz.sum() == int((levels >= 0).sum())


def test_msbfs_parents_golden():
    g = json.load(open(os.path.join(GOLDEN, "alg3_parents_small.json")))
    A = undirected(g["n"], g["edges_undirected"])
    levels, parents, prods, fnnz = oracle.msbfs_parents(A, np.array(g["sources"]))
    np.testing.assert_array_equal(levels, np.array(g["levels"]))
    np.testing.assert_array_equal(parents, np.array(g["parents"]))
    assert prods == g["products"]
    # the same graph's levels from the (or, select2nd) Alg. 3
    lv2, prods2, _ = oracle.msbfs(A, np.array(g["sources"]))
    np.testing.assert_array_equal(lv2, levels)
    assert prods2 == prods


def check_bfs_tree(A, srcs, levels, parents):
    """The BFS-tree definition, checked edge by edge without the oracle:
    a source is its own parent, an unreached vertex has -1, and any other
    vertex's parent is its smallest neighbour one level closer."""
    for si, s in enumerate(srcs):
        ref = queue_bfs(A, int(s))
        np.testing.assert_array_equal(levels[:, si], ref)
        for v in range(A.nrows):
            nb = A.col[A.rowptr[v]:A.rowptr[v + 1]]
            if ref[v] < 0:
                assert parents[v, si] == -1
            elif v == s:
                assert parents[v, si] == s
            else:
                closer = [int(u) for u in nb if ref[u] == ref[v] - 1]
                assert closer and parents[v, si] == min(closer), (v, si)


@pytest.mark.parametrize("kind", ["rmat", "er", "chain", "directed"])
def test_msbfs_parents_are_min_bfs_tree(kind):
    if kind == "rmat":
        A = synth.rmat(8, 8, 23, symmetrize=True)
    elif kind == "er":
        A0 = synth.er(200, 3, 24)
        A = undirected(200, list(zip(np.repeat(np.arange(200), 3).tolist(), A0.col.tolist())))
    elif kind == "chain":
        A = undirected(30, [(i, i + 1) for i in range(29)] + [(0, 29)])
    else:
        A = synth.rmat(7, 6, 25)  # directed: the pull follows A's rows (a BFS over A^T)
    srcs = synth.sources(A, 16, 6)
    levels, parents, prods, fnnz = oracle.msbfs_parents(A, srcs)
    if kind == "directed":
        lv2, _, _ = oracle.msbfs(A, srcs)
        np.testing.assert_array_equal(levels, lv2)
        # parent p of v: stored A(v, p), level one less, smallest such
        for si in range(len(srcs)):
            for v in range(A.nrows):
                if levels[v, si] > 0:
                    nb = A.col[A.rowptr[v]:A.rowptr[v + 1]]
                    closer = [int(u) for u in nb if levels[u, si] == levels[v, si] - 1]
                    assert parents[v, si] == min(closer)
    else:
        check_bfs_tree(A, srcs, levels, parents)
    assert prods == int(levels.max()) + 1
    assert fnnz.sum() == int((levels >= 0).sum())


def test_backward_matches_dense_formulas_and_finite_differences():
    rng = np.random.default_rng(5)
    n, d = 30, 12
    A = random_csr(rng, n, n, 0.15, full_rows=(3,), empty_rows=(7,), vals="normal")
    B = random_csr(rng, n, d, 0.35, empty_rows=(2,), vals="normal")
    Cp, Ci, Cx, _ = oracle.spgemm(A, B)
    dC = rng.standard_normal(Ci.size)
    dA, dAb, dB, dBb = oracle.backward(A, B, Cp, Ci, dC)
    G = dense(CSR(n, d, Cp, Ci, dC))
    dA_dense = G @ dense(B).T
    dB_dense = dense(A).T @ G
    for i in range(n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            assert abs(dA[e] - dA_dense[i, A.col[e]]) <= 1e-12 * max(1.0, dAb[e])
    for k in range(n):
        for f in range(B.rowptr[k], B.rowptr[k + 1]):
            assert abs(dB[f] - dB_dense[k, B.col[f]]) <= 1e-12 * max(1.0, dBb[f])

    def loss(Av, Bv):
        _, _, X, _ = oracle.spgemm(A.with_values(Av), B.with_values(Bv))
        return float(np.dot(dC, X))

    # L is linear in each of A.val and B.val separately, so the central
    # difference with h = 1 is the exact derivative (up to FP64 rounding)
    h = 1.0
    for e in rng.choice(A.nnz, size=min(40, A.nnz), replace=False):
        ap, am = A.val.copy(), A.val.copy()
        ap[e] += h
        am[e] -= h
        fd = (loss(ap, B.val) - loss(am, B.val)) / (2 * h)
        assert abs(fd - dA[e]) <= 1e-10 * max(1.0, dAb[e])
    for f in rng.choice(B.nnz, size=min(40, B.nnz), replace=False):
        bp, bm = B.val.copy(), B.val.copy()
        bp[f] += h
        bm[f] -= h
        fd = (loss(A.val, bp) - loss(A.val, bm)) / (2 * h)
        assert abs(fd - dB[f]) <= 1e-10 * max(1.0, dBb[f])


def test_backward_sampled_rows_match_full():
    A, B = synth.rmat_embedding(scale=9, edge_factor=8, d=32, density=0.25, seed=13)
    Cp, Ci, Cx, _ = oracle.spgemm(A, B)
    dC = synth.grad_output(Ci.size, 13).astype(np.float64)
    dA, _, dB, _ = oracle.backward(A, B, Cp, Ci, dC)
    rows = np.array([0, 3, 100, A.nrows - 1], dtype=np.int64)
    sA, _ = oracle.backward_dA_rows(A, B, Cp, Ci, dC, rows)
    ref = np.concatenate([dA[A.rowptr[r]:A.rowptr[r + 1]] for r in rows])
    np.testing.assert_allclose(sA, ref, rtol=1e-13, atol=1e-13)
    krows = np.array([1, 2, 50, B.nrows - 1], dtype=np.int64)
    sB, _ = oracle.backward_dB_rows(A, B, Cp, Ci, dC, krows)
    ref = np.concatenate([dB[B.rowptr[k]:B.rowptr[k + 1]] for k in krows])
    np.testing.assert_allclose(sB, ref, rtol=1e-12, atol=1e-12)


# --- sparse Force2Vec step (paper Sec. IV, sparse embedding) --------------

def _dense_rows(Z):
    D = np.zeros((Z.nrows, Z.ncols))
    for i in range(Z.nrows):
        D[i, Z.col[Z.rowptr[i]:Z.rowptr[i + 1]]] = Z.val[Z.rowptr[i]:Z.rowptr[i + 1]]
    return D


def test_f2v_topk_golden():
    g = json.load(open(os.path.join(GOLDEN, "f2v_topk_small.json")))
    U = np.array(g["U"], dtype=np.float64)
    cols, vals = oracle.f2v_topk(U, g["k"])
    np.testing.assert_array_equal(cols, np.array(g["cols"]))
    np.testing.assert_array_equal(vals, np.array(g["vals"], dtype=np.float64))


def test_f2v_topk_extremes():
    rng = np.random.default_rng(3)
    U = rng.normal(size=(5, 16))
    cols, vals = oracle.f2v_topk(U, 16)          # k = d keeps the whole row
    np.testing.assert_array_equal(cols, np.tile(np.arange(16), (5, 1)))
    np.testing.assert_array_equal(vals, U)
    cols, _ = oracle.f2v_topk(U, 1)              # k = 1: the argmax of |U|
    np.testing.assert_array_equal(cols[:, 0], np.argmax(np.abs(U), axis=1))


def test_f2v_zero_rate_is_identity():
    A = synth.rmat(8, 8, 41, symmetrize=True)
    Z = synth.sparse_embedding(A.nrows, 32, 6, 42)
    neg = synth.negatives(50, 4, A.nrows, 43)
    U, Ub, ncol, nval = oracle.f2v_step(A, Z, 10, 50, neg, 4, 0.0, 6)
    D = _dense_rows(Z)
    np.testing.assert_array_equal(U, D[10:60])
    # the k stored entries are nonzero, so they are exactly the k largest in magnitude
    np.testing.assert_array_equal(ncol, Z.col.reshape(-1, 6)[10:60])
    np.testing.assert_array_equal(nval, Z.val.reshape(-1, 6)[10:60].astype(np.float64))


def test_f2v_gradient_is_derivative_of_the_objective():
    # G_i = (U_i - z_i) / lr must be the gradient, with respect to z_i, of
    # L_i(z) = sum over neighbours j of log sigmoid(z . z_j)
    #        + sum over negatives q of log sigmoid(-z . z_q)
    # (the other endpoints held at their old values); central differences
    A = synth.rmat(8, 6, 44, symmetrize=True)
    n, d, k, s, lr = A.nrows, 24, 5, 3, 0.5
    Z = synth.sparse_embedding(n, d, k, 45, scale=0.7)
    r0, b = 20, 12
    neg = synth.negatives(b, s, n, 46)
    U, _, _, _ = oracle.f2v_step(A, Z, r0, b, neg, s, lr, k)
    D = _dense_rows(Z)
    logsig = lambda x: -np.log1p(np.exp(-x))
    for r in range(b):
        i = r0 + r
        nb = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        ng = neg[r * s:(r + 1) * s]

        def L(z):
            return sum(logsig(z @ D[j]) for j in nb) + sum(logsig(-(z @ D[q])) for q in ng)

        G = (U[r] - D[i]) / lr
        h = 1e-6
        for c in range(d):
            e = np.zeros(d)
            e[c] = h
            fd = (L(D[i] + e) - L(D[i] - e)) / (2 * h)
            assert abs(G[c] - fd) <= 1e-6 * (1 + abs(fd)), (r, c, G[c], fd)


def test_f2v_duplicate_negatives_and_self_terms():
    # a negative equal to a neighbour, or repeated, or the row itself, is one
    # more term of its own: compare with the per-term sum written with numpy
    A = synth.rmat(7, 4, 47, symmetrize=True)
    n, d, k, s, lr = A.nrows, 16, 4, 4, 0.3
    Z = synth.sparse_embedding(n, d, k, 48, scale=0.5)
    D = _dense_rows(Z)
    r0, b = 5, 6
    neg = synth.negatives(b, s, n, 49)
    for r in range(b):
        i = r0 + r
        nb = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        neg[r * s] = i
        if nb.size:
            neg[r * s + 1] = nb[0]
        neg[r * s + 2] = neg[r * s + 3]
    U, _, _, _ = oracle.f2v_step(A, Z, r0, b, neg, s, lr, k)
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    for r in range(b):
        i = r0 + r
        g = np.zeros(d)
        for j in A.col[A.rowptr[i]:A.rowptr[i + 1]]:
            g += (1 - sig(D[i] @ D[j])) * D[j]
        for q in neg[r * s:(r + 1) * s]:
            g -= sig(D[i] @ D[q]) * D[q]
        np.testing.assert_allclose(U[r], D[i] + lr * g, rtol=1e-12, atol=1e-13)
