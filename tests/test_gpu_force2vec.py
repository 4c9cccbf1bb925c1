"""GPU parity of the sparse Force2Vec step (paper Sec. IV, sparse embedding).

The dense update U = Z_batch + lr * (W * Z) must be within 1e-5 of the FP64
oracle's error scale per entry; the sparsified rows are an integer decision
(which columns survive), taken on the GPU's own FP32 U: they must equal the
oracle's top-k applied to that same U, bit for bit.  Rows outside the batch
must be untouched.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import CSR

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import DeviceCSR, TSError
from paper_2408_11988_gb300.force2vec import Force2Vec


def _host_Z(Zd, n, d):
    return CSR(n, d, Zd.rowptr.cpu().numpy(), Zd.col.cpu().numpy().copy(), Zd.val.cpu().numpy().copy())


def _check_step(A, Z, r0, b, s, lr, k, neg, batch=None):
    n, d = A.nrows, Z.ncols
    Ad = DeviceCSR.from_host(A, with_values=False)
    Zd = DeviceCSR.from_host(Z)
    f = Force2Vec(Ad, Zd, k, negatives=s, lr=lr, batch=batch or max(b, 1))
    U = f.step(r0, torch.as_tensor(neg), b=b, want_u=True)
    Uo, Ub, _, _ = oracle.f2v_step(A, Z, r0, b, neg, s, lr, k)
    Ug = U.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Ug - Uo) <= 1e-5 * Ub), np.max(np.abs(Ug - Uo) / np.maximum(Ub, 1e-30))
    ncol, nval = oracle.f2v_topk(Ug, k)
    Zn = _host_Z(Zd, n, d)
    zc, zv = Zn.col.reshape(n, k), Zn.val.reshape(n, k)
    np.testing.assert_array_equal(zc[r0:r0 + b], ncol)
    np.testing.assert_array_equal(zv[r0:r0 + b].astype(np.float64), nval)
    outside = np.r_[0:r0, r0 + b:n]
    np.testing.assert_array_equal(zc[outside], Z.col.reshape(n, k)[outside])
    np.testing.assert_array_equal(zv[outside], Z.val.reshape(n, k)[outside])
    return Zn


@pytest.mark.parametrize("d,k,s,lr", [(128, 26, 5, 0.02), (128, 26, 5, 0.5), (64, 8, 3, 0.3), (200, 40, 7, 0.1),
                                      (256, 51, 5, 0.05), (32, 32, 2, 0.2), (96, 1, 4, 1.0), (128, 26, 0, 0.5)])
def test_f2v_step_matches_oracle(d, k, s, lr):
    A = synth.rmat(10, 8, 100 + d, symmetrize=True)
    Z = synth.sparse_embedding(A.nrows, d, k, 101 + k, scale=0.3)
    r0, b = 37, 300
    neg = synth.negatives(b, s, A.nrows, 102)
    _check_step(A, Z, r0, b, s, lr, k, neg)


def test_f2v_batch_edges_and_repeated_negatives():
    A = synth.rmat(9, 12, 103, symmetrize=True)
    n, d, k, s = A.nrows, 128, 20, 6
    Z = synth.sparse_embedding(n, d, k, 104, scale=0.5)
    # last rows of Z, negatives repeating, equal to the row, equal to a neighbour
    b = 64
    r0 = n - b
    neg = synth.negatives(b, s, n, 105)
    for r in range(b):
        i = r0 + r
        neg[r * s] = i
        neg[r * s + 1] = neg[r * s + 2]
        nb = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        if nb.size:
            neg[r * s + 3] = nb[-1]
    _check_step(A, Z, r0, b, s, 0.25, k, neg)
    # an empty batch changes nothing
    Ad, Zd = DeviceCSR.from_host(A, with_values=False), DeviceCSR.from_host(Z)
    Force2Vec(Ad, Zd, k, negatives=s, batch=8).step(0, torch.zeros(0, dtype=torch.int32), b=0)
    np.testing.assert_array_equal(Zd.val.cpu().numpy(), Z.val)


def test_f2v_consecutive_steps():
    # three minibatches in a row, each checked against the oracle run on the
    # GPU's embedding before that step (the FP32 path is the state)
    A = synth.rmat(10, 10, 106, symmetrize=True)
    n, d, k, s = A.nrows, 128, 26, 5
    Z = synth.sparse_embedding(n, d, k, 107, scale=0.3)
    Ad, Zd = DeviceCSR.from_host(A, with_values=False), DeviceCSR.from_host(Z)
    f = Force2Vec(Ad, Zd, k, negatives=s, lr=0.3, batch=400)
    for step, r0 in enumerate((0, 400, 150)):
        cur = _host_Z(Zd, n, d)
        neg = synth.negatives(400, s, n, 108 + step)
        U = f.step(r0, torch.as_tensor(neg), want_u=True).cpu().numpy().astype(np.float64)
        Uo, Ub, _, _ = oracle.f2v_step(A, cur, r0, 400, neg, s, 0.3, k)
        assert np.all(np.abs(U - Uo) <= 1e-5 * Ub)
        ncol, nval = oracle.f2v_topk(U, k)
        zc = Zd.col.cpu().numpy().reshape(n, k)
        np.testing.assert_array_equal(zc[r0:r0 + 400], ncol)


def test_f2v_full_size_sampled():
    # the Force2Vec workload at full size: R-MAT scale 20, d = 128, k = 26,
    # five negatives, a 64K-row minibatch; 4 windows of 32 rows checked
    A, Z = synth.force2vec_inputs()
    n, d, k, s, b = A.nrows, 128, 26, 5, 65536
    Ad, Zd = DeviceCSR.from_host(A, with_values=False), DeviceCSR.from_host(Z)
    f = Force2Vec(Ad, Zd, k, negatives=s, lr=0.02, batch=b)
    r0 = 123456
    neg = synth.negatives(b, s, n, 109)
    U = f.step(r0, torch.as_tensor(neg), want_u=True).cpu().numpy().astype(np.float64)
    zc = Zd.col.cpu().numpy().reshape(n, k)
    for w0 in (0, 1000, 40000, b - 32):
        Uo, Ub, _, _ = oracle.f2v_step(A, Z, r0 + w0, 32, neg[w0 * s:(w0 + 32) * s], s, 0.02, k)
        assert np.all(np.abs(U[w0:w0 + 32] - Uo) <= 1e-5 * Ub)
        ncol, _ = oracle.f2v_topk(U[w0:w0 + 32], k)
        np.testing.assert_array_equal(zc[r0 + w0:r0 + w0 + 32], ncol)


def test_f2v_argument_errors():
    A = synth.rmat(8, 4, 110, symmetrize=True)
    Z = synth.sparse_embedding(A.nrows, 64, 8, 111)
    Ad, Zd = DeviceCSR.from_host(A, with_values=False), DeviceCSR.from_host(Z)
    f = Force2Vec(Ad, Zd, 8, negatives=2, batch=16)
    with pytest.raises(TSError):
        f.step(A.nrows - 4, torch.zeros(32, dtype=torch.int32))  # batch past the last row
    bad = DeviceCSR(Zd.nrows, Zd.ncols, Zd.rowptr, Zd.col[:-1], Zd.val[:-1])  # not k per row
    with pytest.raises(TSError):
        Force2Vec(Ad, bad, 8, negatives=2, batch=16).step(0, torch.zeros(32, dtype=torch.int32))
