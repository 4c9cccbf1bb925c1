"""GPU parity of the backward kernels and the autograd Function.

dA = SDDMM(dC, B^T) on A's pattern, dB = A^T dC on B's pattern.  The CUDA
gradients must be within 1e-5 * (sum of absolute terms) of the FP64 oracle
per entry, and within 1e-4 relative of FP64 central differences of
L = <dC, A*B> (exact for a bilinear L) wherever the gradient is not
dominated by cancellation.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _cmp import REL

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import ACC_HASH, DeviceCSR, Plan
from paper_2408_11988_gb300.autograd import ts_spgemm


def dev(M):
    return DeviceCSR.from_host(M)


def _run(A, B, tuning=None, seed=1):
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning=tuning)
    C = plan.forward(Ad, Bd)
    dC = synth.grad_output(C.nnz, seed)
    dA, dB = plan.backward(Ad, Bd, C, torch.as_tensor(dC, device="cuda"))
    rp, col, _ = C.to_host()
    return rp, col, dC, dA.cpu().numpy(), dB.cpu().numpy()


@pytest.mark.parametrize("tuning", [None, {"cta_min_flops": 1}, {"cta_min_flops": 128, "warps_per_cta": 4},
                                    {"warps_per_cta": 1}, {"group": 1}, {"group": 4}, {"group": 32},
                                    {"pack_b": 1}, {"pack_b": 1, "group": 1, "cta_min_flops": 64},
                                    {"bwd_group": 1}, {"bwd_group": 4}, {"bwd_group": 32, "sym_group": 1},
                                    {"bwd_group": 16}, {"bwd_group": 2}, {"bwd_group": 2, "pack_b": 2},
                                    {"bwd_group": 2, "cta_min_flops": 1}, {"bwd_group": 2, "warps_per_cta": 1},
                                    {"row_lanes": 32}, {"row_lanes": 8, "pack_b": 2}, {"row_lanes": 8, "warps_per_cta": 3}])
def test_backward_matches_oracle(tuning):
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=256, density=0.05, seed=50)
    rp, col, dC, dA, dB = _run(A, B, tuning)
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.astype(np.float64))
    assert np.all(np.abs(dA - rA) <= REL * bA), np.max(np.abs(dA - rA) / np.maximum(bA, 1e-30))
    assert np.all(np.abs(dB - rB) <= REL * bB), np.max(np.abs(dB - rB) / np.maximum(bB, 1e-30))


@pytest.mark.parametrize("tuning", [None, {"group": 1}, {"group": 8, "pack_b": 1}, {"bwd_group": 16},
                                    {"bwd_group": 2, "cta_min_flops": 16}, {"row_lanes": 32},
                                    {"row_lanes": 8, "cta_min_flops": 1 << 20}])
def test_backward_ragged_and_empty_rows(tuning):
    A, B = synth.er_product(n=3000, k=5, d=100, density=0.05, seed=51)
    rp, col, dC, dA, dB = _run(A, B, tuning)
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.astype(np.float64))
    assert np.all(np.abs(dA - rA) <= REL * bA)
    assert np.all(np.abs(dB - rB) <= REL * bB)


def test_backward_unaligned_db_and_b_tail():
    # dB one float into a buffer (not 16-byte aligned: the quad kernel must
    # not be used), and B whose last row ends at an entry count that is not a
    # multiple of four (the quads at the end of B take the scalar atomics)
    for seed in range(54, 70):
        A, B = synth.er_product(n=2001, k=5, d=96, density=0.07, seed=seed)
        if B.nnz % 4:
            break
    assert B.nnz % 4 != 0
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning={"bwd_group": 2, "row_lanes": 8})
    C = plan.forward(Ad, Bd)
    dC = synth.grad_output(C.nnz, 5)
    rp, col, _ = C.to_host()
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.astype(np.float64))
    g = torch.as_tensor(dC, device="cuda")
    for off in (0, 1):
        buf = torch.full((B.nnz + 4,), 7.0, device="cuda")
        dA, dB = plan.backward(Ad, Bd, C, g, out_dB=buf[off:off + B.nnz])
        assert np.all(np.abs(dA.cpu().numpy() - rA) <= REL * bA)
        assert np.all(np.abs(dB.cpu().numpy() - rB) <= REL * bB)
        rest = torch.cat([buf[:off], buf[off + B.nnz:]]).cpu().numpy()
        assert np.all(rest == 7.0)  # nothing written outside dB


@pytest.mark.parametrize("tuning", [None, {"dB_mode": 2}])
def test_backward_finite_differences(tuning):
    A, B = synth.rmat_embedding(scale=9, edge_factor=8, d=64, density=0.1, seed=52)
    rp, col, dC, dA, dB = _run(A, B, tuning=tuning, seed=3)
    dC64 = dC.astype(np.float64)
    Cp, Ci, Cx, _ = oracle.spgemm(A, B)

    def loss(Av, Bv):
        _, _, X, _ = oracle.spgemm(A.with_values(Av), B.with_values(Bv))
        return float(np.dot(dC64, X))

    rng = np.random.default_rng(0)
    _, bA, _, bB = oracle.backward(A, B, rp, col, dC64)
    Av, Bv = A.val.astype(np.float64), B.val.astype(np.float64)
    checked = 0
    for e in rng.choice(A.nnz, 128, replace=False):
        p, m = Av.copy(), Av.copy()
        p[e] += 1.0
        m[e] -= 1.0
        fd = (loss(p, Bv) - loss(m, Bv)) / 2.0
        assert abs(dA[e] - fd) <= REL * bA[e] + 1e-12
        if abs(fd) >= 1e-2 * bA[e]:
            assert abs(dA[e] - fd) <= 1e-4 * abs(fd)
            checked += 1
    for f in rng.choice(B.nnz, 128, replace=False):
        p, m = Bv.copy(), Bv.copy()
        p[f] += 1.0
        m[f] -= 1.0
        fd = (loss(Av, p) - loss(Av, m)) / 2.0
        assert abs(dB[f] - fd) <= REL * bB[f] + 1e-12
        if abs(fd) >= 1e-2 * bB[f]:
            assert abs(dB[f] - fd) <= 1e-4 * abs(fd)
            checked += 1
    assert checked > 100


def test_autograd_function():
    A, B = synth.rmat_embedding(scale=11, edge_factor=16, d=128, density=0.1, seed=53)
    Ad, Bd = dev(A), dev(B)
    a = Ad.val.clone().requires_grad_(True)
    b = Bd.val.clone().requires_grad_(True)
    C = ts_spgemm(Ad, Bd, a, b)
    g = torch.as_tensor(synth.grad_output(C.nnz, 9), device="cuda")
    (C.val * g).sum().backward()
    rp, col, _ = C.to_host()
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, g.double().cpu().numpy())
    assert np.all(np.abs(a.grad.cpu().numpy() - rA) <= REL * bA)
    assert np.all(np.abs(b.grad.cpu().numpy() - rB) <= REL * bB)


@pytest.mark.parametrize("tuning", [None, {"dB_mode": 2}])
def test_backward_full_size_sampled(tuning):
    # sparse-embedding workload at full size (R-MAT scale 22, d = 256, 5 %),
    # dB by float atomics and by the deterministic transpose pull
    A, B = synth.rmat_embedding()
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning=tuning)
    C = plan.forward(Ad, Bd)
    dC = synth.grad_output(C.nnz, 11)
    dA, dB = plan.backward(Ad, Bd, C, torch.as_tensor(dC, device="cuda"))
    rp, col, _ = C.to_host()
    rng = np.random.default_rng(1)
    deg = np.diff(A.rowptr)
    rows = np.concatenate([np.argsort(deg)[-4:], rng.choice(A.nrows, 2000, replace=False)])
    sA, bA = oracle.backward_dA_rows(A, B, rp, col, dC.astype(np.float64), rows)
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
    gA = dA.cpu().numpy()[idx]
    assert np.all(np.abs(gA - sA) <= REL * bA)
    indeg = np.bincount(A.col, minlength=A.nrows)
    krows = np.unique(np.concatenate([np.argsort(indeg)[-4:], rng.choice(B.nrows, 2000, replace=False)]))
    sB, bB = oracle.backward_dB_rows(A, B, rp, col, dC.astype(np.float64), krows)
    idx = np.concatenate([np.arange(B.rowptr[k], B.rowptr[k + 1]) for k in krows])
    gB = dB.cpu().numpy()[idx]
    assert np.all(np.abs(gB - sB) <= REL * bB)


def test_backward_split_rows():
    n, d = 4000, 256
    rng = np.random.default_rng(80)
    rows = [np.arange(n), rng.choice(n, 2500, replace=False)]
    rows += [rng.choice(n, size=int(rng.integers(0, 10)), replace=False) for _ in range(n - 2)]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.sort(r) for r in rows]).astype(np.int32)
    from synth import CSR
    A = CSR(n, n, rowptr, col, synth.uniform(col.size, 81))
    B = synth.tall_skinny(n, d, 0.05, 82)
    B.val = synth.normal(B.nnz, 83)
    for t in (None, {"group": 1}, {"pack_b": 1}, {"row_lanes": 32}):
        rp, ci, dC, dA, dB = _run(A, B, t, seed=4)
        rA, bA, rB, bB = oracle.backward(A, B, rp, ci, dC.astype(np.float64))
        assert np.all(np.abs(dA - rA) <= REL * bA)
        assert np.all(np.abs(dB - rB) <= REL * bB)


@pytest.mark.parametrize("d", [1024, 700, 288])
@pytest.mark.parametrize("tuning", [None, {"cta_min_flops": 1 << 20}, {"cta_min_flops": 64, "warps_per_cta": 4},
                                    {"bwd_group": 16}, {"row_lanes": 32}])
def test_backward_wide_rows(d, tuning):
    # products of one column tile of 256 < W <= 1024 (the wide numeric
    # kernel's range), their backward under several tunings
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=d, density=0.01, seed=57 + d % 5, b_values="uniform")
    rp, col, dC, dA, dB = _run(A, B, tuning)
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.astype(np.float64))
    assert np.all(np.abs(dA - rA) <= REL * bA)
    assert np.all(np.abs(dB - rB) <= REL * bB)


def test_backward_wide_rows_long_b_rows_and_hub():
    # rows of B of about 30 entries and a hub row of A split into parts
    rng = np.random.default_rng(58)
    n, d = 3000, 512
    A = synth.er(n, 6, 59)
    A.val = synth.uniform(A.nnz, 60)
    hub = np.sort(rng.choice(n, 2500, replace=False)).astype(np.int32)
    rows = [A.col[A.rowptr[i]:A.rowptr[i + 1]] if i != 5 else hub for i in range(n)]
    vals = [A.val[A.rowptr[i]:A.rowptr[i + 1]] if i != 5 else rng.random(hub.size, dtype=np.float32) for i in range(n)]
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    from synth import CSR
    A2 = CSR(n, n, rp, np.concatenate(rows), np.concatenate(vals))
    B = synth.tall_skinny(n, d, 0.06, 61)
    B.val = synth.normal(B.nnz, 62)
    rp, col, dC, dA, dB = _run(A2, B)
    rA, bA, rB, bB = oracle.backward(A2, B, rp, col, dC.astype(np.float64))
    assert np.all(np.abs(dA - rA) <= REL * bA)
    assert np.all(np.abs(dB - rB) <= REL * bB)


@pytest.mark.parametrize("case", ["rmat256", "rmat1024", "er64", "hub"])
def test_backward_deterministic_db(case):
    # option T: dB without float atomics, identical bit for bit on repeated
    # calls, and within the bound of the FP64 oracle like option S
    if case == "rmat256":
        A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=256, density=0.05, seed=70)
    elif case == "rmat1024":
        A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=1024, density=0.01, seed=71, b_values="uniform")
    elif case == "er64":
        A, B = synth.er_product(n=3000, k=5, d=64, density=0.1, seed=72)
    else:  # a column of A with thousands of entries (several chunks of the pull) and empty rows of B
        n = 5000
        rng = np.random.default_rng(73)
        rows = [np.unique(np.concatenate([[7], rng.choice(n, 4, replace=False)])) for _ in range(n)]
        rowptr = np.zeros(n + 1, dtype=np.int64)
        rowptr[1:] = np.cumsum([len(r) for r in rows])
        from synth import CSR
        A = CSR(n, n, rowptr, np.concatenate(rows).astype(np.int32), synth.uniform(int(rowptr[-1]), 74))
        B = synth.tall_skinny(n, 128, 0.05, 75)
        B.val = synth.normal(B.nnz, 76)
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning={"dB_mode": 2})
    C = plan.forward(Ad, Bd)
    dC = torch.as_tensor(synth.grad_output(C.nnz, 77), device="cuda")
    dA1, dB1 = plan.backward(Ad, Bd, C, dC)
    dA2, dB2 = plan.backward(Ad, Bd, C, dC)
    plan.check()
    assert torch.equal(dB1, dB2)
    rp, col, _ = C.to_host()
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.double().cpu().numpy())
    assert np.all(np.abs(dA1.cpu().numpy() - rA) <= REL * bA)
    assert np.all(np.abs(dB1.cpu().numpy() - rB) <= REL * bB)
    # option S on the same product agrees within the bound
    plan_s = Plan(Ad, Bd, tuning={"dB_mode": 1})
    Cs = plan_s.forward(Ad, Bd)
    _, dBs = plan_s.backward(Ad, Bd, Cs, dC)
    assert np.all(np.abs(dBs.cpu().numpy() - rB) <= REL * bB)


def _tiny_rows_case(n=4000, d=700, seed=77):
    # rows of A with 1-3 entries (and some longer ones) whose rows of B draw
    # their columns from a few narrow windows, so that the products of a row
    # share columns often: the duplicate handling of the tiny-row kernels
    # (merge, sort, runs of equal columns) in every pass
    rng = np.random.default_rng(seed)
    windows = np.array([0, 6, 350, d - 16])
    brow = []
    for k in range(n):
        w = windows[rng.integers(0, len(windows))]
        cols = np.sort(rng.choice(16, size=int(rng.integers(1, 12)), replace=False)) + w
        brow.append(cols)
    Bp = np.zeros(n + 1, np.int64)
    Bp[1:] = np.cumsum([len(c) for c in brow])
    Bc = np.concatenate(brow).astype(np.int32)
    Bv = rng.uniform(-1.0, 1.0, size=Bc.size).astype(np.float32)
    arow = []
    for i in range(n):
        r = rng.random()
        na = 0 if r < 0.1 else (1 if r < 0.45 else (2 if r < 0.7 else (3 if r < 0.9 else int(rng.integers(4, 40)))))
        arow.append(np.sort(rng.choice(n, size=na, replace=False)))
    Ap = np.zeros(n + 1, np.int64)
    Ap[1:] = np.cumsum([len(c) for c in arow])
    Ac = np.concatenate(arow).astype(np.int32)
    Av = rng.uniform(0.0, 1.0, size=Ac.size).astype(np.float32)
    return synth.CSR(n, n, Ap, Ac, Av), synth.CSR(n, d, Bp, Bc, Bv)


@pytest.mark.parametrize("d", [700, 1024])
def test_tiny_rows_with_shared_columns(d):
    from _cmp import compare_full
    from paper_2408_11988_gb300 import spgemm
    A, B = _tiny_rows_case(d=d)
    compare_full(spgemm(dev(A), dev(B)), A, B)
    rp, col, dC, dA, dB = _run(A, B)
    rA, bA, rB, bB = oracle.backward(A, B, rp, col, dC.astype(np.float64))
    assert np.all(np.abs(dA - rA) <= REL * bA), np.max(np.abs(dA - rA) / np.maximum(bA, 1e-30))
    assert np.all(np.abs(dB - rB) <= REL * bB), np.max(np.abs(dB - rB) / np.maximum(bB, 1e-30))
