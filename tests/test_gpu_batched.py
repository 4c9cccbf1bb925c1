"""GPU parity of the batched product (one launch per phase over all
instances, graph capturable) against the oracle, instance by instance."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _cmp import REL, assert_pattern_equal, assert_values_close

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import OR_SELECT2ND, PLUS_TIMES, DeviceCSR
from paper_2408_11988_gb300.batched import BatchedProduct


def _instances(seed=3, count=7):
    out = []
    rng = np.random.default_rng(seed)
    for b in range(count):
        d = int(rng.choice([32, 64, 100, 256]))
        if b % 3 == 0:
            A, B = synth.er_product(n=int(rng.integers(50, 3000)), k=int(rng.integers(1, 9)), d=d,
                                    density=float(rng.uniform(0.02, 0.5)), seed=seed * 100 + b)
        else:
            A, B = synth.rmat_embedding(scale=int(rng.integers(6, 12)), edge_factor=int(rng.integers(4, 20)), d=d,
                                        density=float(rng.uniform(0.01, 0.3)), seed=seed * 100 + b,
                                        b_values="uniform")
        out.append((A, B))
    return out


def _check(C, A, B, semiring=oracle.PLUS_TIMES):
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B, semiring=semiring)
    rp = C.rowptr.cpu().numpy()
    nnz = int(rp[-1])
    col = C.col[:nnz].cpu().numpy()
    assert_pattern_equal(rp, col, Cp, Ci)
    if semiring == oracle.PLUS_TIMES:
        assert_values_close(C.val[:nnz].cpu().numpy(), Cx, Cb)
    return Cp, Ci


@pytest.mark.parametrize("tuning", [None, {"cta_min_flops": 64}, {"stage": 2, "group": 32}])
def test_batched_forward_backward_and_graph(tuning):
    inst = _instances()
    As = [DeviceCSR.from_host(A) for A, _ in inst]
    Bs = [DeviceCSR.from_host(B) for _, B in inst]
    bp = BatchedProduct(As, Bs, tuning=tuning)
    Cs = bp.forward()
    bp.check()
    pats = []
    for (A, B), C, cap in zip(inst, Cs, bp.capacity):
        Cp, Ci = _check(C, A, B)
        assert Cp[-1] <= cap                      # the bound holds
        pats.append((Cp, Ci))
    dCs = [torch.as_tensor(synth.grad_output(int(Cp[-1]), 5 + i), device="cuda") for i, (Cp, _) in enumerate(pats)]
    bp.bind_grads(dCs)
    dAs, dBs = bp.backward()
    bp.check()
    for i, ((A, B), (Cp, Ci)) in enumerate(zip(inst, pats)):
        rA, bA, rB, bB = oracle.backward(A, B, Cp, Ci, dCs[i].double().cpu().numpy())
        assert np.all(np.abs(dAs[i][:A.nnz].cpu().numpy() - rA) <= REL * bA)
        assert np.all(np.abs(dBs[i][:B.nnz].cpu().numpy() - rB) <= REL * bB)
    # capture forward + backward in a CUDA graph; change B's values in place and replay
    g = bp.capture(backward=True)
    for (A, B), Bd in zip(inst, Bs):
        Bd.val.mul_(2.0)
        B.val = B.val * 2.0
    g.replay()
    torch.cuda.synchronize()
    bp.check()
    for i, ((A, B), C) in enumerate(zip(inst, Cs)):
        Cp, Ci = _check(C, A, B)
        rA, bA, rB, bB = oracle.backward(A, B, Cp, Ci, dCs[i].double().cpu().numpy())
        assert np.all(np.abs(dAs[i][:A.nnz].cpu().numpy() - rA) <= REL * bA)


def test_batched_boolean():
    inst = _instances(seed=4, count=5)
    As = [DeviceCSR.from_host(A, with_values=False) for A, _ in inst]
    Bs = [DeviceCSR.from_host(B, with_values=False) for _, B in inst]
    bp = BatchedProduct(As, Bs, semiring=OR_SELECT2ND)
    Cs = bp.forward()
    bp.check()
    for (A, B), C in zip(inst, Cs):
        _check(C, A, B, semiring=oracle.OR_SELECT2ND)


def test_batched_full_size_sampled():
    # the uneven batch at its full size: 64 instances, n in [2^12, 2^18]
    inst = synth.batched_instances()
    As = [DeviceCSR.from_host(A) for A, _ in inst]
    Bs = [DeviceCSR.from_host(B) for _, B in inst]
    bp = BatchedProduct(As, Bs)
    g = bp.capture()
    g.replay()
    torch.cuda.synchronize()
    bp.check()
    # C's row pointers of every instance against the oracle's count pass
    for b, (A, B) in enumerate(inst):
        np.testing.assert_array_equal(bp.Cs[b].rowptr.cpu().numpy(), oracle.spgemm_count(A, B),
                                      err_msg=f"instance {b}")
    rng = np.random.default_rng(2)
    for b in rng.choice(len(inst), 6, replace=False):
        A, B = inst[b]
        C = bp.Cs[b]
        rows = rng.choice(A.nrows, min(300, A.nrows), replace=False)
        Sp, Si, Sx, Sb = oracle.spgemm(A, B, rows=rows)
        rp = C.rowptr.cpu().numpy()
        cnt = np.array([rp[r + 1] - rp[r] for r in rows])
        np.testing.assert_array_equal(cnt, np.diff(Sp))
        idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
        it = torch.as_tensor(idx, device="cuda")
        np.testing.assert_array_equal(C.col[it].cpu().numpy(), Si)
        assert_values_close(C.val[it].cpu().numpy(), Sx, Sb)


def _mixed_instances(seed=5):
    # uneven instances, two of them with dense B (the dense-B form applies)
    out = _instances(seed=seed, count=6)
    A, B = synth.rmat_embedding(scale=10, edge_factor=12, d=128, density=0.7, seed=seed * 10 + 1,
                                b_values="uniform")
    out.append((A, B))
    A, B = synth.rmat_embedding(scale=9, edge_factor=20, d=256, density=0.6, seed=seed * 10 + 2,
                                b_values="uniform")
    out.append((A, B))
    return out


@pytest.mark.parametrize("tuning", [None, {"accum": 4}, {"accum": 1, "cta_min_flops": 32}])
def test_batched_per_instance_tuning_and_autotune(tuning):
    inst = _mixed_instances()
    As = [DeviceCSR.from_host(A) for A, _ in inst]
    Bs = [DeviceCSR.from_host(B) for _, B in inst]
    bp = BatchedProduct(As, Bs, tuning=tuning)
    summary = bp.tuning_summary()
    assert len(summary["per_instance"]) == len(inst)
    if tuning is None:   # the two dense instances take the dense-B form by default
        assert [x["accum"] for x in summary["per_instance"]][-2:] == ["dense_b", "dense_b"]
    Cs = bp.forward()
    bp.check()
    for (A, B), C in zip(inst, Cs):
        _check(C, A, B)
    bp.autotune(reps=1)
    after = bp.tuning_summary()["per_instance"]
    # each threshold is a candidate, or the one the autotuner started from
    # (kept when the whole batch runs fastest under it)
    start = (tuning or {}).get("cta_min_flops", 4096)
    assert all(x["heavy_min_flops"] in (1024, 4096, 16384, 1 << 50, start) for x in after)
    Cs = bp.forward()
    bp.check()
    for (A, B), C in zip(inst, Cs):
        _check(C, A, B)
    dCs = [torch.as_tensor(synth.grad_output(int(C.rowptr[-1].item()), 30 + i), device="cuda")
           for i, C in enumerate(Cs)]
    bp.bind_grads(dCs)
    dAs, dBs = bp.backward()
    bp.check()
    for i, ((A, B), C) in enumerate(zip(inst, Cs)):
        Cp, Ci = _check(C, A, B)
        rA, bA, rB, bB = oracle.backward(A, B, Cp, Ci, dCs[i].double().cpu().numpy())
        assert np.all(np.abs(dAs[i][:A.nnz].cpu().numpy() - rA) <= REL * bA)
        assert np.all(np.abs(dBs[i][:B.nnz].cpu().numpy() - rB) <= REL * bB)
