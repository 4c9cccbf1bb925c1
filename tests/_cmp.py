"""Comparison helpers shared by the GPU parity tests (CUDA path vs oracle)."""
import numpy as np

import oracle

# FP32 tolerance of the plus-times product: |C_gpu - C_oracle| <= REL * sum |a_ik||b_kj|
# per entry (FP64 oracle; FP32 products and FP32 sums in any order).
REL = 1e-5


def assert_pattern_equal(rp, col, Cp, Ci, what="C"):
    assert rp.shape == Cp.shape, f"{what}: rowptr length {rp.shape} vs {Cp.shape}"
    bad = np.nonzero(rp != Cp)[0]
    assert bad.size == 0, f"{what}: rowptr differs first at {bad[:5]}: {rp[bad[:5]]} vs {Cp[bad[:5]]}"
    n = int(Cp[-1])
    assert col.shape[0] >= n
    badc = np.nonzero(col[:n] != Ci)[0]
    assert badc.size == 0, f"{what}: columns differ at {badc[:5]}"


def assert_values_close(val, Cx, Cb, rel=REL, what="C"):
    err = np.abs(val.astype(np.float64) - Cx)
    lim = rel * Cb
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, (f"{what}: {bad.size} values outside {rel}*bound, first {bad[:5]}: "
                           f"err {err[bad[:5]]} bound {Cb[bad[:5]]}")


def compare_full(Cdev, A, B, semiring=oracle.PLUS_TIMES):
    rp, col, val = Cdev.to_host()
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B, semiring=semiring)
    assert_pattern_equal(rp, col, Cp, Ci)
    if semiring == oracle.PLUS_TIMES:
        assert_values_close(val[: Cx.size], Cx, Cb)
    return Cp, Ci, Cx, Cb


def compare_rows(Cdev, A, B, rows, semiring=oracle.PLUS_TIMES):
    """Compare selected rows of a large GPU product with the oracle's rows."""
    rows = np.asarray(rows, dtype=np.int64)
    rp = Cdev.rowptr.cpu().numpy()
    Sp, Si, Sx, Sb = oracle.spgemm(A, B, semiring=semiring, rows=rows)
    col_all = Cdev.col
    val_all = Cdev.val
    import torch
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    cnt = np.array([rp[r + 1] - rp[r] for r in rows], dtype=np.int64)
    np.testing.assert_array_equal(cnt, np.diff(Sp), err_msg="row counts differ")
    it = torch.as_tensor(idx, device=col_all.device)
    col = col_all[it].cpu().numpy()
    np.testing.assert_array_equal(col, Si, err_msg="columns differ")
    if semiring == oracle.PLUS_TIMES:
        val = val_all[it].cpu().numpy()
        assert_values_close(val, Sx, Sb)
