"""ts_spgemm_forward_noalloc: the forward product for callers that cannot
allocate device memory when they need it (a fixed memory budget owned by
another framework, serving loops that must not call cudaMalloc because it can
synchronise the device).  It takes its scratch from an array built into the
library; the test checks it against the allocating entry points
(ts_spgemm_symbolic + ts_spgemm_numeric with a caller workspace) on two calls
in a row, and that products too large for the built-in scratch are refused.

This file is collected last so that a failure here does not hide others.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from _cmp import REL

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import DeviceCSR, Plan
from paper_2408_11988_gb300 import _native as N


def _noalloc(plan, Ad, Bd, capacity):
    n = Ad.nrows
    rowptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(capacity, dtype=torch.int32, device="cuda")
    val = torch.empty(capacity, dtype=torch.float32, device="cuda")
    C = DeviceCSR(n, Bd.ncols, rowptr, col, val)
    da, db, dc = Ad.desc(), Bd.desc(), C.desc()
    nnz = ctypes.c_int64(-1)
    st = N.lib().ts_spgemm_forward_noalloc(plan.handle, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc),
                                           ctypes.byref(nnz), torch.cuda.current_stream().cuda_stream)
    return st, int(nnz.value), C


@pytest.mark.parametrize("case", ["er16k", "rmat13"])
def test_noalloc_matches_workspace_entry_points(case):
    if case == "er16k":
        A, B = synth.er_product(n=16384, k=8, d=64, density=0.10)
    else:
        A, B = synth.rmat_embedding(scale=13, edge_factor=16, d=256, density=0.05, seed=90)
    Ad, Bd = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    plan = Plan(Ad, Bd)
    ref = plan.forward(Ad, Bd)          # allocating path: caller workspace
    rp_ref, col_ref, val_ref = ref.to_host()
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B)
    for _ in range(2):                  # two calls in a row share the built-in scratch
        st, nnz, C = _noalloc(plan, Ad, Bd, capacity=ref.nnz)
        assert st == N.TS_OK, N.last_error()
        assert nnz == ref.nnz
        rp, col, val = C.to_host()
        np.testing.assert_array_equal(rp, rp_ref)
        np.testing.assert_array_equal(col, col_ref)
        assert np.all(np.abs(val.astype(np.float64) - val_ref) <= 2 * REL * Cb)
        assert np.all(np.abs(val.astype(np.float64) - Cx) <= REL * Cb)


def test_noalloc_reports_capacity_and_size_limits():
    A, B = synth.er_product(n=4096, k=8, d=64, density=0.10, seed=91)
    Ad, Bd = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    plan = Plan(Ad, Bd)
    st, nnz, _ = _noalloc(plan, Ad, Bd, capacity=10)
    assert st == N.TS_ERR_CAPACITY and nnz > 10
    st, nnz2, C = _noalloc(plan, Ad, Bd, capacity=nnz)
    assert st == N.TS_OK and nnz2 == nnz
    # a product whose workspace exceeds the built-in scratch is refused up front
    big_n = 1 << 24
    Ab = N.CsrDesc(big_n, big_n, 1 << 28, 256, 256, 256)
    Bb = N.CsrDesc(big_n, 256, 1 << 28, 256, 256, 256)
    h = ctypes.c_void_p()
    assert N.lib().ts_plan_create(ctypes.byref(Ab), ctypes.byref(Bb), 0, None, ctypes.byref(h)) == N.TS_OK
    Cb = N.CsrDesc(big_n, 256, 0, 256, None, None)
    out = ctypes.c_int64(0)
    st = N.lib().ts_spgemm_forward_noalloc(h, ctypes.byref(Ab), ctypes.byref(Bb), ctypes.byref(Cb),
                                           ctypes.byref(out), None)
    assert st == N.TS_ERR_UNSUPPORTED and "scratch" in N.last_error()
    N.lib().ts_plan_destroy(h)
    assert int(N.lib().ts_noalloc_scratch_bytes()) == 32 << 20


def test_noalloc_size_check_counts_only_the_forward_layout():
    """A product whose autotuner-covering workspace (ts_workspace_size) is
    larger than the built-in scratch while the forward passes' own layout fits
    must still run: the size check counts the forward layout only."""
    A, B = synth.er_product(n=86016, k=8, d=256, density=0.05, seed=92)
    Ad, Bd = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    plan = Plan(Ad, Bd)
    cover = ctypes.c_size_t(0)
    assert N.lib().ts_workspace_size(plan.handle, ctypes.byref(cover)) == N.TS_OK
    assert cover.value > int(N.lib().ts_noalloc_scratch_bytes())
    ref = plan.forward(Ad, Bd)
    rp_ref, col_ref, val_ref = ref.to_host()
    st, nnz, C = _noalloc(plan, Ad, Bd, capacity=ref.nnz)
    assert st == N.TS_OK, N.last_error()
    assert nnz == ref.nnz
    rp, col, val = C.to_host()
    np.testing.assert_array_equal(rp, rp_ref)
    np.testing.assert_array_equal(col, col_ref)
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B)
    assert np.all(np.abs(val.astype(np.float64) - Cx) <= REL * Cb)
