"""The C-ABI library builds, loads and exports every symbol include/tsspgemm.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_11988_gb300.build import build
    from paper_2408_11988_gb300 import _native as N
    build()
    return N.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "tsspgemm.h")).read()
    return sorted(set(re.findall(r"^TS_API [^(]*?\b([A-Za-z_][A-Za-z0-9_]*)\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 28
    for n in names:
        assert hasattr(lib, n), n


def test_host_side_errors(lib):
    from paper_2408_11988_gb300 import _native as N
    A = N.CsrDesc(100, 100, 0, 8, None, None)      # fake non-NULL pointer, never dereferenced
    B = N.CsrDesc(100, 64, 0, 8, None, None)
    h = ctypes.c_void_p()
    assert lib.ts_plan_create(None, ctypes.byref(B), 0, None, ctypes.byref(h)) == N.TS_ERR_INVALID_ARG
    Abad = N.CsrDesc(100, 99, 0, 8, None, None)
    assert lib.ts_plan_create(ctypes.byref(Abad), ctypes.byref(B), 0, None, ctypes.byref(h)) == N.TS_ERR_INVALID_ARG
    assert "square" in N.last_error()
    assert lib.ts_plan_create(ctypes.byref(A), ctypes.byref(B), 7, None, ctypes.byref(h)) == N.TS_ERR_INVALID_ARG
    Bbig = N.CsrDesc(100, 1 << 21, 0, 8, None, None)
    assert lib.ts_plan_create(ctypes.byref(A), ctypes.byref(Bbig), 0, None, ctypes.byref(h)) == N.TS_ERR_UNSUPPORTED
    bad_t = N.Tuning(0, 48, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    assert lib.ts_plan_create(ctypes.byref(A), ctypes.byref(B), 0, ctypes.byref(bad_t), ctypes.byref(h)) == N.TS_ERR_INVALID_ARG
    for bad in ({"bwd_group": 3}, {"group": 64}, {"row_lanes": 2}, {"accum": 5}, {"accum": N.ACC_COPIES, "col_tile": 4096 + 32}):
        bt = N.Tuning.from_dict(bad)
        assert lib.ts_plan_create(ctypes.byref(A), ctypes.byref(B), 0, ctypes.byref(bt), ctypes.byref(h)) \
            == N.TS_ERR_INVALID_ARG, bad
    assert lib.ts_plan_create(ctypes.byref(A), ctypes.byref(B), 0, None, ctypes.byref(h)) == N.TS_OK
    t = N.Tuning()
    assert lib.ts_plan_get_tuning(h, ctypes.byref(t)) == N.TS_OK
    assert t.accum == N.ACC_DENSE and t.col_tile == 64 and t.warps_per_cta == 8
    assert t.group in (1, 2, 4, 8, 16, 32) and t.pack_b in (1, 2)
    assert t.sym_group in (1, 2, 4, 8, 16, 32) and t.bwd_group in (1, 2, 4, 8, 16, 32)
    assert t.row_lanes in (4, 8, 16, 32)
    sz = ctypes.c_size_t()
    assert lib.ts_workspace_size(h, ctypes.byref(sz)) == N.TS_OK and sz.value > 100 * 12
    # missing workspace and missing C row pointers are argument errors
    assert lib.ts_spgemm_symbolic(h, ctypes.byref(A), ctypes.byref(B), None, None, None, 0, None) == N.TS_ERR_INVALID_ARG
    rp = ctypes.c_void_p(256)
    assert lib.ts_spgemm_symbolic(h, ctypes.byref(A), ctypes.byref(B), rp, None, ctypes.c_void_p(256), 16, None) \
        == N.TS_ERR_WORKSPACE_TOO_SMALL
    # numeric before symbolic is a state error, found before any launch
    C = N.CsrDesc(100, 64, 0, 8, None, None)
    assert lib.ts_spgemm_numeric(h, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), ctypes.c_void_p(256),
                                 sz.value, None) == N.TS_ERR_STATE
    assert lib.ts_plan_destroy(h) == N.TS_OK
    assert lib.msbfs_workspace_size(10, 30, 0, ctypes.byref(sz)) == N.TS_ERR_INVALID_ARG
    assert lib.msbfs_workspace_size(10, 30, 128, ctypes.byref(sz)) == N.TS_OK
    # parents: the bitmap pull form only (d <= 256); caught on the host
    A2 = N.CsrDesc(10, 10, 0, 8, None, None)
    F2 = N.CsrDesc(10, 300, 0, 8, None, None)
    nn = ctypes.c_int64()
    assert lib.msbfs_step_parents(ctypes.byref(A2), ctypes.byref(F2), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                  ctypes.c_void_p(256), 1, ctypes.byref(F2), 0, ctypes.byref(nn),
                                  ctypes.c_void_p(256), 1 << 30, None) == N.TS_ERR_UNSUPPORTED
    assert lib.msbfs_step_parents(ctypes.byref(A2), ctypes.byref(F2), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                  None, 1, ctypes.byref(F2), 0, ctypes.byref(nn),
                                  ctypes.c_void_p(256), 1 << 30, None) == N.TS_ERR_INVALID_ARG
    assert lib.msbfs_init_parents(10, 300, ctypes.c_void_p(256), ctypes.c_void_p(256), None) == N.TS_ERR_UNSUPPORTED
    # Force2Vec limits, caught on the host
    sz2 = ctypes.c_size_t()
    assert lib.f2v_workspace_size(100, 64, 800, 10, 5, 8, ctypes.byref(sz2)) == N.TS_OK and sz2.value > 0
    assert lib.f2v_workspace_size(100, 64, 800, 10, 5, 65, ctypes.byref(sz2)) == N.TS_ERR_UNSUPPORTED  # k > d
    assert lib.f2v_workspace_size(100, 64, 800, 10, 33, 8, ctypes.byref(sz2)) == N.TS_ERR_UNSUPPORTED  # s > 32
    Zbad = N.CsrDesc(100, 64, 799, 8, 8, 8)  # not k = 8 entries per row
    Af = N.CsrDesc(100, 100, 0, 8, None, None)
    assert lib.f2v_step(ctypes.byref(Af), ctypes.byref(Zbad), 0, 10, ctypes.c_void_p(256), 5, ctypes.c_float(0.1), 8,
                        None, ctypes.c_void_p(256), sz2.value, None) == N.TS_ERR_INVALID_ARG
    assert N.status_string(N.TS_ERR_CAPACITY) == "TS_ERR_CAPACITY"
    assert lib.ts_version() >= 100


def test_automatic_accumulator_choice(lib):
    # plan creation only (no launch): the dense-B form above the measured
    # density crossovers (60 % for 64 < d <= 128, 45 % for d <= 256, never for
    # d <= 64), the wide shared accumulator for one tile of 256 < W <= 1024,
    # row groups up to 256 columns, hash above 4096; boolean products never
    # take the dense-B form
    from paper_2408_11988_gb300 import _native as N

    def tuning(n, d, nnzB, semiring=0, force=None):
        A = N.CsrDesc(n, n, 8 * n, 8, 8, 8)
        B = N.CsrDesc(n, d, nnzB, 8, 8, 8)
        h = ctypes.c_void_p()
        f = N.Tuning.from_dict(force) if force else None
        st = lib.ts_plan_create(ctypes.byref(A), ctypes.byref(B), semiring, ctypes.byref(f) if f else None,
                                ctypes.byref(h))
        if st != N.TS_OK:
            return st
        t = N.Tuning()
        assert lib.ts_plan_get_tuning(h, ctypes.byref(t)) == N.TS_OK
        assert lib.ts_plan_destroy(h) == N.TS_OK
        return t.as_dict()

    n = 1000
    assert tuning(n, 128, int(0.59 * n * 128))["accum"] == N.ACC_DENSE
    assert tuning(n, 128, int(0.60 * n * 128))["accum"] == N.ACC_DENSE_B
    assert tuning(n, 128, n * 128, semiring=1)["accum"] == N.ACC_DENSE
    assert tuning(n, 256, int(0.44 * n * 256))["accum"] == N.ACC_DENSE
    assert tuning(n, 256, int(0.45 * n * 256))["accum"] == N.ACC_DENSE_B
    assert tuning(n, 64, n * 64)["accum"] == N.ACC_DENSE
    assert tuning(n, 300, n * 300)["accum"] == N.ACC_DENSE
    assert tuning(n, 300, 10, force={"accum": N.ACC_DENSE_B}) == N.TS_ERR_INVALID_ARG
    t = tuning(n, 1024, 10 * n)
    assert t["accum"] == N.ACC_DENSE and t["col_tile"] == 1024 and t["row_lanes"] == 1
    t = tuning(n, 256, 13 * n)
    assert t["accum"] == N.ACC_DENSE and t["row_lanes"] == 8
    assert tuning(n, 5000, 10 * n)["accum"] == N.ACC_HASH
    assert tuning(n, 1024, 10 * n, force={"row_lanes": 1, "col_tile": 256}) == N.TS_ERR_INVALID_ARG
