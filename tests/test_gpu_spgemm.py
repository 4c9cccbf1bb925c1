"""GPU parity: the CUDA product (through the C ABI) against the FP64 oracle.

Patterns and boolean results must be bit-exact; plus-times values must be
within 1e-5 * sum |a_ik||b_kj| of the FP64 oracle per entry.  Every accumulator,
tile width, row-bin threshold and block size is forced at least once.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import CSR
from _cmp import REL, compare_full, compare_rows, assert_pattern_equal, assert_values_close

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import (ACC_COPIES, ACC_DENSE, ACC_DENSE_B, ACC_HASH, OR_SELECT2ND, PLUS_TIMES, DeviceCSR, Plan,
                                    TSError, spgemm, validate)


def dev(M):
    return DeviceCSR.from_host(M)


TUNINGS = [
    None,
    {"col_tile": 32},                         # two column tiles of B (d = 64)
    {"cta_min_flops": 1},                      # every row CTA-per-row
    {"cta_min_flops": 64},
    {"warps_per_cta": 1},
    {"warps_per_cta": 8, "cta_min_flops": 16},
    {"stage": 2},                              # direct gathers (no cp.async staging)
    {"sym_group": 1}, {"sym_group": 32}, {"sym_group": 4, "group": 8},
    {"stage": 2, "group": 1},                  # flattened products
    {"stage": 2, "group": 4}, {"stage": 2, "group": 16}, {"stage": 2, "group": 32, "cta_min_flops": 32},
    {"stage": 2, "pack_b": 1}, {"stage": 2, "pack_b": 1, "group": 1, "col_tile": 32},
    {"stage": 2, "pack_b": 1, "cta_min_flops": 1}, {"col_tile": 32, "cta_min_flops": 1},
    {"accum": ACC_HASH, "hash_slots": 128},
    {"accum": ACC_HASH, "hash_slots": 1024, "warps_per_cta": 4},
    {"accum": ACC_COPIES},                     # private accumulator copies, no atomics
    {"accum": ACC_COPIES, "group": 16}, {"accum": ACC_COPIES, "group": 32, "cta_min_flops": 1},
    {"accum": ACC_COPIES, "col_tile": 32}, {"accum": ACC_COPIES, "pack_b": 2, "warps_per_cta": 1},
    {"accum": ACC_COPIES, "group": 8, "cta_min_flops": 16, "warps_per_cta": 3},
    {"group": 2}, {"sym_group": 2}, {"group": 2, "sym_group": 2, "cta_min_flops": 1},   # quads
    {"group": 2, "pack_b": 2}, {"group": 2, "col_tile": 32}, {"sym_group": 2, "warps_per_cta": 1},
    {"row_lanes": 4}, {"row_lanes": 8}, {"row_lanes": 16}, {"row_lanes": 4, "col_tile": 32},   # row groups
    {"row_lanes": 4, "pack_b": 2}, {"row_lanes": 8, "cta_min_flops": 1 << 20, "warps_per_cta": 2},
    {"row_lanes": 32}, {"row_lanes": 32, "sym_group": 16},   # one warp per light row in every pass
    {"accum": ACC_COPIES, "row_lanes": 32}, {"accum": ACC_COPIES, "row_lanes": 4, "group": 32},
    {"row_lanes": 1}, {"row_lanes": 1, "cta_min_flops": 1}, {"row_lanes": 1, "warps_per_cta": 3},  # shared accumulators
]


@pytest.fixture(scope="module")
def er_case():
    # the Erdos-Renyi workload at its full size: n = 16384, 8 per row, d = 64, 10 %
    return synth.er_product(n=16384, k=8, d=64, density=0.10)


@pytest.mark.parametrize("tuning", TUNINGS)
def test_er_full_size(er_case, tuning):
    A, B = er_case
    C = spgemm(dev(A), dev(B), tuning=tuning)
    compare_full(C, A, B)


@pytest.mark.parametrize("tuning", [None, {"col_tile": 32}, {"cta_min_flops": 1}, {"accum": ACC_HASH},
                                    {"stage": 2, "group": 1}, {"stage": 2, "group": 32}, {"accum": ACC_COPIES},
                                    {"group": 2, "sym_group": 2}])
def test_er_boolean(er_case, tuning):
    A, B = er_case
    C = spgemm(dev(A).pattern(), dev(B).pattern(), semiring=OR_SELECT2ND, tuning=tuning)
    assert C.val is None
    compare_full(C, A, B, semiring=oracle.OR_SELECT2ND)


@pytest.mark.parametrize("tuning", [None, {"col_tile": 64}, {"col_tile": 96}, {"cta_min_flops": 128},
                                    {"accum": ACC_HASH, "hash_slots": 512}, {"stage": 2, "group": 1},
                                    {"stage": 2, "group": 8}, {"stage": 2, "group": 32, "pack_b": 1},
                                    {"stage": 2, "pack_b": 1, "col_tile": 64}, {"col_tile": 64, "warps_per_cta": 2},
                                    {"accum": ACC_COPIES}, {"accum": ACC_COPIES, "group": 8, "col_tile": 64},
                                    {"accum": ACC_COPIES, "cta_min_flops": 128, "pack_b": 2},
                                    {"group": 2, "sym_group": 2}, {"group": 2, "col_tile": 64, "cta_min_flops": 128},
                                    {"row_lanes": 4}, {"row_lanes": 8, "col_tile": 64}, {"row_lanes": 16, "group": 2},
                                    {"row_lanes": 32}])
def test_rmat_embedding_small(tuning):
    A, B = synth.rmat_embedding(scale=13, edge_factor=16, d=256, density=0.05, seed=31)
    C = spgemm(dev(A), dev(B), tuning=tuning)
    compare_full(C, A, B)


def test_rmat_tiled_d1024():
    # the large tiled product's shape at small scale: d = 1024, 1 %, tiles of 256
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=1024, density=0.01, seed=32, b_values="uniform")
    for t in (None, {"col_tile": 256}, {"col_tile": 256, "cta_min_flops": 32}, {"accum": ACC_HASH},
              {"accum": ACC_COPIES}, {"accum": ACC_COPIES, "col_tile": 256, "cta_min_flops": 32}):
        compare_full(spgemm(dev(A), dev(B), tuning=t), A, B)


@pytest.fixture(scope="module")
def tiled_full():
    A, B = synth.rmat_embedding(scale=24, edge_factor=16, d=1024, density=0.01, b_values="uniform",
                                seed=synth.BASE_SEED + 5)
    return A, B, oracle.spgemm_count(A, B)


@pytest.mark.parametrize("tuning", [None, {"col_tile": 256}])
def test_tiled_full_size_sampled(tiled_full, tuning):
    # the large product at its full size (R-MAT scale 24, d = 1024, 1 %) in
    # the launch configuration the benchmark times (default: one 1024-wide
    # accumulator made of the four 256-column tiles) and with B walked in
    # column tiles of 256: C's row pointers for all rows, and sampled rows of
    # C, of dA and of dB against the oracle
    A, B, Cp_all = tiled_full
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning=tuning)
    C = plan.forward(Ad, Bd)
    rp = C.rowptr.cpu().numpy()
    np.testing.assert_array_equal(rp, Cp_all)
    rng = np.random.default_rng(24)
    deg = np.diff(A.rowptr)
    rows = np.concatenate([np.argsort(deg)[-8:], rng.choice(A.nrows, 1000, replace=False)])
    compare_rows(C, A, B, rows)
    dC = synth.grad_output(C.nnz, 25)
    dA, dB = plan.backward(Ad, Bd, C, torch.as_tensor(dC, device="cuda"))
    col = C.col.cpu().numpy()
    dC = dC.astype(np.float64)
    arows = np.concatenate([np.argsort(deg)[-4:], rng.choice(A.nrows, 500, replace=False)])
    sA, bA = oracle.backward_dA_rows(A, B, rp, col, dC, arows)
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in arows])
    assert np.all(np.abs(dA.cpu().numpy()[idx] - sA) <= REL * bA)
    indeg = np.bincount(A.col, minlength=A.nrows)
    krows = np.unique(np.concatenate([np.argsort(indeg)[-4:], rng.choice(B.nrows, 200, replace=False)]))
    sB, bB = oracle.backward_dB_rows(A, B, rp, col, dC, krows)
    idx = np.concatenate([np.arange(B.rowptr[k], B.rowptr[k + 1]) for k in krows])
    assert np.all(np.abs(dB.cpu().numpy()[idx] - sB) <= REL * bB)


def test_large_d_hash_and_tiles():
    A = synth.rmat(11, 8, 33)
    A.val = synth.uniform(A.nnz, 34)
    B = synth.tall_skinny(A.nrows, 5000, 0.002, 35)
    B.val = synth.normal(B.nnz, 36)
    for t in (None, {"accum": ACC_HASH, "hash_slots": 256}, {"accum": ACC_DENSE, "col_tile": 2048}):
        compare_full(spgemm(dev(A), dev(B), tuning=t), A, B)


def _csr(n, ncols, rows, vals=True, seed=0):
    rng = np.random.default_rng(seed)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for i, r in enumerate(rows):
        r = np.unique(np.asarray(r, dtype=np.int64))
        cols.append(r)
        rowptr[i + 1] = rowptr[i] + r.size
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = rng.random(col.size).astype(np.float32) if vals else None
    return CSR(n, ncols, rowptr, col, val)


@pytest.mark.parametrize("n,d", [(1, 1), (3, 33), (200, 100), (64, 32)])
def test_small_shapes_and_ragged_d(n, d):
    rng = np.random.default_rng(n * 7 + d)
    A = _csr(n, n, [rng.choice(n, size=rng.integers(0, n + 1), replace=False) for _ in range(n)], seed=1)
    B = _csr(n, d, [rng.choice(d, size=rng.integers(0, d + 1), replace=False) for _ in range(n)], seed=2)
    for t in (None, {"col_tile": 32}, {"cta_min_flops": 1}, {"accum": ACC_HASH, "hash_slots": 256},
              {"stage": 2, "group": 1}, {"stage": 2, "group": 4, "pack_b": 1},
              {"stage": 2, "group": 32, "cta_min_flops": 1}, {"warps_per_cta": 1}, {"accum": ACC_COPIES},
              {"accum": ACC_COPIES, "group": 32, "cta_min_flops": 1}, {"accum": ACC_COPIES, "col_tile": 32},
              {"group": 2, "sym_group": 2}, {"group": 2, "sym_group": 2, "cta_min_flops": 1},
              {"row_lanes": 4}, {"row_lanes": 16, "col_tile": 32}):
        compare_full(spgemm(dev(A), dev(B), tuning=t), A, B)


def test_empty_operands():
    n, d = 500, 64
    A, B = synth.er_product(n=n, k=4, d=d, density=0.1, seed=5)
    Z = CSR(n, n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    Zb = CSR(n, d, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    for a, b in ((Z, B), (A, Zb), (Z, Zb)):
        C = spgemm(dev(a), dev(b))
        rp, col, val = C.to_host()
        assert np.all(rp == 0) and C.nnz == 0


def test_identity_is_exact():
    n, d = 3000, 96
    B = synth.tall_skinny(n, d, 0.3, 7)
    B.val = synth.normal(B.nnz, 8)
    I = CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n, np.float32))
    for t in (None, {"col_tile": 32}, {"accum": ACC_HASH}, {"accum": ACC_COPIES},
              {"accum": ACC_COPIES, "cta_min_flops": 1}, {"group": 2, "sym_group": 2}, {"row_lanes": 4}):
        rp, col, val = spgemm(dev(I), dev(B), tuning=t).to_host()
        np.testing.assert_array_equal(rp, B.rowptr)
        np.testing.assert_array_equal(col, B.col)
        assert np.array_equal(val, B.val)  # one term 1*b per entry: bit-exact


def test_hub_row_and_dense_b():
    n, d = 6000, 128
    rng = np.random.default_rng(9)
    rows = [np.arange(n)] + [rng.choice(n, size=3, replace=False) for _ in range(n - 1)]
    A = _csr(n, n, rows, seed=10)                  # row 0 touches every row of B
    B = synth.tall_skinny(n, d, 1.0, 11)           # fully dense rows
    B.val = synth.uniform(B.nnz, 12)
    for t in (None, {"cta_min_flops": 1 << 20}, {"warps_per_cta": 2}, {"stage": 2, "group": 1},
              {"stage": 2, "group": 32}, {"accum": ACC_COPIES}, {"accum": ACC_COPIES, "group": 8},
              {"accum": ACC_COPIES, "cta_min_flops": 1 << 20}, {"group": 2, "sym_group": 2},
              {"group": 2, "sym_group": 2, "cta_min_flops": 1 << 20}, {"row_lanes": 4},
              {"row_lanes": 8, "cta_min_flops": 1 << 20}):
        compare_full(spgemm(dev(A), dev(B), tuning=t), A, B)


@pytest.mark.parametrize("d", [100, 1000, 1100])
def test_heavy_rows_reaching_every_column(d):
    # Heavy rows and split parts stop marking once all d columns are marked.
    # Row 0 reaches every column only through its last entry's row of B;
    # row 1 never reaches column d - 1; rows 2-3 saturate early (split rows).
    n = 3000
    rng = np.random.default_rng(80 + d)
    B0 = synth.tall_skinny(n, d, 0.12, 81 + d)
    Bp, Bc = B0.rowptr, B0.col
    cols = [Bc[Bp[r]:Bp[r + 1]][Bc[Bp[r]:Bp[r + 1]] < d - 1] for r in range(n)]
    cols[n - 1] = np.union1d(cols[n - 1], [d - 1])  # column d - 1 only in row n - 1 of B
    B = _csr(n, d, cols, seed=83 + d)
    rows = [np.arange(n), np.arange(n - 1), rng.choice(n - 1, 2500, replace=False), rng.choice(n - 1, 1500, replace=False)]
    rows += [rng.choice(n, size=int(rng.integers(0, 40)), replace=False) for _ in range(n - 4)]
    A = _csr(n, n, rows, seed=84 + d)
    for t in (None, {"cta_min_flops": 1}, {"sym_group": 1}, {"sym_group": 16}, {"row_lanes": 32},
              {"cta_min_flops": 64, "warps_per_cta": 2}):
        Cp, _, _, _ = compare_full(spgemm(dev(A), dev(B), tuning=t), A, B)
        assert Cp[1] - Cp[0] == d and Cp[2] - Cp[1] == d - 1
        compare_full(spgemm(dev(A).pattern(), dev(B).pattern(), semiring=OR_SELECT2ND, tuning=t), A, B,
                     semiring=oracle.OR_SELECT2ND)


@pytest.fixture(scope="module")
def embed_full():
    return synth.rmat_embedding()


@pytest.fixture(scope="module")
def embed_full_rowptr(embed_full):
    # C's row pointers for every row, from the oracle's count pass
    A, B = embed_full
    return oracle.spgemm_count(A, B)


@pytest.mark.parametrize("tuning", [None, {"accum": ACC_COPIES}, {"group": 2, "sym_group": 2}, {"row_lanes": 4},
                                    {"row_lanes": 32}])
def test_embedding_full_size_sampled(embed_full, embed_full_rowptr, tuning):
    # sparse-embedding workload at full size: R-MAT scale 22, d = 256, 5 %:
    # C's row pointers for all rows, columns and values on sampled rows
    A, B = embed_full
    Ad, Bd = dev(A), dev(B)
    C = spgemm(Ad, Bd, tuning=tuning)
    rp = C.rowptr.cpu().numpy()
    np.testing.assert_array_equal(rp, embed_full_rowptr)
    deg = np.diff(A.rowptr)
    rng = np.random.default_rng(0)
    rows = np.concatenate([np.argsort(deg)[-8:], rng.choice(A.nrows, 3000, replace=False)])
    compare_rows(C, A, B, rows)


def test_validate_and_device_checks():
    n, d = 1000, 64
    A, B = synth.er_product(n=n, k=6, d=d, density=0.1, seed=14)
    validate(dev(A))
    validate(dev(B))
    bad = CSR(n, d, B.rowptr.copy(), B.col.copy(), B.val)
    r = int(np.nonzero(np.diff(B.rowptr) >= 2)[0][0])
    s = int(B.rowptr[r])
    bad.col[s], bad.col[s + 1] = bad.col[s + 1], bad.col[s]   # unsorted row
    with pytest.raises(TSError) as ei:
        validate(dev(bad))
    assert ei.value.status == -2
    # a column of B outside [0, d) is caught by the kernels' own checks
    oob = CSR(n, d, B.rowptr.copy(), B.col.copy(), B.val)
    oob.col[s] = d + 5
    plan = Plan(dev(A), dev(oob))
    with pytest.raises(TSError) as ei:
        plan.forward(dev(A), dev(oob))
    assert ei.value.status == -2


def test_state_and_argument_errors():
    A, B = synth.er_product(n=300, k=4, d=64, density=0.1, seed=15)
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd)
    rowptr = torch.zeros(301, dtype=torch.int64, device="cuda")
    C = plan.alloc_c(rowptr, 0)
    with pytest.raises(TSError) as ei:       # numeric before any symbolic pass
        plan.numeric(Ad, Bd, C)
    assert ei.value.status == -8
    with pytest.raises(TSError):
        Plan(Ad, dev(synth.tall_skinny(299, 64, 0.1, 1)))
    with pytest.raises(TSError):
        Plan(Ad, Bd, tuning={"col_tile": 48})


def test_autotune_keeps_results():
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=256, density=0.05, seed=40)
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd)
    C = plan.forward(Ad, Bd)
    dC = torch.randn(C.nnz, device="cuda")
    best = plan.autotune(Ad, Bd, C, dC_val=dC, reps=1)
    assert best["col_tile"] % 32 == 0
    compare_full(C, A, B)
    compare_full(plan.forward(Ad, Bd), A, B)


@pytest.mark.parametrize("tuning", [None, {"col_tile": 256}, {"col_tile": 256, "stage": 2, "group": 1},
                                    {"stage": 2, "pack_b": 1}, {"stage": 2}, {"accum": ACC_COPIES},
                                    {"accum": ACC_COPIES, "col_tile": 256}, {"group": 2, "sym_group": 2},
                                    {"group": 2, "sym_group": 2, "col_tile": 256}, {"row_lanes": 8},
                                    {"row_lanes": 4, "col_tile": 256}])
def test_split_rows_with_tiles(tuning):
    # rows longer than 1024 entries of A are cut into parts processed by
    # different blocks and merged through a staging row; with d = 1024 and
    # 256-wide tiles every part adds four tiles
    n, d = 5000, 1024
    rng = np.random.default_rng(70)
    rows = [np.arange(n), rng.choice(n, 3000, replace=False), np.arange(0, n, 2)]
    rows += [rng.choice(n, size=int(rng.integers(0, 12)), replace=False) for _ in range(n - 3)]
    A = _csr(n, n, rows, seed=71)
    B = synth.tall_skinny(n, d, 0.01, 72)
    B.val = synth.normal(B.nnz, 73)
    compare_full(spgemm(dev(A), dev(B), tuning=tuning), A, B)
    Cb = spgemm(dev(A).pattern(), dev(B).pattern(), semiring=OR_SELECT2ND, tuning=tuning)
    compare_full(Cb, A, B, semiring=oracle.OR_SELECT2ND)


def test_more_long_rows_than_split_slots():
    # 8300 rows of 1100 entries: more long rows than the 8192 split slots, so
    # some run as whole rows
    n, d, per = 8300, 32, 1100
    rng = np.random.default_rng(74)
    col = np.sort(np.stack([rng.choice(n, per, replace=False) for _ in range(n)]), axis=1)
    A = CSR(n, n, np.arange(n + 1, dtype=np.int64) * per, col.reshape(-1).astype(np.int32),
            synth.uniform(n * per, 75))
    B = synth.tall_skinny(n, d, 1.0 / 32, 76)
    B.val = synth.uniform(B.nnz, 77)
    rng2 = np.random.default_rng(1)
    rows = rng2.choice(n, 400, replace=False)
    for t in (None, {"accum": ACC_COPIES}, {"row_lanes": 4}):
        compare_rows(spgemm(dev(A), dev(B), tuning=t), A, B, rows)


@pytest.mark.parametrize("tuning", [None, {"accum": ACC_COPIES}, {"accum": ACC_COPIES, "cta_min_flops": 1},
                                    {"accum": ACC_HASH}, {"group": 2}, {"row_lanes": 4}])
def test_nan_products_keep_their_columns(tuning):
    # NaN values of B (one of them with the copies kernel's empty-column bit
    # pattern) must give NaN entries at their columns, never drop them
    A, B = synth.er_product(n=2000, k=6, d=64, density=0.1, seed=90)
    bits = B.val.view(np.uint32).copy()
    bits[::97] = 0x7FC00000
    bits[5::211] = 0xFFBADBAD
    B.val = bits.view(np.float32)
    rp, col, val = spgemm(dev(A), dev(B), tuning=tuning).to_host()
    Cp, Ci, Cx, bound = oracle.spgemm(A, B)
    np.testing.assert_array_equal(rp, Cp)
    np.testing.assert_array_equal(col, Ci)
    nan = np.isnan(Cx)
    assert nan.any()
    assert np.array_equal(np.isnan(val), nan)
    assert np.all(np.abs(val[~nan] - Cx[~nan]) <= 1e-5 * bound[~nan])


@pytest.mark.parametrize("tuning", [{"group": 2, "sym_group": 2}, None])
def test_unaligned_b_columns_and_b_tail(tuning):
    # B's column array one int into a buffer (not 16-byte aligned: symbolic
    # quads must not be used) and nnz(B) not a multiple of four (the last
    # quads of B take single loads)
    for seed in range(91, 110):
        A, B = synth.er_product(n=1500, k=6, d=80, density=0.09, seed=seed)
        if B.nnz % 4:
            break
    assert B.nnz % 4
    Bd = dev(B)
    buf = torch.zeros(B.nnz + 8, dtype=torch.int32, device="cuda")
    buf[1:1 + B.nnz] = Bd.col
    Bu = DeviceCSR(B.nrows, B.ncols, Bd.rowptr, buf[1:1 + B.nnz], Bd.val)
    assert Bu.col.data_ptr() % 16 != 0
    for Bx in (Bd, Bu):
        compare_full(spgemm(dev(A), Bx, tuning=tuning), A, B)


def _wide_hub_product(seed=93, n=4096, d=8192, hub=7, hub_len=3000, density=None):
    """d = 8192 (hash accumulator) with one hub row of A whose row of C holds
    about 7,700 distinct columns, more than a block's hash table holds at
    75% load with the default 8 warps x 1024 slots (6,144)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        k = hub_len if i == hub else 8
        rows.append(np.sort(rng.choice(n, k, replace=False)))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    A = CSR(n, n, rp, np.concatenate(rows).astype(np.int32), rng.random(int(rp[-1]), dtype=np.float32))
    B = synth.tall_skinny(n, d, density or 8.0 / d, seed + 1)
    B.val = synth.uniform(B.nnz, seed + 2)
    return A, B


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 2}, {"hash_slots": 64, "warps_per_cta": 1},
                                    {"hash_slots": 256, "warps_per_cta": 4}])
def test_hash_block_row_wider_than_table(tuning):
    A, B = _wide_hub_product()
    t = dict(tuning or {}, accum=ACC_HASH)
    C = spgemm(dev(A), dev(B), tuning=t)
    Cp, _, _, _ = compare_full(C, A, B)
    assert Cp[8] - Cp[7] > 6144  # the hub row really is wider than the default table


def test_autotune_wide_hub_row():
    # the autotuner tries hash tables of several sizes on a product with a row
    # wider than some of them; it must finish and leave the right product
    A, B = _wide_hub_product(seed=94)
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd)
    C = plan.forward(Ad, Bd)
    plan.autotune(Ad, Bd, C, reps=1)
    plan.check()
    compare_full(C, A, B)
    compare_full(plan.forward(Ad, Bd), A, B)


WIDE_TUNINGS = [None, {"cta_min_flops": 1}, {"cta_min_flops": 1 << 20}, {"warps_per_cta": 1},
                {"warps_per_cta": 4, "cta_min_flops": 64}, {"warps_per_cta": 8, "cta_min_flops": 300}]


@pytest.mark.parametrize("d", [1024, 700, 288])
@pytest.mark.parametrize("tuning", WIDE_TUNINGS)
def test_wide_rows_shared_accumulator(d, tuning):
    # one column tile of 256 < W <= 1024 columns: light rows one warp each,
    # heavy rows and split parts one block each, on one shared accumulator
    # per team with occupancy bits (row_lanes = 1, the default there)
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=d, density=0.01, seed=60 + d % 7, b_values="uniform")
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning=tuning)
    assert plan.tuning["row_lanes"] == 1
    compare_full(plan.forward(Ad, Bd), A, B)


@pytest.mark.parametrize("tuning", [None, {"cta_min_flops": 1}, {"warps_per_cta": 2}, {"cta_min_flops": 1 << 20}])
def test_wide_rows_split_hub(tuning):
    # a hub row of 3000 entries of A (three split parts) reaching all 1024
    # columns, and dense-ish rows of B (5 %)
    A, B = _wide_hub_product(seed=95, d=1024, density=0.05)
    C = spgemm(dev(A), dev(B), tuning=tuning)
    Cp, _, _, _ = compare_full(C, A, B)
    assert Cp[8] - Cp[7] == 1024


def test_wide_rows_nan_and_empty():
    # NaN products keep their columns; empty rows of A and of B
    A, B = synth.rmat_embedding(scale=11, edge_factor=8, d=1024, density=0.01, seed=96, b_values="uniform")
    B.val = B.val.copy()
    B.val[::97] = np.nan
    C = spgemm(dev(A), dev(B))
    rp, col, val = C.to_host()
    Cp, Ci, Cx, Cb = oracle.spgemm(A, B)
    assert_pattern_equal(rp, col, Cp, Ci)
    both = np.isnan(Cx)
    np.testing.assert_array_equal(np.isnan(val[: Cx.size]), both)
    assert_values_close(val[: Cx.size][~both], Cx[~both], Cb[~both])


def _full_b(n, d, seed):
    """B with every one of its n*d entries stored (the dense-B SpMM case)."""
    rp = np.arange(0, n * d + 1, d, dtype=np.int64)
    col = np.tile(np.arange(d, dtype=np.int32), n)
    return CSR(n, d, rp, col, synth.normal(n * d, seed))


@pytest.mark.parametrize("tuning", [{"accum": ACC_DENSE_B}, {"accum": ACC_DENSE_B, "cta_min_flops": 1},
                                    {"accum": ACC_DENSE_B, "cta_min_flops": 1 << 20},
                                    {"accum": ACC_DENSE_B, "warps_per_cta": 2}])
@pytest.mark.parametrize("d", [32, 64, 100, 128, 256])
def test_dense_b_all_entries(tuning, d):
    # B given all of its entries: a row-wise SpMM over a dense B; C's rows are
    # full wherever A's row is non-empty
    A = synth.rmat(11, 16, 80 + d)
    A.val = synth.uniform(A.nnz, 81)
    B = _full_b(A.nrows, d, 82)
    C = spgemm(dev(A), dev(B), tuning=tuning)
    compare_full(C, A, B)


@pytest.mark.parametrize("d,density,auto_dense_b", [(128, 0.02, False), (128, 0.3, False), (128, 0.7, True),
                                                     (128, 0.95, True), (256, 0.35, False), (256, 0.55, True),
                                                     (64, 0.95, False)])
def test_dense_b_partial_density_and_auto_switch(d, density, auto_dense_b):
    # B partly dense: the dense-B form keeps the structural pattern of Eq. 1;
    # without a forced accumulator the plan takes it above the measured
    # crossover (60 % for d <= 128, 45 % for d <= 256, never for d <= 64)
    A, B = synth.rmat_embedding(scale=12, edge_factor=16, d=d, density=density, seed=83, b_values="uniform")
    Ad, Bd = dev(A), dev(B)
    auto = Plan(Ad, Bd)
    assert auto.tuning["accum"] == (ACC_DENSE_B if auto_dense_b else ACC_DENSE)
    compare_full(auto.forward(Ad, Bd), A, B)
    compare_full(spgemm(Ad, Bd, tuning={"accum": ACC_DENSE_B}), A, B)


def test_dense_b_split_hub_and_boolean():
    # a split hub row (three parts) over a 60 % dense B, and the boolean
    # semiring with the dense-B accumulator requested (it runs the sparse
    # dense-accumulator path: the dense-B form is plus-times only)
    A, B = _wide_hub_product(seed=84, d=256, density=0.6)
    Ad, Bd = dev(A), dev(B)
    compare_full(spgemm(Ad, Bd, tuning={"accum": ACC_DENSE_B}), A, B)
    C = spgemm(Ad.pattern(), Bd.pattern(), semiring=OR_SELECT2ND, tuning={"accum": ACC_DENSE_B})
    compare_full(C, A, B, semiring=oracle.OR_SELECT2ND)


@pytest.mark.parametrize("tuning", [None, {"accum": ACC_HASH}, {"row_lanes": 1}, {"cta_min_flops": 1}])
def test_capture_forward_replays(er_case, tuning):
    # symbolic + numeric captured once in a CUDA graph (no host synchronisation
    # inside), replayed: C from scratch each time, and new values of B picked
    # up by a replay with the same pattern
    A, B = er_case
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd, tuning=tuning)
    g, C = plan.capture_forward(Ad, Bd)
    C.rowptr.fill_(0)
    C.col.fill_(-1)
    C.val.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    compare_full(C, A, B)
    Bd.val.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    compare_full(C, A, CSR(B.nrows, B.ncols, B.rowptr, B.col, (B.val * np.float32(2.0)).astype(np.float32)))


def test_capture_forward_capacity_overflow(er_case):
    # a C too small for the product: nothing is written past its capacity and
    # the check reports the rows that did not fit
    A, B = er_case
    Ad, Bd = dev(A), dev(B)
    plan = Plan(Ad, Bd)
    nnz = plan.forward(Ad, Bd).nnz
    guard = 64
    g, C = plan.capture_forward(Ad, Bd, capacity=nnz - 7)
    # the graph writes through C.col / C.val; a longer buffer behind them
    # shows that nothing lands past the capacity
    big_col = torch.full((nnz - 7 + guard,), -5, dtype=torch.int32, device="cuda")
    big_val = torch.full((nnz - 7 + guard,), 3.0, dtype=torch.float32, device="cuda")
    C2 = DeviceCSR(C.nrows, C.ncols, C.rowptr, big_col[: nnz - 7], big_val[: nnz - 7])
    plan.forward_into(Ad, Bd, C2)
    with pytest.raises(TSError):
        plan.check()
    assert int(C2.rowptr[-1].item()) == nnz
    assert bool((big_col[nnz - 7:] == -5).all()) and bool((big_val[nnz - 7:] == 3.0).all())
    g.replay()
    with pytest.raises(TSError):
        plan.check()
