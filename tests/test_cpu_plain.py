"""The multi-threaded CPU baseline (cpu_plain) against the FP64 oracle: the
same pattern bit for bit, values within the FP32 bound of the GPU tests."""
import numpy as np
import pytest

import cpu_plain
import oracle
import synth
from _cmp import REL


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("case", ["rmat", "er", "wide"])
def test_cpu_plain_matches_oracle(case, threads):
    if case == "rmat":
        A, B = synth.rmat_embedding(scale=10, edge_factor=16, d=256, density=0.05, seed=3)
    elif case == "er":
        A, B = synth.er_product(n=2000, k=6, d=64, density=0.1, seed=4)
    else:
        A, B = synth.rmat_embedding(scale=10, edge_factor=8, d=1024, density=0.01, seed=5)
    Cp, Ci, Cx = cpu_plain.spgemm(A, B, threads=threads)
    rp, col, val, bound = oracle.spgemm(A, B)
    assert np.array_equal(Cp, rp)
    assert np.array_equal(Ci, col)
    assert np.all(np.abs(Cx.astype(np.float64) - val) <= REL * bound)


def test_cpu_plain_rejects_bad_columns():
    A, B = synth.er_product(n=300, k=4, d=32, density=0.2, seed=6)
    B.col[5] = 40  # outside [0, 32)
    with pytest.raises(ValueError):
        cpu_plain.spgemm(A, B, threads=2)
