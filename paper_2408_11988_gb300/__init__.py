"""GB300 (sm_103a) TS-SpGEMM: C = A * B with A square sparse (n x n) and B
sparse tall-and-skinny (n x d), after the local product of arXiv 2408.11988
(row-wise Gustavson, Eq. 1; dense/hash accumulators, Sec. III-C), plus the
multi-source BFS of its Alg. 3, a differentiable plus-times product and a
batched, graph-capturable launch.  The kernels live in libtsspgemm.so (C ABI:
include/tsspgemm.h); this package only marshals torch tensors to it.
"""
from ._native import (ACC_AUTO, ACC_COPIES, ACC_DENSE, ACC_DENSE_B, ACC_HASH, OR_SELECT2ND, PLUS_TIMES, TSError)

from .ops import DeviceCSR, Plan, spgemm, validate

__all__ = ["ACC_AUTO", "ACC_COPIES", "ACC_DENSE", "ACC_DENSE_B", "ACC_HASH", "OR_SELECT2ND", "PLUS_TIMES", "TSError",
           "DeviceCSR", "Plan", "spgemm", "validate"]
