"""Sparse Force2Vec training on the f2v_step kernels (paper Sec. IV, sparse
embedding): minibatch SGD with attractive forces along the graph's edges and
repulsive forces from negative samples, the force product run as this
library's TS-SpGEMM, and each updated row sparsified to its k largest
entries.  This module only marshals tensors to the C ABI."""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _native as N
from .ops import DeviceCSR, _ptr, _stream


class Force2Vec:
    """Sparse embedding Z (n x d, exactly k entries per row, updated in place)
    of the graph A (n x n pattern)."""

    def __init__(self, A: DeviceCSR, Z: DeviceCSR, k: int, negatives: int = 5, lr: float = 0.02,
                 batch: int = 65536):
        if Z.val is None:
            raise ValueError("Force2Vec: Z needs values")
        self.A, self.Z, self.k, self.s, self.lr = A, Z, int(k), int(negatives), float(lr)
        self.batch = int(min(batch, A.nrows)) if A.nrows else 0
        sz = ctypes.c_size_t()
        N.call("f2v_workspace_size", A.nrows, Z.ncols, A.nnz, self.batch, self.s, self.k, ctypes.byref(sz))
        self._ws = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=A.rowptr.device)

    def step(self, r0: int, neg: torch.Tensor, b: Optional[int] = None, want_u: bool = False, stream=None):
        """One minibatch: rows [r0, r0+b) with negatives neg (int32[b*s], device).
        Returns the dense pre-sparsification update U (b x d) when want_u."""
        b = self.batch if b is None else int(b)
        if b > self.batch:
            raise ValueError("Force2Vec.step: batch larger than the workspace's")
        neg = neg.to(device=self.A.rowptr.device, dtype=torch.int32).contiguous()
        U = torch.empty(b * self.Z.ncols, dtype=torch.float32, device=self.A.rowptr.device) if want_u else None
        a, z = self.A.desc(), self.Z.desc()
        N.call("f2v_step", ctypes.byref(a), ctypes.byref(z), int(r0), b, _ptr(neg), self.s, self.lr, self.k,
               _ptr(U) if U is not None else None, _ptr(self._ws), self._ws.numel(), _stream(stream))
        return None if U is None else U.view(b, self.Z.ncols)

    def epoch(self, negatives: torch.Tensor, stream=None) -> int:
        """All rows once, in minibatches of `batch` consecutive rows; negatives:
        int32[n*s] (row i's samples at i*s).  Returns the number of minibatches."""
        n, s = self.A.nrows, self.s
        steps = 0
        for r0 in range(0, n, self.batch):
            b = min(self.batch, n - r0)
            self.step(r0, negatives[r0 * s:(r0 + b) * s], b=b, stream=stream)
            steps += 1
        return steps
