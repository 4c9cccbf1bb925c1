"""Differentiable plus-times TS-SpGEMM (torch.autograd.Function).

Forward: C = A * B (symbolic + numeric kernels).  Backward, with the
patterns of A, B and C fixed: dA = SDDMM(dC, B^T) on A's pattern and
dB = A^T dC on B's pattern, both from one fused kernel (ts_spgemm_backward).
The boolean semiring has no gradient.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _native as N
from .ops import DeviceCSR, Plan


class TSSpGEMMFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_val, B_val, A: DeviceCSR, B: DeviceCSR, plan: Plan):
        Av, Bv = A.with_values(A_val.detach()), B.with_values(B_val.detach())
        C = plan.forward(Av, Bv)
        ctx.plan, ctx.A, ctx.B, ctx.C = plan, Av, Bv, C.pattern()
        ctx.mark_non_differentiable(C.rowptr, C.col)
        return C.val, C.rowptr, C.col

    @staticmethod
    def backward(ctx, dC_val, _drowptr=None, _dcol=None):
        want_dA, want_dB = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if dC_val is None or not (want_dA or want_dB):
            return None, None, None, None, None
        dA, dB = ctx.plan.backward(ctx.A, ctx.B, ctx.C, dC_val.contiguous().float(),
                                   want_dA=want_dA, want_dB=want_dB)
        return dA, dB, None, None, None


def ts_spgemm(A: DeviceCSR, B: DeviceCSR, A_val: Optional[torch.Tensor] = None,
              B_val: Optional[torch.Tensor] = None, plan: Optional[Plan] = None):
    """Differentiable C = A * B.  A_val/B_val default to A.val/B.val; returns
    C as a DeviceCSR whose val carries the autograd graph."""
    A_val = A.val if A_val is None else A_val
    B_val = B.val if B_val is None else B_val
    plan = plan or Plan(A, B, N.PLUS_TIMES)
    val, rowptr, col = TSSpGEMMFn.apply(A_val, B_val, A.pattern(), B.pattern(), plan)
    return DeviceCSR(A.nrows, B.ncols, rowptr, col, val)
