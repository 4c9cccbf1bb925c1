"""Torch-facing wrappers of the TS-SpGEMM C ABI (marshalling only).

Every step of the product runs in the library's CUDA kernels; this module
only turns torch tensors into descriptors, owns the workspace tensor and
passes the current CUDA stream.  See include/tsspgemm.h for the contracts.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import torch

from . import _native as N


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@dataclass
class DeviceCSR:
    """CSR matrix on the GPU: rowptr int64[nrows+1], col int32[nnz],
    val float32[nnz] or None (pattern only)."""

    nrows: int
    ncols: int
    rowptr: torch.Tensor
    col: torch.Tensor
    val: Optional[torch.Tensor] = None
    nnz_: Optional[int] = None

    @property
    def nnz(self) -> int:
        return int(self.col.numel()) if self.nnz_ is None else int(self.nnz_)

    def desc(self) -> N.CsrDesc:
        return N.CsrDesc(self.nrows, self.ncols, self.nnz, self.rowptr.data_ptr(),
                         self.col.data_ptr() if self.col.numel() else None,
                         self.val.data_ptr() if (self.val is not None and self.val.numel()) else None)

    @staticmethod
    def from_host(M, device="cuda", with_values=True) -> "DeviceCSR":
        """From an object with nrows/ncols/rowptr/col/val numpy arrays."""
        rp = torch.as_tensor(M.rowptr, dtype=torch.int64).to(device)
        ci = torch.as_tensor(M.col, dtype=torch.int32).to(device)
        va = None
        if with_values and M.val is not None:
            va = torch.as_tensor(M.val, dtype=torch.float32).to(device)
        return DeviceCSR(int(M.nrows), int(M.ncols), rp, ci, va)

    def with_values(self, val: Optional[torch.Tensor]) -> "DeviceCSR":
        return DeviceCSR(self.nrows, self.ncols, self.rowptr, self.col, val, self.nnz_)

    def pattern(self) -> "DeviceCSR":
        return self.with_values(None)

    def to_host(self):
        rp = self.rowptr.cpu().numpy()
        n = int(rp[-1])
        col = self.col[:n].cpu().numpy()
        val = None if self.val is None else self.val[:n].detach().cpu().numpy()
        return rp, col, val


def _desc_ref(M: DeviceCSR):
    d = M.desc()
    return d, ctypes.byref(d)


class Plan:
    """A product plan (shapes, semiring, tuning) plus its device workspace."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, semiring: int = N.PLUS_TIMES,
                 tuning: Optional[dict] = None):
        self.n, self.d = A.nrows, B.ncols
        self.semiring = semiring
        h = ctypes.c_void_p()
        dA, dB = A.desc(), B.desc()
        force = N.Tuning.from_dict(tuning)
        N.call("ts_plan_create", ctypes.byref(dA), ctypes.byref(dB), semiring, ctypes.byref(force),
               ctypes.byref(h))
        self._h = h
        self._ws: Optional[torch.Tensor] = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib().ts_plan_destroy(h)
            except Exception:
                pass

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        sz = ctypes.c_size_t()
        N.call("ts_workspace_size", self._h, ctypes.byref(sz))
        return int(sz.value)

    def workspace(self, device="cuda") -> torch.Tensor:
        need = max(self.workspace_bytes(), 256)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws

    @property
    def tuning(self) -> dict:
        t = N.Tuning()
        N.call("ts_plan_get_tuning", self._h, ctypes.byref(t))
        return t.as_dict()

    def set_tuning(self, tuning: dict) -> None:
        t = N.Tuning.from_dict(tuning)
        N.call("ts_plan_set_tuning", self._h, ctypes.byref(t))

    # -- passes ------------------------------------------------------------
    def symbolic(self, A: DeviceCSR, B: DeviceCSR, sync: bool = True, stream=None):
        """C's row pointers (int64[n+1]) and nnz(C) (None if sync=False)."""
        ws = self.workspace(A.rowptr.device)
        rowptr = torch.empty(self.n + 1, dtype=torch.int64, device=A.rowptr.device)
        dA, dB = A.desc(), B.desc()
        nnz = ctypes.c_int64(-1)
        N.call("ts_spgemm_symbolic", self._h, ctypes.byref(dA), ctypes.byref(dB),
               _ptr(rowptr), ctypes.byref(nnz) if sync else None, _ptr(ws), ws.numel(),
               _stream(stream))
        return rowptr, (int(nnz.value) if sync else None)

    def alloc_c(self, rowptr: torch.Tensor, nnz: int) -> DeviceCSR:
        dev = rowptr.device
        col = torch.empty(max(nnz, 0), dtype=torch.int32, device=dev)
        val = (torch.empty(max(nnz, 0), dtype=torch.float32, device=dev)
               if self.semiring == N.PLUS_TIMES else None)
        return DeviceCSR(self.n, self.d, rowptr, col, val)

    def numeric(self, A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, stream=None) -> DeviceCSR:
        ws = self.workspace(A.rowptr.device)
        dA, dB, dC = A.desc(), B.desc(), C.desc()
        N.call("ts_spgemm_numeric", self._h, ctypes.byref(dA), ctypes.byref(dB), ctypes.byref(dC),
               _ptr(ws), ws.numel(), _stream(stream))
        return C

    def forward(self, A: DeviceCSR, B: DeviceCSR, stream=None) -> DeviceCSR:
        rowptr, nnz = self.symbolic(A, B, sync=True, stream=stream)
        C = self.alloc_c(rowptr, nnz)
        return self.numeric(A, B, C, stream=stream)

    def forward_into(self, A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, stream=None) -> DeviceCSR:
        """Symbolic + numeric into preallocated C (C.col / C.val hold
        C.nnz >= nnz(C) entries) with no host synchronisation: nnz(C) ends up
        in C.rowptr[n].  Capturable in a CUDA graph."""
        ws = self.workspace(A.rowptr.device)
        dA, dB = A.desc(), B.desc()
        N.call("ts_spgemm_symbolic", self._h, ctypes.byref(dA), ctypes.byref(dB), _ptr(C.rowptr), None,
               _ptr(ws), ws.numel(), _stream(stream))
        return self.numeric(A, B, C, stream=stream)

    def capture_forward(self, A: DeviceCSR, B: DeviceCSR, capacity: Optional[int] = None):
        """A CUDA graph of forward_into (for small products, where launches
        and the host synchronisation dominate).  C is sized by one eager
        forward (or `capacity`); returns (graph, C).  Replaying recomputes C
        from the current values of A and B; their patterns may change only
        while nnz(C) stays within C's capacity (else plan.check() raises)."""
        if capacity is None:
            capacity = self.forward(A, B).nnz
        rowptr = torch.empty(self.n + 1, dtype=torch.int64, device=A.rowptr.device)
        C = self.alloc_c(rowptr, capacity)
        self.workspace(A.rowptr.device)
        self.forward_into(A, B, C)  # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.forward_into(A, B, C, stream=torch.cuda.current_stream())
        return g, C

    def backward(self, A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, dC_val: torch.Tensor,
                 want_dA: bool = True, want_dB: bool = True, out_dA=None, out_dB=None, stream=None):
        ws = self.workspace(A.rowptr.device)
        dev = A.rowptr.device
        dA = out_dA if out_dA is not None else (
            torch.empty(A.nnz, dtype=torch.float32, device=dev) if want_dA else None)
        dB = out_dB if out_dB is not None else (
            torch.empty(B.nnz, dtype=torch.float32, device=dev) if want_dB else None)
        da, db, dc = A.desc(), B.desc(), C.desc()
        dC_val = dC_val.contiguous()
        N.call("ts_spgemm_backward", self._h, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc),
               _ptr(dC_val), _ptr(dA) if (dA is not None and dA.numel()) else None,
               _ptr(dB) if (dB is not None and dB.numel()) else None, _ptr(ws), ws.numel(),
               _stream(stream))
        return dA, dB

    def autotune(self, A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, dC_val=None, reps: int = 2,
                 stream=None) -> dict:
        ws = self.workspace(A.rowptr.device)
        dev = A.rowptr.device
        dA = dB = None
        if dC_val is not None:
            dA = torch.empty(max(A.nnz, 1), dtype=torch.float32, device=dev)
            dB = torch.empty(max(B.nnz, 1), dtype=torch.float32, device=dev)
        da, db, dc = A.desc(), B.desc(), C.desc()
        out = N.Tuning()
        N.call("ts_plan_autotune", self._h, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc),
               _ptr(dC_val), _ptr(dA), _ptr(dB), reps, ctypes.byref(out), _ptr(ws), ws.numel(),
               _stream(stream))
        return out.as_dict()

    def check(self, stream=None) -> None:
        """Synchronise and raise if a device-side check failed."""
        ws = self.workspace()
        N.call("ts_workspace_check", self._h, _ptr(ws), ws.numel(), _stream(stream))


def spgemm(A: DeviceCSR, B: DeviceCSR, semiring: int = N.PLUS_TIMES,
           tuning: Optional[dict] = None, plan: Optional[Plan] = None) -> DeviceCSR:
    """C = A * B over the semiring (symbolic + numeric)."""
    plan = plan or Plan(A, B, semiring, tuning)
    return plan.forward(A, B)


def validate(M: DeviceCSR, stream=None) -> None:
    """Raise TSError(TS_ERR_BAD_CSR) if M breaks the CSR rules of the ABI."""
    ws = torch.empty(int(N.lib().ts_validate_workspace_size()), dtype=torch.uint8,
                     device=M.rowptr.device)
    bad = ctypes.c_int64(-1)
    d = M.desc()
    N.call("ts_csr_validate", ctypes.byref(d), ctypes.byref(bad), _ptr(ws), ws.numel(),
           _stream(stream))
