"""Batched TS-SpGEMM through the ts_batched_* / ts_spgemm_batched* C ABI.

All instances run together, one launch per phase, each read and written in
place; every instance keeps its own tuning (accumulator, heavy threshold).
`forward` and `backward` never synchronise with the host, so they can be
captured once in a CUDA graph (`capture`) and replayed.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import torch

from . import _native as N
from .ops import DeviceCSR, _ptr, _stream



def _descs(ms: Sequence[DeviceCSR]):
    arr = (N.CsrDesc * len(ms))()
    for i, m in enumerate(ms):
        arr[i] = m.desc()
    return arr


def _ptrs(ts: Sequence[Optional[torch.Tensor]]):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if (t is None or t.numel() == 0) else t.data_ptr()
    return arr


class BatchedProduct:
    """count products C_b = A_b * B_b over one semiring, bound to fixed buffers."""

    def __init__(self, As: Sequence[DeviceCSR], Bs: Sequence[DeviceCSR], semiring: int = N.PLUS_TIMES,
                 tuning: Optional[dict] = None, stream=None):
        assert len(As) == len(Bs) and len(As) > 0
        self.As, self.Bs, self.count, self.semiring = list(As), list(Bs), len(As), semiring
        dev = As[0].rowptr.device
        self._dA, self._dB = _descs(self.As), _descs(self.Bs)
        h = ctypes.c_void_p()
        force = N.Tuning.from_dict(tuning)
        N.call("ts_batched_plan_create", self.count, self._dA, self._dB, semiring, ctypes.byref(force),
               ctypes.byref(h))
        self._h = h
        st = _stream(stream)
        self._ws = torch.empty(self._ws_bytes(), dtype=torch.uint8, device=dev)
        caps = (ctypes.c_int64 * self.count)()
        N.call("ts_batched_bounds", h, self._dA, self._dB, caps, _ptr(self._ws), self._ws.numel(), st)
        self.capacity = [int(c) for c in caps]
        self._ws = torch.empty(self._ws_bytes(), dtype=torch.uint8, device=dev)
        vals = semiring == N.PLUS_TIMES
        self.Cs: List[DeviceCSR] = []
        for A, B, cap in zip(self.As, self.Bs, self.capacity):
            self.Cs.append(DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device=dev),
                                     torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
                                     torch.empty(max(cap, 1), dtype=torch.float32, device=dev) if vals else None))
        self._dC = _descs(self.Cs)
        N.call("ts_batched_bind", h, self._dA, self._dB, self._dC, _ptr(self._ws), self._ws.numel(), st)
        self._grads = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib().ts_batched_plan_destroy(h)
            except Exception:
                pass

    def _ws_bytes(self) -> int:
        sz = ctypes.c_size_t()
        N.call("ts_batched_workspace_size", self._h, ctypes.byref(sz))
        return max(int(sz.value), 256)

    def forward(self, stream=None) -> List[DeviceCSR]:
        N.call("ts_spgemm_batched", self._h, self.count, self._dA, self._dB, self._dC, _ptr(self._ws),
               self._ws.numel(), _stream(stream))
        return self.Cs

    def bind_grads(self, dCs: Sequence[torch.Tensor], want_dA: bool = True, want_dB: bool = True, stream=None):
        dev = self.As[0].rowptr.device
        self.dCs = [t.contiguous() for t in dCs]
        self.dAs = [torch.empty(max(A.nnz, 1), dtype=torch.float32, device=dev) if want_dA else None for A in self.As]
        self.dBs = [torch.empty(max(B.nnz, 1), dtype=torch.float32, device=dev) if want_dB else None for B in self.Bs]
        self._grads = (_ptrs(self.dCs), _ptrs(self.dAs) if want_dA else None, _ptrs(self.dBs) if want_dB else None)
        N.call("ts_batched_bind_grads", self._h, self.count, self._grads[0], self._grads[1], self._grads[2],
               _ptr(self._ws), self._ws.numel(), _stream(stream))

    def backward(self, stream=None):
        g = self._grads
        N.call("ts_spgemm_batched_backward", self._h, self.count, g[0], g[1], g[2], _ptr(self._ws),
               self._ws.numel(), _stream(stream))
        return self.dAs, self.dBs

    def check(self, stream=None) -> None:
        N.call("ts_batched_check", self._h, _ptr(self._ws), self._ws.numel(), _stream(stream))

    def autotune(self, reps: int = 2, stream=None) -> dict:
        t = N.Tuning()
        N.call("ts_batched_autotune", self._h, reps, ctypes.byref(t), _ptr(self._ws), self._ws.numel(),
               _stream(stream))
        return t.as_dict()

    def tuning_summary(self) -> dict:
        """Per-instance tuning: counts of each accumulator kind and heavy
        threshold, and the list per instance."""
        per = []
        for b in range(self.count):
            t = N.Tuning()
            N.call("ts_batched_get_tuning", self._h, b, ctypes.byref(t))
            per.append({"accum": "dense_b" if t.accum == N.ACC_DENSE_B else "shared",
                        "width": int(t.col_tile), "heavy_min_flops": int(t.cta_min_flops)})
        kinds, mins = {}, {}
        for x in per:
            kinds[x["accum"]] = kinds.get(x["accum"], 0) + 1
            mins[str(x["heavy_min_flops"])] = mins.get(str(x["heavy_min_flops"]), 0) + 1
        return {"accumulators": kinds, "heavy_thresholds": mins, "per_instance": per}

    def capture(self, backward: bool = False) -> torch.cuda.CUDAGraph:
        """Capture forward (and backward) once; replay() recomputes them."""
        self.forward()
        if backward:
            self.backward()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.forward()
            if backward:
                self.backward()
        return g
