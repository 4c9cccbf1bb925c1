"""Multi-source BFS (paper Alg. 3) on the msbfs_init / msbfs_step kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from . import _native as N
from .ops import DeviceCSR, _ptr, _stream


@dataclass
class BfsResult:
    levels: torch.Tensor          # int32[n, d], -1 = unreached
    products: int                 # TS-SpGEMM products computed (loop iterations)
    frontier_nnz: List[int] = field(default_factory=list)  # nnz(F) entering each iteration
    parents: Optional[torch.Tensor] = None  # int32[n, d] BFS-tree parents (with parents=True)


def msbfs(A: DeviceCSR, sources: torch.Tensor, max_levels: int = 1 << 20, stream=None,
          parents: bool = False) -> BfsResult:
    """Levels of every vertex from each of the d sources (columns); with
    parents=True also the BFS tree of each source by the (sel2nd, min)
    semiring (the smallest neighbour on the previous level; d <= 256)."""
    dev = A.rowptr.device
    n = A.nrows
    src = sources.to(device=dev, dtype=torch.int32).contiguous()
    d = int(src.numel())
    if d < 1:
        raise ValueError("msbfs: need at least one source")
    s_host = src.cpu()
    if int(s_host.min()) < 0 or int(s_host.max()) >= n:
        raise ValueError("msbfs: source out of range")
    dw = (d + 31) // 32
    sz = ctypes.c_size_t()
    N.call("msbfs_workspace_size", n, A.nnz, d, ctypes.byref(sz))
    ws = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=dev)
    visited = torch.empty(n * dw, dtype=torch.int32, device=dev)
    levels = torch.empty(n * d, dtype=torch.int32, device=dev)
    cap = max(d, n)
    F = DeviceCSR(n, d, torch.empty(n + 1, dtype=torch.int64, device=dev),
                  torch.empty(cap, dtype=torch.int32, device=dev))
    G = DeviceCSR(n, d, torch.empty(n + 1, dtype=torch.int64, device=dev),
                  torch.empty(cap, dtype=torch.int32, device=dev))
    st = _stream(stream)
    f0 = F.desc()
    N.call("msbfs_init", n, d, _ptr(src), _ptr(visited), _ptr(levels), ctypes.byref(f0), st)
    par = None
    if parents:
        par = torch.empty(n * d, dtype=torch.int32, device=dev)
        N.call("msbfs_init_parents", n, d, _ptr(src), _ptr(par), st)
    F.nnz_ = d
    sizes = [d]
    products = 0
    Ad = A.desc()
    level = 0
    while F.nnz > 0 and level < max_levels:
        level += 1
        fd, gd = F.desc(), G.desc()
        nnz = ctypes.c_int64(0)
        if par is None:
            status = N.lib().msbfs_step(ctypes.byref(Ad), ctypes.byref(fd), _ptr(visited), _ptr(levels),
                                        level, ctypes.byref(gd), G.col.numel(), ctypes.byref(nnz),
                                        _ptr(ws), ws.numel(), st)
        else:
            status = N.lib().msbfs_step_parents(ctypes.byref(Ad), ctypes.byref(fd), _ptr(visited),
                                                _ptr(levels), _ptr(par), level, ctypes.byref(gd),
                                                G.col.numel(), ctypes.byref(nnz), _ptr(ws), ws.numel(), st)
        if status == N.TS_ERR_CAPACITY:
            G.col = torch.empty(int(nnz.value), dtype=torch.int32, device=dev)
            gd = G.desc()
            N.call("msbfs_emit", ctypes.byref(gd), G.col.numel(), _ptr(ws), ws.numel(), st)
        else:
            N.check(status, "msbfs_step")
        products += 1
        G.nnz_ = int(nnz.value)
        sizes.append(G.nnz)
        F, G = G, F
    return BfsResult(levels.view(n, d), products, sizes, None if par is None else par.view(n, d))
