"""Benchmark of the TS-SpGEMM hot path on GB300.

One step = one pass of the whole hot path over the workload: the symbolic
pass (row flops, binning, per-row nnz, scan), the numeric pass and the fused
backward (dA = SDDMM on A's pattern, dB = A^T dC on B's pattern).  The
default workload is the sparse-embedding product: R-MAT scale 22 (n =
4,194,304, edge factor 16, U(0,1) values) times B (n x 256, 5 % dense, N(0,1)),
plus-times, forward + backward.

Prints one JSON line.  `value` is useful GFLOP/s of forward + backward with
inputs resident in HBM (forward 2 flops per product, backward 4: dA and dB
each multiply and add once per product).  `e2e` is the same metric through
the public API with the inputs copied from pinned host memory and C, dA and
dB copied back inside the timed region (copies on their own streams,
overlapping the compute of neighbouring steps).  `roofline` is for the
numeric pass, `cpu_baseline` the FP64 oracle on a bounded sample of rows on
the host; before timing, the same sample of the GPU's C and dA is checked
against the oracle's (`verified`).

With the default workload on one GPU the line also carries two nested
records: `tiled_s24` (R-MAT scale 24, d = 1024, 1 %: phases, roofline,
oracle check and baseline, clocks) and `batched_64` (64 uneven instances:
plain per-instance forwards against one CUDA-graph replay of the batched
forward and forward + backward).  `--no-extra` leaves them out.

Under torchrun with N > 1, every rank runs an independent replica of the
workload (the product has no exchange step on one GPU per replica).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, generator kwargs, tuning, backward)
    "embed-s22": ("R-MAT scale 22, edge factor 16, U(0,1) A; B 4194304x256 at 5% N(0,1); "
                  "plus-times forward + backward",
                  dict(scale=22, edge_factor=16, d=256, density=0.05, b_values="normal"), None, True),
    "tiled-s24": ("R-MAT scale 24, edge factor 16, U(0,1) A; B 16777216x1024 at 1% U(0,1); "
                  "plus-times forward + backward; the four 256-column tiles of B held side by side "
                  "in one 1024-wide accumulator, so A is walked once",
                  dict(scale=24, edge_factor=16, d=1024, density=0.01, b_values="uniform"),
                  None, True),
    "er-16k": ("Erdos-Renyi A n=16384, 8 per row, U(0,1); B 16384x64 at 10% U(0,1); plus-times "
               "forward only", None, None, False),
    "batched-64": ("64 uneven R-MAT instances, n log-uniform in [2^12, 2^18], edge factor U{8..32}, "
                   "d in {32,64,128,256}, density log-uniform 1-50%, U(0,1); plus-times forward + backward "
                   "as one CUDA-graph replay", None, None, True),
    "msbfs-s20": ("multi-source BFS, R-MAT scale 20, edge factor 16, symmetrised, 128 sources, "
                  "(or, select2nd) iterated to an empty frontier", None, None, False),
    "force2vec-s20": ("sparse Force2Vec epoch: R-MAT scale 20, edge factor 16, symmetrised; embedding "
                      "1048576x128 with 26 entries per row (80% sparse), 5 negatives per row, lr 0.02, "
                      "minibatches of 65536 rows", None, None, False),
    "msbfs-parents-s20": ("multi-source BFS with BFS-tree parents, R-MAT scale 20, edge factor 16, "
                          "symmetrised, 128 sources, (sel2nd, min) iterated to an empty frontier",
                          None, None, False),
}

# FP32 tolerance of the plus-times product and gradients against the FP64
# oracle: |x_gpu - x_oracle| <= REL * sum |terms| per entry
REL = 1e-5


def _kernel_sources_hash():
    import hashlib
    h = hashlib.sha1()
    for f in ("numeric.cu", "numeric.cuh", "numeric_tiny.cu", "common.cuh", "staged.cuh", "layout.h", "wide.cuh",
              "rowgroup.cuh"):
        with open(os.path.join(ROOT, "paper_2408_11988_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(workload):
    """DRAM bytes per launch of the numeric pass from profiles/traffic.json (an
    ncu capture of the same workload), or None if that capture was taken on
    different kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(workload)
    if not rec or rec.get("sources_sha1") != _kernel_sources_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_info():
    """Host cores and CPU model (from lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu model")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)  # let the sampler start before the timed region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    from paper_2408_11988_gb300.replicas import world
    return world()


def _override_tag(args):
    """Suffix of the workload name for a run with a shape override ('' without)."""
    tag = ""
    for key in ("scale", "d", "density"):
        v = getattr(args, key, None)
        if v is not None:
            tag += f"@{key}{v}"
    return tag


def _override_desc(args, desc):
    """The workload's description, with the overridden shape named after it."""
    tag = _override_tag(args)
    return desc if not tag else desc + " [overridden: " + ", ".join(tag[1:].split("@")) + "]"


def make_inputs(name, seed_offset=0, scale=None, d=None, density=None):
    import synth
    desc, kw, tuning, bwd = WORKLOADS[name]
    if kw is not None:
        over = {k: v for k, v in (("scale", scale), ("d", d), ("density", density)) if v is not None}
        kw = dict(kw, **over)
    if name == "er-16k":
        A, B = synth.er_product(seed=synth.BASE_SEED + 1 + 1000 * seed_offset)
    else:
        from paper_2408_11988_gb300.replicas import replica_seed
        seed = replica_seed(synth.BASE_SEED + (3 if name == "embed-s22" else 5), seed_offset)
        A, B = synth.rmat_embedding(seed=seed, **kw)
    return A, B


def products_per_row(A, B):
    blen = np.diff(B.rowptr)
    per_entry = blen[A.col]
    cs = np.concatenate([[0], np.cumsum(per_entry, dtype=np.int64)])
    return cs[A.rowptr[1:]] - cs[A.rowptr[:-1]]


def cpu_plain_record(A, B, F, reps=2):
    """The forward on all host cores (cpu_plain: the paper's local kernel,
    Sec. III-C, OpenMP with a dense SPA per thread, FP32), full size, best of
    `reps` after one warm-up: a plain multi-core baseline beside the FP64
    single-thread oracle."""
    import cpu_plain
    threads = cpu_plain.max_threads()
    cpu_plain.spgemm(A, B, threads)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        cpu_plain.spgemm(A, B, threads)
        best = min(best, time.perf_counter() - t0)
    return {"value": round(2.0 * F / best / 1e9, 3), "unit": "GFLOP/s", "ms": round(best * 1e3, 2),
            "threads": threads, "host": host_info(),
            "what": "forward (row counts + values) of the whole product, FP32, rows of A over all host cores "
                    "(OpenMP) with a dense accumulator per thread; a plain baseline, not the oracle"}


def cpu_baseline(A, B, want_bwd, target_s=12.0, gpu=None):
    """The FP64 oracle on the first m rows of A (rows are randomly labelled by
    the R-MAT permutation, so a prefix is a uniform sample), sized to about
    target_s seconds of single-core work.

    With gpu = (C_rowptr, C_col, C_val, dA, dC) -- the GPU's results of the
    configuration about to be timed, as torch tensors, and the host dC it
    used -- the same rows of C and of dA are checked against the oracle's
    (patterns bit-exact, values within REL * sum |terms|); the result is in
    the returned dict under "verified"."""
    import oracle
    from synth import CSR
    fl = products_per_row(A, B)
    cum = np.cumsum(fl)

    def run(m):
        Asub = CSR(m, A.ncols, A.rowptr[: m + 1], A.col[: A.rowptr[m]], A.val[: A.rowptr[m]])
        t0 = time.perf_counter()
        Cp, Ci, Cx, Cb = oracle.spgemm(Asub, B)
        grads = None
        if want_bwd:
            if gpu is not None:
                dCs = gpu[4][: Ci.size].astype(np.float64)
            else:
                import synth
                dCs = synth.grad_output(Ci.size, 1).astype(np.float64)
            grads = oracle.backward(Asub, B, Cp, Ci, dCs)
        return time.perf_counter() - t0, int(cum[m - 1]) if m > 0 else 0, (Cp, Ci, Cx, Cb, grads, Asub)

    m = max(1, min(A.nrows, int(np.searchsorted(cum, min(cum[-1], 2_000_000)))))
    t, f, res = run(m)
    rate = f / max(t, 1e-6)
    m2 = int(np.searchsorted(cum, min(cum[-1], rate * target_s)))
    m2 = max(m, min(A.nrows, m2))
    if m2 > m:
        t, f, res = run(m2)
        m = m2
    flops = (6.0 if want_bwd else 2.0) * f
    out = {"value": flops / t / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
           "sample": f"rows 0..{m - 1} of {A.nrows} ({f} products, "
                     f"{'forward+backward' if want_bwd else 'forward'}), {t:.1f} s single-threaded FP64",
           "host": host_info()}
    if gpu is not None:
        out["verified"] = _verify_rows(m, res, gpu, A, want_bwd)
    return out


def _verify_rows(m, res, gpu, A, want_bwd):
    """Rows 0..m-1 of the GPU's C (and dA) against the oracle's results."""
    Cp, Ci, Cx, Cb, grads, _ = res
    rp_d, col_d, val_d, dA_d, _ = gpu
    rp = rp_d[: m + 1].cpu().numpy()
    nnz = int(Cp[-1])
    ok = bool(np.array_equal(rp, Cp))
    bad_vals = bad_da = -1
    if ok:
        ok = bool(np.array_equal(col_d[:nnz].cpu().numpy(), Ci))
    if ok:
        err = np.abs(val_d[:nnz].cpu().numpy().astype(np.float64) - Cx)
        bad_vals = int((err > REL * Cb).sum())
        ok = bad_vals == 0
    checked = f"rows 0..{m - 1}: C pattern bit-exact and values within {REL} * sum |a||b|"
    if want_bwd and grads is not None and dA_d is not None:
        na = int(A.rowptr[m])
        rA, bA = grads[0][:na], grads[1][:na]
        err = np.abs(dA_d[:na].cpu().numpy().astype(np.float64) - rA)
        bad_da = int((err > REL * bA).sum())
        ok = ok and bad_da == 0
        checked += f"; dA of their {na} entries within {REL} * sum |terms|"
    return {"ok": ok, "checked": checked, "bad_values": bad_vals, "bad_dA": bad_da}


def product_config(workload, desc, A, B, F, ws):
    """The `config` of a product workload (the same dict in both arms)."""
    return {"workload": workload, "description": desc, "n": int(A.nrows), "d": int(B.ncols),
            "nnz_A": int(A.nnz), "nnz_B": int(B.nnz), "products": int(F),
            "l2": "inputs larger than L2 (A+B+C > 129 MB)", "parallelism": f"replicas x{ws}"}


def measure_product(args, name, ws, rank, local, dist, tuning_json=None, steps=None, warmup=None,
                    want_e2e=True, want_cpu=True, nested=False):
    """Time the workload's forward (+ backward) step; returns the JSON record."""
    import torch
    from paper_2408_11988_gb300 import DeviceCSR, Plan
    from paper_2408_11988_gb300 import _native as N
    import synth
    desc, _, wl_tuning, want_bwd = WORKLOADS[name]
    steps = steps or args.steps
    warmup = warmup or args.warmup
    A, B = make_inputs(name, seed_offset=rank, scale=args.scale, d=args.d, density=args.density)
    flops_row = products_per_row(A, B)
    F = int(flops_row.sum())
    Ad, Bd = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    tuning = dict(wl_tuning or {})
    if tuning_json:
        tuning.update(json.loads(tuning_json))
    plan = Plan(Ad, Bd, tuning=tuning or None)
    C = plan.forward(Ad, Bd)
    nnzC = C.nnz
    dC_host = synth.grad_output(nnzC, 1) if want_bwd else None
    dC = torch.as_tensor(dC_host, device="cuda") if want_bwd else None
    if args.autotune:
        plan.autotune(Ad, Bd, C, dC_val=dC, reps=2)
    stream = torch.cuda.current_stream()
    last = {}

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        rowptr, nnz = plan.symbolic(Ad, Bd, sync=True)
        if ev:
            ev[1].record(stream)
        Cs = plan.alloc_c(rowptr, nnz)
        plan.numeric(Ad, Bd, Cs)
        if ev:
            ev[2].record(stream)
        dA = None
        if want_bwd:
            dA, _ = plan.backward(Ad, Bd, Cs, dC)
        if ev:
            ev[3].record(stream)
        last["C"], last["dA"] = Cs, dA
        return Cs

    for _ in range(warmup):
        step()
    plan.check()
    torch.cuda.synchronize()
    # the configuration about to be timed, checked against the oracle on the
    # rows the CPU baseline runs (rank 0)
    cpu = None
    if rank == 0 and want_cpu and not args.no_cpu_baseline:
        Cl = last["C"]
        cpu = cpu_baseline(A, B, want_bwd, target_s=8.0 if nested else 12.0,
                           gpu=(Cl.rowptr, Cl.col, Cl.val, last["dA"], dC_host))
    plain = cpu_plain_record(A, B, F) if (rank == 0 and want_cpu and not args.no_cpu_baseline and not nested) else None
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    l0 = N.lib().ts_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(steps):
            step(evs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = N.lib().ts_kernel_launches() - l0
    total_ms = t_start.elapsed_time(t_end)
    sym = [e[0].elapsed_time(e[1]) for e in evs]
    num = [e[1].elapsed_time(e[2]) for e in evs]
    bwd = [e[2].elapsed_time(e[3]) for e in evs]
    total_ms = _max_over_ranks(dist, total_ms)
    ms = total_ms / steps
    flop_step = (6.0 if want_bwd else 2.0) * F
    value = flop_step * ws / (ms * 1e-3) / 1e9

    # roofline of the numeric pass: algorithmic bytes per launch / mean duration
    # (A's row pointers, columns, values and B's row bounds once per column
    # tile that the pass walks A for)
    n, nnzA = A.nrows, A.nnz
    tiles = 1
    if plan.tuning.get("accum") != 2 and plan.tuning.get("col_tile"):
        tiles = -(-B.ncols // int(plan.tuning["col_tile"]))
    num_bytes = tiles * (16 * (n + 1) + 24 * nnzA) + 8 * F + 8 * nnzC
    # compulsory bytes: every array of A, B and C touched once
    comp_bytes = 8 * (n + 1) + 8 * nnzA + 8 * (B.nrows + 1) + 8 * B.nnz + 8 * (n + 1) + 8 * nnzC
    bwd_bytes = 16 * (n + 1) + 28 * nnzA + 8 * F + 8 * nnzC + 4 * B.nnz
    sym_bytes = 8 * (n + 1) + 20 * nnzA + 4 * F + 8 * n
    peak, peak_kind = _peaks()
    num_ms = statistics.mean(num)
    achieved = num_bytes / (num_ms * 1e-3) / 1e9
    del last["C"], last["dA"]
    e2e = None
    if want_e2e and not args.no_e2e:
        e2e = run_e2e(args, A, B, dC_host, want_bwd, tuning, flop_step, ws, dist, steps, warmup)
    rec = {
        "metric": "TS-SpGEMM GFLOP/s (forward + backward, plus-times)" if want_bwd
        else "TS-SpGEMM GFLOP/s (forward, plus-times)",
        "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": ws, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms, 4),
        "ms_per_step_median": round(statistics.median([a + b + c for a, b, c in zip(sym, num, bwd)]), 4),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": product_config(name + _override_tag(args), _override_desc(args, desc), A, B, F, ws),
        "nnz_C": nnzC,
        "tuning": plan.tuning,
        "roofline": {"bound": "hbm", "kernel": "numeric pass (every kernel of ts_spgemm_numeric: packing of B, accumulating kernels)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "bytes_per_launch": num_bytes,
                     "bytes_formula": "tiles*(16(n+1)+24 nnz_A) + 8 products + 8 nnz_C",
                     "traffic": None if _override_tag(args) else _traffic(name),
                     "column_tiles": tiles, "compulsory_bytes": comp_bytes,
                     "compulsory_frac": round(comp_bytes / (num_ms * 1e-3) / 1e9 / peak, 4)},
        "phases_ms": {"symbolic": round(statistics.mean(sym), 4), "numeric": round(num_ms, 4),
                      "backward": round(statistics.mean(bwd), 4) if want_bwd else None},
        "phase_roofline_frac": {
            "symbolic": round(sym_bytes / (statistics.mean(sym) * 1e-3) / 1e9 / peak, 4),
            "numeric": round(achieved / peak, 4),
            "backward": round(bwd_bytes / (statistics.mean(bwd) * 1e-3) / 1e9 / peak, 4)
            if want_bwd else None},
        "forward_gflops": round(2.0 * F / ((statistics.mean(sym) + num_ms) * 1e-3) / 1e9, 3),
        "nnzC_per_s": round(nnzC / ((statistics.mean(sym) + num_ms) * 1e-3), 1),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "verified": cpu.pop("verified") if cpu else None,
        "cpu_plain": plain,
    }
    if not want_bwd:
        rec["graph_forward"] = graph_forward(plan, Ad, Bd, C, F, steps, warmup, dist)
    del plan, Ad, Bd, dC
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def graph_forward(plan, Ad, Bd, C, F, steps, warmup, dist):
    """The forward (symbolic + numeric, no host synchronisation) captured
    once in a CUDA graph and replayed: for small products, where launches
    and the host sync for nnz(C) dominate the eager call."""
    import torch
    from paper_2408_11988_gb300 import _native as N
    c0 = N.lib().ts_kernel_launches()
    g, Cg = plan.capture_forward(Ad, Bd)
    c1 = N.lib().ts_kernel_launches()
    for _ in range(max(warmup, 3)):
        g.replay()
    torch.cuda.synchronize()
    plan.check()
    same = bool(torch.equal(Cg.rowptr, C.rowptr) and torch.equal(Cg.col, C.col))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    ms = _max_over_ranks(dist, a.elapsed_time(b) / steps)
    # capture_forward runs one eager forward, one warm-up and the capture
    launches = (c1 - c0) // 3
    return {"ms": round(ms, 4), "gflops": round(2.0 * F / (ms * 1e-3) / 1e9, 3), "launches_per_replay": launches,
            "same_pattern_as_eager": same, "what": "symbolic + numeric into a preallocated C, one CUDA-graph replay"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="embed-s22", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: leave out the nested scale-24 and batched records")
    ap.add_argument("--autotune", action="store_true", help="autotune the plan before timing")
    ap.add_argument("--tuning", default=None, help="JSON dict of forced tuning fields")
    ap.add_argument("--scale", type=int, default=None,
                    help="R-MAT scale override (smaller copies of a workload for profiling)")
    ap.add_argument("--batched-autotune", default="instance", choices=["instance", "none"],
                    help="batched-64: per-instance autotuning (default) or the plan's default tuning")
    ap.add_argument("--d", type=int, default=None, help="columns of B override (profiling)")
    ap.add_argument("--density", type=float, default=None, help="density of B override (profiling)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    desc, _, wl_tuning, want_bwd = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, ws, rank, desc, want_bwd)
    if args.workload == "batched-64":
        return run_batched(args, ws, rank, local, desc)
    if args.workload in ("msbfs-s20", "msbfs-parents-s20"):
        return run_msbfs(args, ws, rank, local, desc)
    if args.workload == "force2vec-s20":
        return run_force2vec(args, ws, rank, local, desc)

    import torch
    torch.cuda.set_device(local)
    dist = _dist_setup(ws, local)
    line = measure_product(args, args.workload, ws, rank, local, dist, tuning_json=args.tuning)
    failed = line["verified"] is not None and not line["verified"]["ok"]
    if args.workload == "embed-s22" and ws == 1 and not args.no_extra and not _override_tag(args) and not args.tuning:
        # the other two configurations the target names, as nested records
        sub = argparse.Namespace(**vars(args))
        sub.autotune = False
        s24 = measure_product(sub, "tiled-s24", ws, rank, local, dist, steps=min(args.steps, 10),
                              warmup=3, want_e2e=False, nested=True)
        keep = ("value", "unit", "ms_per_step", "config", "nnz_C", "tuning", "roofline", "phases_ms",
                "phase_roofline_frac", "forward_gflops", "nnzC_per_s", "gpu_launches", "clocks", "cpu_baseline",
                "verified", "steps", "warmup")
        line["tiled_s24"] = {k: s24[k] for k in keep}
        failed = failed or (s24["verified"] is not None and not s24["verified"]["ok"])
        b64 = batched_record(args, ws, rank, local, dist, steps=min(args.steps, 10), warmup=3)
        line["batched_64"] = b64
        failed = failed or (b64.get("verified") is not None and not b64["verified"]["ok"])
    if rank == 0:
        print(json.dumps(line), flush=True)
        if failed:
            print("bench: a timed configuration differs from the oracle (see 'verified')", file=sys.stderr)
    if dist:
        dist.destroy_process_group()
    if failed:
        sys.exit(1)


def run_e2e(args, A, B, dC_host, want_bwd, tuning, flop_step, ws, dist, steps, warmup):
    """The step through the public API (Plan.forward / Plan.backward) with
    each step's inputs copied from pinned host memory and C (row pointers,
    columns, values), dA and dB copied back, all inside the timed region.
    Inputs go up on one stream into two alternating device buffers, results
    come down on another, so the copies of neighbouring steps overlap the
    compute of the current one."""
    import torch
    from paper_2408_11988_gb300 import DeviceCSR, Plan
    hin = [torch.as_tensor(x).pin_memory() for x in (A.rowptr, A.col, A.val, B.rowptr, B.col, B.val)]
    if want_bwd:
        hin.append(torch.as_tensor(dC_host).pin_memory())
    bufs = [[torch.empty_like(x, device="cuda") for x in hin] for _ in range(2)]
    comp = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    plan = Plan(DeviceCSR(A.nrows, A.ncols, *bufs[0][0:3]), DeviceCSR(B.nrows, B.ncols, *bufs[0][3:6]),
                tuning=tuning or None)
    n = A.nrows
    out_rp = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    out_col = out_val = None
    out_dA = torch.empty(max(A.nnz, 1), dtype=torch.float32).pin_memory() if want_bwd else None
    out_dB = torch.empty(max(B.nnz, 1), dtype=torch.float32).pin_memory() if want_bwd else None
    free = [None, None]
    h2d = sum(x.numel() * x.element_size() for x in hin)
    d2h = [0]

    def upload(k):
        b = bufs[k % 2]
        with torch.cuda.stream(up):
            if free[k % 2] is not None:
                up.wait_event(free[k % 2])
            for h, d in zip(hin, b):
                d.copy_(h, non_blocking=True)
            return up.record_event()

    def compute(k, ready):
        nonlocal out_col, out_val
        b = bufs[k % 2]
        comp.wait_event(ready)
        Ad = DeviceCSR(A.nrows, A.ncols, b[0], b[1], b[2])
        Bd = DeviceCSR(B.nrows, B.ncols, b[3], b[4], b[5])
        C = plan.forward(Ad, Bd)
        if out_col is None or out_col.numel() < C.nnz:
            out_col = torch.empty(max(C.nnz, 1), dtype=torch.int32).pin_memory()
            out_val = torch.empty(max(C.nnz, 1), dtype=torch.float32).pin_memory()
        fwd_done = comp.record_event()
        tensors = [C.rowptr, C.col, C.val]
        gA = gB = None
        if want_bwd:
            gA, gB = plan.backward(Ad, Bd, C, b[6][: C.nnz])
            tensors += [gA, gB]
        free[k % 2] = comp.record_event()
        done = comp.record_event()
        with torch.cuda.stream(down):
            down.wait_event(fwd_done)
            out_rp.copy_(C.rowptr, non_blocking=True)
            out_col[: C.nnz].copy_(C.col, non_blocking=True)
            out_val[: C.nnz].copy_(C.val, non_blocking=True)
            nb = 8 * (n + 1) + 8 * C.nnz
            if want_bwd:
                down.wait_event(done)
                out_dA[: A.nnz].copy_(gA, non_blocking=True)
                out_dB[: B.nnz].copy_(gB, non_blocking=True)
                nb += 4 * (A.nnz + B.nnz)
        for t in tensors:
            t.record_stream(down)
        d2h[0] = nb

    def run(k_steps):
        nxt = upload(0)
        for k in range(k_steps):
            ready = nxt
            if k + 1 < k_steps:
                nxt = upload(k + 1)
            compute(k, ready)
        comp.wait_stream(down)
        comp.wait_stream(up)

    run(max(1, warmup))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(comp)
    up.wait_event(s0)
    run(steps)
    s1.record(comp)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    ms = _max_over_ranks(dist, ms)
    del plan, bufs
    torch.cuda.empty_cache()
    return {"value": round(flop_step * ws / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
            "ms_per_step": round(ms, 4), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h[0]),
            "what": "Plan.forward + Plan.backward per step; inputs from pinned host memory, C (row pointers, "
                    "columns, values), dA and dB back to pinned host memory; copies on two streams of their "
                    "own, inputs double-buffered"}


def _dist_setup(ws, local):
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist
    return None


def _max_over_ranks(dist, v):
    from paper_2408_11988_gb300.replicas import max_over_ranks
    return max_over_ranks(v, dist, device="cuda")


def batched_record(args, ws, rank, local, dist, steps=None, warmup=None):
    """The uneven batch: plain per-instance forwards (each a symbolic with a
    host sync plus a numeric) against one CUDA-graph replay of the batched
    forward, and of the batched forward + backward.  Before timing, the
    largest instance's C and dA from the replayed graph are checked against
    the oracle on the rows the CPU baseline runs."""
    import torch
    import synth
    from paper_2408_11988_gb300 import DeviceCSR, Plan
    from paper_2408_11988_gb300 import _native as N
    from paper_2408_11988_gb300.batched import BatchedProduct
    steps = steps or args.steps
    warmup = warmup or args.warmup
    desc = WORKLOADS["batched-64"][0]
    inst = synth.batched_instances(seed=synth.BASE_SEED + 4 + 1000 * rank)
    F = sum(int(products_per_row(A, B).sum()) for A, B in inst)
    As = [DeviceCSR.from_host(A) for A, _ in inst]
    Bs = [DeviceCSR.from_host(B) for _, B in inst]
    tuning = json.loads(args.tuning) if args.tuning else None
    plans = [Plan(A, B, tuning=tuning) for A, B in zip(As, Bs)]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def plain():
        for p, A, B in zip(plans, As, Bs):
            p.forward(A, B)

    for _ in range(warmup):
        plain()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(steps):
        plain()
    e1.record()
    torch.cuda.synchronize()
    plain_ms = _max_over_ranks(dist, e0.elapsed_time(e1) / steps)
    del plans
    bp = BatchedProduct(As, Bs, tuning=tuning)
    # per-instance tuning (accumulator kind, heavy-row threshold) by the
    # batched autotuner: each instance timed on its own, then a few
    # whole-batch tunings built from those choices
    t_at = time.perf_counter()
    if args.batched_autotune != "none":
        bp.autotune(reps=1)
    autotune_s = time.perf_counter() - t_at
    Cs = bp.forward()
    torch.cuda.synchronize()
    dC_hosts = [synth.grad_output(int(C.rowptr[-1].item()), 1 + i) for i, C in enumerate(Cs)]
    dCs = [torch.as_tensor(h, device="cuda") for h in dC_hosts]
    bp.bind_grads(dCs)
    c0 = N.lib().ts_kernel_launches()
    gf = bp.capture(backward=False)
    c1 = N.lib().ts_kernel_launches()
    gfb = bp.capture(backward=True)
    c2 = N.lib().ts_kernel_launches()
    # each capture runs the sequence once eagerly (warm-up) and once captured
    per_fwd, per_fb = (c1 - c0) // 2, (c2 - c1) // 2
    nnzC = sum(int(C.rowptr[-1].item()) for C in Cs)
    for _ in range(warmup):
        gfb.replay()
    torch.cuda.synchronize()
    bp.check()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        big = max(range(len(inst)), key=lambda i: inst[i][0].nnz)
        A, B = inst[big]
        C = bp.Cs[big]
        cpu = cpu_baseline(A, B, True, target_s=6.0,
                           gpu=(C.rowptr, C.col, C.val, bp.dAs[big], dC_hosts[big]))
        cpu["sample"] = f"largest instance (#{big}): " + cpu["sample"]

    def timed(g):
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        a, b = ev(), ev()
        a.record()
        for _ in range(steps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        return _max_over_ranks(dist, a.elapsed_time(b) / steps)

    with ClockSampler(local) as clk:
        fwd_ms = timed(gf)
        fb_ms = timed(gfb)
    bp.check()
    n = sum(A.nrows for A, _ in inst)
    nnzA = sum(A.nnz for A, _ in inst)
    num_bytes = 16 * (n + 1) + 24 * nnzA + 8 * F + 8 * nnzC
    peak, peak_kind = _peaks()
    value = 6.0 * F * ws / (fb_ms * 1e-3) / 1e9
    rec = {
        "metric": "TS-SpGEMM GFLOP/s (batched forward + backward, plus-times)", "value": round(value, 3),
        "unit": "GFLOP/s", "n_gpus": ws, "steps": steps, "warmup": warmup,
        "ms_per_step": round(fb_ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched-64", "description": desc, "instances": len(inst), "rows": n,
                   "nnz_A": nnzA, "nnz_C": nnzC, "products": F, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2"},
        "tuning": dict({k: v for k, v in bp.tuning_summary().items() if k != "per_instance"},
                       autotune_s=round(autotune_s, 2),
                       per_instance=[[x["accum"], x["width"], x["heavy_min_flops"]]
                                     for x in bp.tuning_summary()["per_instance"]]),
        "plain_forward": {"ms": round(plain_ms, 4), "gflops": round(2.0 * F / (plain_ms * 1e-3) / 1e9, 3),
                          "what": "64 separate symbolic+numeric calls (host sync each)"},
        "batched_forward": {"ms": round(fwd_ms, 4), "gflops": round(2.0 * F / (fwd_ms * 1e-3) / 1e9, 3),
                            "what": "one CUDA-graph replay", "launches_per_replay": int(per_fwd)},
        "batched_forward_backward": {"ms": round(fb_ms, 4), "gflops": round(value / ws, 3),
                                     "launches_per_replay": int(per_fb)},
        "roofline": {"bound": "hbm", "kernel": "whole batched forward (one graph replay)",
                     "achieved": round(num_bytes / (fwd_ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(num_bytes / (fwd_ms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
                     "bytes_per_launch": num_bytes,
                     "bytes_formula": "16(rows+1) + 24 nnz_A + 8 products + 8 nnz_C over all instances",
                     "traffic": None},
        "e2e": None, "gpu_launches": int(per_fb * steps), "clocks": clk.summary(), "cpu_baseline": cpu,
        "verified": cpu.pop("verified") if cpu else None}
    del bp, gf, gfb, As, Bs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def run_batched(args, ws, rank, local, desc):
    import torch
    torch.cuda.set_device(local)
    dist = _dist_setup(ws, local)
    rec = batched_record(args, ws, rank, local, dist)
    if rank == 0:
        print(json.dumps(rec), flush=True)
    if dist:
        dist.destroy_process_group()
    if rec.get("verified") is not None and not rec["verified"]["ok"]:
        sys.exit(1)


def run_msbfs(args, ws, rank, local, desc):
    """Multi-source BFS to completion; products = the multiplications of the
    boolean products (sum over reached (vertex, source) of the degree)."""
    import numpy as np
    import torch
    import synth
    from paper_2408_11988_gb300 import DeviceCSR
    from paper_2408_11988_gb300 import _native as N
    from paper_2408_11988_gb300.msbfs import msbfs
    dist = _dist_setup(ws, local)
    A, src = synth.msbfs_graph(seed=synth.BASE_SEED + 2 + 1000 * rank)
    Ad = DeviceCSR.from_host(A, with_values=False)
    s = torch.as_tensor(src)
    par = args.workload == "msbfs-parents-s20"
    for _ in range(args.warmup):
        r = msbfs(Ad, s, parents=par)
    torch.cuda.synchronize()
    deg = np.diff(A.rowptr)
    lev = r.levels.cpu().numpy()
    products = int((deg[:, None] * (lev >= 0)).sum())
    l0 = N.lib().ts_kernel_launches()
    with ClockSampler(local) as clk:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            r = msbfs(Ad, s, parents=par)
        b.record()
        torch.cuda.synchronize()
    launches = N.lib().ts_kernel_launches() - l0
    ms = _max_over_ranks(dist, a.elapsed_time(b) / args.steps)
    if rank == 0:
        print(json.dumps({
            "metric": "multi-source BFS (sel2nd, min) products/s" if par else "multi-source BFS boolean products/s",
            "value": round(products * ws / (ms * 1e-3), 1),
            "unit": "products/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": A.nrows, "nnz_A": A.nnz,
                       "sources": len(src), "levels": r.products, "frontier_nnz": r.frontier_nnz,
                       "products": products, "parallelism": f"replicas x{ws}"},
            "levels_per_s": round(r.products * ws / (ms * 1e-3), 1),
            "roofline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk.summary(),
            "cpu_baseline": None}), flush=True)
    if dist:
        dist.destroy_process_group()


def run_force2vec(args, ws, rank, local, desc):
    """One step = one epoch of the sparse Force2Vec training (every row once,
    minibatches of 65536 consecutive rows).  products = multiplications of
    the force products W * Z (per row: (degree + negatives) * k)."""
    import numpy as np
    import torch
    import synth
    from paper_2408_11988_gb300 import DeviceCSR
    from paper_2408_11988_gb300 import _native as N
    from paper_2408_11988_gb300.force2vec import Force2Vec
    dist = _dist_setup(ws, local)
    k, s, lr, batch = 26, 5, 0.02, 65536
    A, Z = synth.force2vec_inputs(seed=synth.BASE_SEED + 6 + 1000 * rank)
    n = A.nrows
    Ad, Zd = DeviceCSR.from_host(A, with_values=False), DeviceCSR.from_host(Z)
    neg = torch.as_tensor(synth.negatives(n, s, n, synth.BASE_SEED + 7 + 1000 * rank), device="cuda")
    f = Force2Vec(Ad, Zd, k, negatives=s, lr=lr, batch=batch)
    products = int((np.diff(A.rowptr) + s).sum()) * k
    for _ in range(args.warmup):
        f.epoch(neg)
    torch.cuda.synchronize()
    l0 = N.lib().ts_kernel_launches()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            mb = f.epoch(neg)
        b.record()
        torch.cuda.synchronize()
    launches = N.lib().ts_kernel_launches() - l0
    ms = _max_over_ranks(dist, a.elapsed_time(b) / args.steps)
    if rank == 0:
        print(json.dumps({
            "metric": "sparse Force2Vec embedding rows/s", "value": round(n * ws / (ms * 1e-3), 1),
            "unit": "rows/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "force2vec-s20", "description": desc, "n": n, "nnz_A": A.nnz, "d": Z.ncols,
                       "k": k, "negatives": s, "lr": lr, "batch": batch, "minibatches": mb,
                       "products": products, "parallelism": f"replicas x{ws}"},
            "force_product_gflops": round(2.0 * products * ws / (ms * 1e-3) / 1e9, 3),
            "ms_per_minibatch": round(ms / mb, 4),
            "roofline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk.summary(),
            "cpu_baseline": None}), flush=True)
    if dist:
        dist.destroy_process_group()


def _reference_other(args, ws, desc):
    """Reference arm (the FP64 oracle, one host core) for the BFS, Force2Vec
    and batched workloads, on bounded samples: 4 of the 128 BFS sources, a
    4096-row Force2Vec minibatch, the largest batched instance."""
    import oracle
    import synth
    import numpy as np
    vals, sample, unit, metric = [], "", "", ""
    for it in range(args.warmup + args.steps):
        if args.workload in ("msbfs-s20", "msbfs-parents-s20"):
            A, src = synth.msbfs_graph()
            src = src[:4]
            t0 = time.perf_counter()
            if args.workload == "msbfs-s20":
                lev, _, _ = oracle.msbfs(A, src)
            else:
                lev, _, _, _ = oracle.msbfs_parents(A, src)
            t = time.perf_counter() - t0
            deg = np.diff(A.rowptr)
            v = float((deg[:, None] * (lev >= 0)).sum()) / t
            unit = "products/s"
            metric = ("multi-source BFS (sel2nd, min) products/s" if args.workload == "msbfs-parents-s20"
                      else "multi-source BFS boolean products/s")
            sample = f"4 of the 128 sources of the R-MAT scale-20 graph, {t:.1f} s single-threaded"
        elif args.workload == "force2vec-s20":
            A, Z = synth.force2vec_inputs()
            b, s = 4096, 5
            neg = synth.negatives(b, s, A.nrows, synth.BASE_SEED + 7)
            t0 = time.perf_counter()
            oracle.f2v_step(A, Z, 0, b, neg, s, 0.02, 26)
            t = time.perf_counter() - t0
            v, unit, metric = b / t, "rows/s", "sparse Force2Vec embedding rows/s"
            sample = f"one minibatch of {b} rows of the scale-20 graph, {t:.1f} s single-threaded"
        else:  # batched-64: the largest instance, forward + backward
            inst = synth.batched_instances()
            A, B = max(inst, key=lambda ab: ab[0].nnz)
            r = cpu_baseline(A, B, True, target_s=6.0)
            v, unit, metric = r["value"], "GFLOP/s", "TS-SpGEMM GFLOP/s (batched forward + backward, plus-times)"
            sample = "largest instance: " + r["sample"]
        if it >= args.warmup:
            vals.append(v)
    v = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": round(v, 4), "unit": unit, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc},
        "cpu_baseline": {"value": round(v, 4), "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": round(v, 4), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def run_reference(args, ws, rank, desc, want_bwd):
    """The oracle (FP64, one host core) timed on a bounded sample per step."""
    if rank != 0:
        return
    if args.workload in ("msbfs-s20", "msbfs-parents-s20", "force2vec-s20", "batched-64"):
        return _reference_other(args, ws, desc)
    A, B = make_inputs(args.workload, scale=args.scale, d=args.d, density=args.density)
    F = int(products_per_row(A, B).sum())
    import oracle  # noqa: F401
    for _ in range(args.warmup):
        cpu_baseline(A, B, want_bwd, target_s=2.0)
    vals = []
    sample = None
    for _ in range(args.steps):
        r = cpu_baseline(A, B, want_bwd, target_s=6.0)
        vals.append(r["value"])
        sample = r["sample"]
    v = statistics.mean(vals)
    line = {
        "impl": "reference",
        "metric": "TS-SpGEMM GFLOP/s (forward + backward, plus-times)" if want_bwd
        else "TS-SpGEMM GFLOP/s (forward, plus-times)",
        "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": product_config(args.workload + _override_tag(args), _override_desc(args, desc), A, B, F, ws),
        "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
