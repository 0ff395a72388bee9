#!/usr/bin/env python3
"""ChFSI filter benchmark on one GB300 (or N replicas under torchrun).

One step = one pass of the hot path over the resident synthetic workload:
  Lanczos bounds (20 steps)  ->  FP64 Chebyshev filter (CSR, degree m)
  ->  CholQR2 + Rayleigh-Ritz (projection, eigensolve, rotation).
Default workload: 40^3 grid, w = 3 (19,248,832 nnz), 1024 states, m = 20.

Prints ONE JSON line (rank 0).  `value` is the step's algorithmic GFLOP/s
(Lanczos + filter + closure GEMMs; the n x n eigensolve is not counted), with the
per-phase numbers, the roofline of the dominant kernel (the fused FP64 CSR step,
bound by the DFMA pipe), the oracle's CPU time on a bounded sample, an end-to-end
number through the public API with host buffers, and the SM clocks seen.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import chfsi_workloads as W  # noqa: E402

METRIC = "ChFSI filter GFLOP/s & % of roofline, FP64 vs mixed precision at stated error"
SLAB_STATES = 512   # column-slab width of a CSR filter (the library's kSlab)
# FP64 DFMA pipe of the whole GPU, measured with a register-resident FMA loop
# (152 SMs x 8 independent chains x 2048 iterations, CUDA events): 1.194-1.201
# TFLOP/s.  The nominal figure is 1.25 TFLOP/s.
FP64_PEAK_GFLOPS = 1200.0
# FP32 FFMA pipe, same method: 74.8-75.1 TFLOP/s.
FP32_PEAK_GFLOPS = 75000.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="g40_w3_n1024_m20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-cols", type=int, default=64)
    ap.add_argument("--cols", type=int, default=0, help="override the workload's state count n")
    ap.add_argument("--filter-only", action="store_true",
                    help="set up, run one FP64 filter (m launches of the CSR step) and exit: a profiling case")
    ap.add_argument("--schedule", default="f64", help="filter-only schedule: f64 | f32:L | bf16:L | f32x2:L")
    ap.add_argument("--layout", default="csr", choices=["csr", "bsr", "hybrid"], help="filter-only operator layout")
    ap.add_argument("--closure-only", action="store_true",
                    help="set up, run one CholQR2 + Rayleigh-Ritz on X and exit: a profiling case")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32x2"], help="closure-only product precision")
    ap.add_argument("--compact", action="store_true",
                    help="largest workloads: variants limited to the FP64 filter, the FP32 prefix and the "
                         "two-float filter (each with its Ritz error) and the two-float step; no adjoint, no BSR")
    ap.add_argument("--quick", action="store_true",
                    help="large one-off workloads: variants timed once without warm-up, no BSR-FP64 variant, "
                         "no end-to-end leg")
    return ap.parse_args()


# ---------------------------------------------------------------- FLOP model (algorithmic)


def filter_flops(nnz, N, n, m):
    """2 nnz n per product; the first step adds 3 N n (shift, scale), later steps 5 N n."""
    return m * 2.0 * nnz * n + 3.0 * N * n + (m - 1) * 5.0 * N * n


def lanczos_flops(nnz, N, k):
    f = 0.0
    for j in range(k):
        f += 2.0 * nnz + 2 * N + 4 * N + 2.0 * N * (j + 1) * 2 + 2 * N + N
    return f


def closure_flops(nnz, N, n, passes):
    """Gram N n^2 and triangular solve N n^2 per CholQR pass, H X_F (2 nnz n),
    projection N n^2 (H_F is symmetric: one triangle, like the Gram), rotation
    2 N n^2 (eigensolve not counted)."""
    return passes * 2.0 * N * n * n + 2.0 * nnz * n + 1.0 * N * n * n + 2.0 * N * n * n


def hbm_peak_gbs():
    """(GB/s, source): the measured copy bandwidth of the GB300s, else the
    earlier single measurement used as the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                continue
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if _isnum(r[1])]
        smax = [float(r[2]) for r in rows if _isnum(r[2])]
        power = [float(r[3]) for r in rows if _isnum(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [x for x, p in zip(sm, power)] if sm else []
        return {"sm_mhz": float(np.median(load)) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": reasons}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ---------------------------------------------------------------- traffic from the committed ncu summary


def _kernel_source_sha():
    p = os.path.join(ROOT, "paper_2110_15853_gb300", "csrc", "filter_csr.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def committed_traffic(workload):
    """dram bytes per filter step (all column slabs) of the FP64 CSR step from
    profiles/, if the kernel source is unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", f"csr_step_f64_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m1 = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m2 = re.search(r"dram_bytes_per_step:\s*([0-9.eE+]+)", text)
    if not m1 or not m2 or m1.group(1) != _kernel_source_sha():
        return None
    return float(m2.group(1))


# ---------------------------------------------------------------- replicas (N > 1)


def replica_max_ms(local_ms: float, device) -> float:
    """Max of the timed region over all ranks (the job ends when the slowest rank
    does); identity without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(step_flops: float, world: int, ms_step: float) -> float:
    """Whole-job GFLOP/s: every rank filters its own replica (weak scaling), so
    the job's work is world x the per-rank step, over the slowest rank's time."""
    return step_flops * world / (ms_step * 1e-3) / 1e9


# ---------------------------------------------------------------- workload setup


def setup_workload(name, cols=0):
    wl = W.workload(name)
    if cols:
        import dataclasses
        wl = dataclasses.replace(wl, n=int(cols))
    H = W.csr_grid(wl.g, wl.w, wl.s, wl.seed, core_frac=wl.core_frac, core_shift=wl.core_shift)
    X = W.start_block(H["N"], wl.n, wl.seed)
    v0 = W.lanczos_start(H["N"], wl.seed)
    return wl, H, X, v0


def cpu_baseline(H, X, v0, wl, ncols, m):
    """The oracle as it stands on a bounded sample: all m filter steps on `ncols`
    of the n columns at full N (columns are independent)."""
    import oracle
    oracle.build()
    a, b, a0 = oracle.lanczos_bounds(H, v0, 20, wl.n)
    cols = W.column_subset(wl.n, ncols, wl.seed)
    Xs = np.ascontiguousarray(X[:, cols])
    t0 = time.perf_counter()
    oracle.filter(H, Xs, m, a, b, a0)
    dt = time.perf_counter() - t0
    fl = filter_flops(H["nnz"], H["N"], ncols, m)
    return {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 filter, all {m} steps, {ncols} of {wl.n} columns at full N={H['N']} "
                      f"({dt:.1f} s; filter only, closure not sampled)",
            "seconds": dt}


# ---------------------------------------------------------------- reference arm (the oracle)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, H, X, v0 = setup_workload(args.workload)
    import oracle
    oracle.build()
    a, b, a0 = oracle.lanczos_bounds(H, v0, 20, wl.n)
    ncols = args.cpu_cols
    cols = W.column_subset(wl.n, ncols, wl.seed)
    Xs = np.ascontiguousarray(X[:, cols])
    for _ in range(args.warmup):
        oracle.filter(H, Xs, 1, a, b, a0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.filter(H, Xs, wl.m, a, b, a0)
        times.append(time.perf_counter() - t0)
    fl = filter_flops(H["nnz"], H["N"], ncols, wl.m)
    t = float(np.median(times))
    val = fl / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "N": H["N"], "n": wl.n, "m": wl.m, "nnz": H["nnz"], "layout": "csr",
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"FP64 oracle filter, all {wl.m} steps on {ncols} of {wl.n} columns, full N "
                                   f"(warm-up steps use m=1)"},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2110_15853_gb300 as P
    from paper_2110_15853_gb300 import build as pbuild
    if rank == 0 or world == 1:
        pbuild.build()
    if world > 1:
        dist.barrier()
    lib = P.load()

    wl, H, X, v0 = setup_workload(args.workload, args.cols)
    N, n, m, nnz = H["N"], wl.n, wl.m, H["nnz"]
    if args.filter_only:
        return run_filter_only(P, torch, dev, wl, H, X, v0, args)
    if args.closure_only:
        Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
        Xd = torch.as_tensor(X).to(dev)
        ws = P.Workspace(dev)
        P.rayleigh_ritz(Hd, Xd, 2, precision=args.precision, workspace=ws)   # warm-up (workspace, solver setup)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ritz, _ = P.rayleigh_ritz(Hd, Xd, 2, precision=args.precision, workspace=ws)
        e1.record()
        torch.cuda.synchronize(dev)
        print(json.dumps({"closure_only": True, "workload": wl.name, "n": n, "precision": args.precision,
                          "ms": e0.elapsed_time(e1), "finite": bool(torch.isfinite(ritz).all().item())}))
        return 0
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    Xd = torch.as_tensor(X).to(dev)
    v0d = torch.as_tensor(v0).to(dev)
    Yd = torch.empty_like(Xd)
    psi = torch.empty_like(Xd)
    ritz = torch.empty(n, dtype=torch.float64, device=dev)
    wsl, wsf, wsr = P.Workspace(dev), P.Workspace(dev), P.Workspace(dev)
    wsf.get(P.filter_workspace_bytes(Hd, n, m))
    wsr.get(P.rayleigh_ritz_workspace_bytes(Hd, n, 2))
    stream = torch.cuda.current_stream(dev)

    def step(ev=None, X_in=None, v0_in=None, psi_out=None, ritz_out=None):
        X_in = Xd if X_in is None else X_in
        if ev:
            ev[0].record(stream)
        a, b, a0 = P.lanczos_bounds(Hd, v0d if v0_in is None else v0_in, 20, n, workspace=wsl)
        if ev:
            ev[1].record(stream)
        P.filter(Hd, X_in, m, a, b, a0, out=Yd, workspace=wsf)
        if ev:
            ev[2].record(stream)
        P.rayleigh_ritz(Hd, Yd, 2, psi=psi if psi_out is None else psi_out,
                        ritz=ritz if ritz_out is None else ritz_out, workspace=wsr)
        if ev:
            ev[3].record(stream)
        return a, b, a0

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    flops_l = lanczos_flops(nnz, N, 20)
    flops_f = filter_flops(nnz, N, n, m)
    flops_c = closure_flops(nnz, N, n, 2)
    step_flops = flops_l + flops_f + flops_c

    clocks = ClockSampler(local)
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = lib.chfsi_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        bounds = step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = lib.chfsi_kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = replica_max_ms(t_start.elapsed_time(t_end), dev)
    ms_step = total_ms / args.steps
    lan_ms = float(np.median([e[0].elapsed_time(e[1]) for e in evs]))
    fil_ms = float(np.median([e[1].elapsed_time(e[2]) for e in evs]))
    rr_ms = float(np.median([e[2].elapsed_time(e[3]) for e in evs]))
    value = replica_throughput(step_flops, world, ms_step)

    # roofline of the dominant kernel: the fused FP64 CSR step.  The unit is one filter
    # step over all n states: the library runs a CSR filter in column slabs of 512 states
    # (all m steps per slab), so a step is one launch per slab and H is read once per slab.
    slabs = -(-n // SLAB_STATES)
    step_ms = fil_ms / m
    achieved = (flops_f / m) / (step_ms * 1e-3) / 1e9
    traffic = committed_traffic(wl.name)
    roofline = {"bound": "alu", "pipe": "fp64 dfma", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                "kernel": "csr_step_kernel<double> (fused SpMM + recurrence)",
                "unit_of_work": f"one filter step over all {n} states ({slabs} column-slab launches)",
                "peak_source": "measured FP64 FMA loop on this GB300 (not in MEASURED_PEAKS.json)",
                "hbm_bytes_algorithmic": 24.0 * N * n + slabs * (12.0 * nnz + 8.0 * (N + 1))}

    # End to end through the public API with host buffers: every step copies its X (and
    # the Lanczos start vector) from pinned host memory and reads its Psi and Ritz values
    # back.  The copies run on a second stream with double-buffered device blocks, so the
    # input of step k+1 and the result of step k-1 move while step k computes.
    e2e = None
    if not (args.quick or args.compact):
        Xh = torch.empty((N, n), dtype=torch.float64).pin_memory()
        Xh.copy_(torch.as_tensor(X))
        v0h = torch.as_tensor(v0).pin_memory()
        psih = torch.empty((N, n), dtype=torch.float64).pin_memory()
        ritzh = torch.empty(n, dtype=torch.float64).pin_memory()
        copy_stream = torch.cuda.Stream(dev)
        bufs = [(Xd, v0d, psi, ritz),
                (torch.empty_like(Xd), torch.empty_like(v0d), torch.empty_like(psi), torch.empty_like(ritz))]
        ev = lambda: torch.cuda.Event()  # noqa: E731
        h2d_done, step_done, d2h_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]

        def h2d(slot):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(d2h_done[slot])        # slot's previous result has been read
                bufs[slot][0].copy_(Xh, non_blocking=True)
                bufs[slot][1].copy_(v0h, non_blocking=True)
                h2d_done[slot].record(copy_stream)

        def d2h(slot):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(step_done[slot])
                psih.copy_(bufs[slot][2], non_blocking=True)
                ritzh.copy_(bufs[slot][3], non_blocking=True)
                d2h_done[slot].record(copy_stream)

        def e2e_run(steps):
            copy_stream.wait_stream(stream)                    # nothing moves before the timed region opens
            for slot in (0, 1):
                d2h_done[slot].record(copy_stream)
            h2d(0)
            for k in range(steps):
                cur, nxt = k % 2, (k + 1) % 2
                if k + 1 < steps:
                    h2d(nxt)
                stream.wait_event(h2d_done[cur])
                Xb, vb, pb, rb = bufs[cur]
                step(X_in=Xb, v0_in=vb, psi_out=pb, ritz_out=rb)
                step_done[cur].record(stream)
                d2h(cur)
            stream.wait_stream(copy_stream)

        e2e_run(2)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_run(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = e0.elapsed_time(e1) / args.steps
        e2e = {"value": step_flops * world / (e2e_ms * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(Xh.numel() * 8 + v0h.numel() * 8),
               "d2h_bytes_per_step": int(psih.numel() * 8 + ritzh.numel() * 8),
               "copies": "pinned host <-> device on a second stream, double-buffered, overlapped with compute"}
        del Xh, psih, bufs

    variants = {}
    if not args.no_variants and rank == 0:
        variants = measure_variants(P, torch, dev, stream, wl, H, Hd, Xd, bounds, quick=args.quick or args.compact,
                                    compact=args.compact)
        v2 = variants.get("step_f32x2_filter_and_closure")
        if v2 and v2.get("ms"):
            v2["speedup_vs_f64_step"] = ms_step / v2["ms"]
            v2["gflops"] = step_flops / (v2["ms"] * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(H, X, v0, wl, args.cpu_cols, m)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "grid": f"{wl.g}^3", "w": wl.w, "N": N, "n": n, "m": m, "nnz": nnz,
                       "layout": "csr", "step": "lanczos(20) + filter(m, FP64) + CholQR2 + Rayleigh-Ritz",
                       "l2": "inputs larger than L2 (each N x n block is %.0f MB)" % (N * n * 8 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single"},
            "phases": {"lanczos_ms": lan_ms, "filter_ms": fil_ms, "closure_ms": rr_ms,
                       "filter_gflops": flops_f / (fil_ms * 1e-3) / 1e9,
                       "closure_gflops": flops_c / (rr_ms * 1e-3) / 1e9,
                       "step_gflop": step_flops / 1e9},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(launches),
            "mixed_precision": mixed_summary(variants, fil_ms),
            "variants": variants,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def mixed_summary(variants, f64_filter_ms):
    """The metric's 'FP64 vs mixed precision at stated error' in one place: each
    measured low-precision filter schedule against the FP64 filter of the timed step,
    with its Ritz-value error against the all-FP64 run and whether it meets the 1e-8
    target.  Details stay in `variants`."""
    out = {"target_ritz_rel_err": 1e-8, "f64_filter_ms": f64_filter_ms, "schedules": {}}
    for k, v in variants.items():
        if not k.startswith(("filter_csr_", "filter_hybrid_")) or "ritz_max_rel_err_vs_f64" not in v:
            continue
        err = v["ritz_max_rel_err_vs_f64"]
        out["schedules"][k] = {"ms": v["ms"], "speedup_vs_f64_filter": f64_filter_ms / v["ms"],
                               "ritz_max_rel_err_vs_f64": err, "meets_target": bool(err <= 1e-8)}
    step = variants.get("step_f32x2_filter_and_closure")
    if step and step.get("ms"):
        out["whole_step_two_float"] = {"ms": step["ms"], "speedup_vs_f64_step": step.get("speedup_vs_f64_step"),
                                       "ritz_max_rel_err_vs_f64": step.get("ritz_max_rel_err_vs_f64")}
    return out or None


def run_filter_only(P, torch, dev, wl, H, X, v0, args):
    """One filter call on the resident workload (a small, self-ending ncu case)."""
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    Xd = torch.as_tensor(X).to(dev)
    a, b, a0 = P.lanczos_bounds(Hd, torch.as_tensor(v0).to(dev), 20, wl.n)
    if args.layout != "csr":
        B = W.bsr_from_csr(H, wl.g)
        Bd = P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device=dev)
        Hp = W.permute_csr(H, B["perm"])
        Hd = Bd if args.layout == "bsr" else P.HybridMatrix(
            P.CsrMatrix.from_arrays(Hp["row_ptr"], Hp["col"], Hp["val"], device=dev), Bd)
        Xd = Xd[torch.as_tensor(B["perm"]).to(dev)].contiguous()
    sched = None
    if args.schedule != "f64":
        low, L = args.schedule.split(":")
        sched = P.mixed_schedule(wl.m, int(L), low)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Y = P.filter(Hd, Xd, wl.m, a, b, a0, schedule=sched)
    e1.record()
    torch.cuda.synchronize(dev)
    print(json.dumps({"filter_only": True, "workload": wl.name, "n": wl.n, "schedule": args.schedule,
                      "layout": args.layout,
                      "ms": e0.elapsed_time(e1), "finite": bool(torch.isfinite(Y).all().item())}))
    return 0


class _Skipped(Exception):
    """A variant group left out on purpose (reported as skipped)."""


def measure_variants(P, torch, dev, stream, wl, H, Hd, Xd, bounds, quick=False, compact=False):
    """Filter-only timings of the other layouts / schedules on the same workload
    (outside the main timed region), each with its error against the FP64 CSR run."""
    a, b, a0 = bounds
    N, n, m, nnz = H["N"], wl.n, wl.m, H["nnz"]
    out = {}

    def timeit(fn, reps=2):
        if quick:
            reps = 1
        else:
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    fl = filter_flops(nnz, N, n, m)
    Yref = torch.empty_like(Xd)
    ws = P.Workspace(dev)
    t = timeit(lambda: P.filter(Hd, Xd, m, a, b, a0, out=Yref, workspace=ws))
    out["filter_csr_f64"] = {"ms": t, "gflops": fl / (t * 1e-3) / 1e9}
    rr_ws = P.Workspace(dev)
    theta_ref, _ = P.rayleigh_ritz(Hd, Yref, 2, workspace=rr_ws)
    theta_ref = theta_ref.cpu().numpy()

    schedules = (("f32", m - 4), ("f32x2", m)) if compact else (("f32", m - 4), ("bf16", m - 4), ("f32x2", m),
                                                                  ("f32x2", m - 4))
    for low, L in schedules:
        Ym = torch.empty_like(Xd)
        sched = P.mixed_schedule(m, L, low)
        try:
            t = timeit(lambda: P.filter(Hd, Xd, m, a, b, a0, schedule=sched, out=Ym, workspace=ws))
        except P.ChfsiError as e:
            out[f"filter_csr_{low}x{L}_f64x{m - L}"] = {"error": str(e)}
            continue
        th, _ = P.rayleigh_ritz(Hd, Ym, 2, workspace=rr_ws)
        rel = float(np.max(np.abs(th.cpu().numpy() - theta_ref)) / np.max(np.abs(theta_ref)))
        yerr = float(torch.linalg.norm(Ym - Yref) / torch.linalg.norm(Yref))
        out[f"filter_csr_{low}x{L}_f64x{m - L}"] = {
            "ms": t, "gflops": fl / (t * 1e-3) / 1e9, "speedup_vs_f64": out["filter_csr_f64"]["ms"] / t,
            "ritz_max_rel_err_vs_f64": rel, "y_rel_fro_err_vs_f64": yerr}
        del Ym
    # adjoint (reverse sweep with sqrt(m) checkpoints), FP64 and two-float; algorithmic
    # work m (4 nnz n + 5 N n) plus one forward replay
    try:
        if compact:
            raise _Skipped("--compact")
        wts = torch.as_tensor(W.loss_weights(N, wl.seed)).to(dev)
        G = 2.0 * wts[:, None] * Yref
        adj_fl = m * (4.0 * nnz * n + 5.0 * N * n) + fl
        bw_ws = P.Workspace(dev)
        t = timeit(lambda: P.filter_backward(Hd, Xd, G, m, a, b, a0, workspace=bw_ws), reps=1)
        dX64, dH64 = P.filter_backward(Hd, Xd, G, m, a, b, a0, workspace=bw_ws)
        out["adjoint_f64"] = {"ms": t, "gflops": adj_fl / (t * 1e-3) / 1e9}
        t2 = timeit(lambda: P.filter_backward(Hd, Xd, G, m, a, b, a0, workspace=bw_ws, precision="f32x2"), reps=1)
        dX2, dH2 = P.filter_backward(Hd, Xd, G, m, a, b, a0, workspace=bw_ws, precision="f32x2")
        out["adjoint_f32x2"] = {
            "ms": t2, "gflops": adj_fl / (t2 * 1e-3) / 1e9, "speedup_vs_f64_adjoint": t / t2,
            "speedup_vs_f64_forward_filter": out["filter_csr_f64"]["ms"] / t2,
            "dX_rel_err_vs_f64": float(torch.linalg.norm(dX2 - dX64) / torch.linalg.norm(dX64)),
            "dH_rel_err_vs_f64": float(torch.linalg.norm(dH2 - dH64) / torch.linalg.norm(dH64))}
        del G, dX64, dH64, dX2, dH2, bw_ws
    except _Skipped as e:
        out["adjoint"] = {"skipped": str(e)}
    except Exception as e:  # noqa: BLE001 - report, do not hide
        out["adjoint_error"] = repr(e)

    # the whole step with the FP64-accurate two-float filter and closure products
    try:
        Ys = torch.empty_like(Xd)
        rr2_ws = P.Workspace(dev)
        wsl2 = P.Workspace(dev)
        v0d = torch.as_tensor(W.lanczos_start(N, wl.seed)).to(dev)
        sch2 = ["f32x2"] * m

        def step2():
            a_, b_, a0_ = P.lanczos_bounds(Hd, v0d, 20, n, workspace=wsl2)
            P.filter(Hd, Xd, m, a_, b_, a0_, schedule=sch2, out=Ys, workspace=ws)
            return P.rayleigh_ritz(Hd, Ys, 2, workspace=rr2_ws, precision="f32x2")

        t = timeit(step2)
        th2, _ = step2()
        t_rr = timeit(lambda: P.rayleigh_ritz(Hd, Yref, 2, workspace=rr2_ws, precision="f32x2"))
        th_rr, _ = P.rayleigh_ritz(Hd, Yref, 2, workspace=rr2_ws, precision="f32x2")
        out["step_f32x2_filter_and_closure"] = {
            "ms": t, "speedup_vs_f64_step": None,
            "ritz_max_rel_err_vs_f64": float(np.max(np.abs(th2.cpu().numpy() - theta_ref)) /
                                             np.max(np.abs(theta_ref)))}
        out["closure_f32x2"] = {"ms": t_rr, "ritz_max_rel_err_vs_f64_closure": float(
            np.max(np.abs(th_rr.cpu().numpy() - theta_ref)) / np.max(np.abs(theta_ref)))}
        del Ys
    except Exception as e:  # noqa: BLE001 - report, do not hide
        out["step_f32x2_error"] = repr(e)

    # BSR layout of the same operator, and the hybrid (blocked CSR + BSR) operator
    try:
        if compact:
            raise _Skipped("--compact")
        B = W.bsr_from_csr(H, wl.g)
        Bd = P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device=dev)
        Hpd = P.CsrMatrix.from_arrays(**{k: v for k, v in W.permute_csr(H, B["perm"]).items()
                                         if k in ("row_ptr", "col", "val")}, device=dev)
        Hy = P.HybridMatrix(Hpd, Bd)
        perm = torch.as_tensor(B["perm"]).to(dev)
        Xp = Xd[perm].contiguous()
        Yb = torch.empty_like(Xp)
        Yback = torch.empty_like(Yb)

        def err_vs_ref():
            Yback[perm] = Yb
            return float(torch.linalg.norm(Yback - Yref) / torch.linalg.norm(Yref))

        def ritz_err():
            Yback[perm] = Yb
            th, _ = P.rayleigh_ritz(Hd, Yback, 2, workspace=rr_ws)
            return float(np.max(np.abs(th.cpu().numpy() - theta_ref)) / np.max(np.abs(theta_ref)))

        if quick:
            t = None
        else:
            t = timeit(lambda: P.filter(Bd, Xp, m, a, b, a0, out=Yb, workspace=ws), reps=1)
        out["filter_bsr_f64"] = {"skipped": "--quick"} if t is None else {"ms": t, "gflops": fl / (t * 1e-3) / 1e9,
                                 "executed_gflop": m * 2.0 * B["n_blocks"] * 64 * 64 * n / 1e9,
                                 "y_rel_fro_err_vs_csr": err_vs_ref()}
        t = timeit(lambda: P.filter(Hy, Xp, m, a, b, a0, out=Yb, workspace=ws))
        out["filter_csr_blocked_order_f64"] = {"ms": t, "gflops": fl / (t * 1e-3) / 1e9,
                                               "y_rel_fro_err_vs_csr": err_vs_ref()}
        sched = ["bf16"] * m
        t = timeit(lambda: P.filter(Bd, Xp, m, a, b, a0, schedule=sched, out=Yb, workspace=ws))
        out["filter_bsr_bf16_tc_all_steps"] = {
            "ms": t, "ms_per_step": t / m, "gflops": fl / (t * 1e-3) / 1e9,
            # products of the stored dense blocks (the step also multiplies the zero block that
            # stands in for a block missing from one row of a block-row pair)
            "stored_block_tflops": m * 2.0 * B["n_blocks"] * 64 * 64 * n / (t * 1e-3) / 1e12,
            "y_rel_fro_err_vs_f64": err_vs_ref()}
        # compulsory bytes of one BF16 step: Ysh^T in (2 N n), Y_cur and Y_prev (8 N n), the BF16
        # blocks (8 KB each), Y_out in FP32 and its BF16 copy (6 N n); the per-step time also
        # carries the call's one-off conversions, so this fraction is a lower bound for the kernel
        step_bytes = 16.0 * N * n + 8192.0 * B["n_blocks"]
        hbm = hbm_peak_gbs()
        out["filter_bsr_bf16_tc_all_steps"].update({
            "compulsory_bytes_per_step": step_bytes,
            "hbm_gbs_per_step": step_bytes / (t / m * 1e-3) / 1e9,
            "hbm_frac": step_bytes / (t / m * 1e-3) / 1e9 / hbm[0], "hbm_peak_gbs": hbm[0],
            "hbm_peak_source": hbm[1]})
        for low, L in (("bf16", m - 4), ("f32", m - 4), ("f32", m // 2)):
            sched = P.mixed_schedule(m, L, low)
            t = timeit(lambda: P.filter(Hy, Xp, m, a, b, a0, schedule=sched, out=Yb, workspace=ws))
            out[f"filter_hybrid_{low}x{L}_f64x{m - L}"] = {
                "ms": t, "gflops": fl / (t * 1e-3) / 1e9, "speedup_vs_f64": out["filter_csr_f64"]["ms"] / t,
                "y_rel_fro_err_vs_f64": err_vs_ref(), "ritz_max_rel_err_vs_f64": ritz_err()}
        del Bd, Xp, Yb, Yback, Hpd, Hy
    except _Skipped as e:
        out["bsr_variants"] = {"skipped": str(e)}
    except Exception as e:  # noqa: BLE001 - report, do not hide
        out["bsr_variants_error"] = repr(e)
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
