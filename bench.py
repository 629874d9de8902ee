"""Benchmark of the stabilised cell-vertex WENO DG stage on one GB300 (or N replicas).

Workload: the 2D KPP problem, f(u) = (sin u, cos u) on [-2,2]^2 periodic, 256 x 256
quadrilaterals, seeded circle datum (radius U(0.5, 1.0)), DG Q1, Q2 and Q3, FP32.
One benchmark step = one SSP-RK3 step (three stages (a)-(e)) of each of the three
degrees, each captured once in a CUDA graph.  The metric is DOF-updates per second
per RK stage: 3 * sum_p ndof_p / step time.  L2 is flushed (a 512 MB write) between
timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the same workload (bounded sample per
step); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage, plain FP32 vs batched/surrogate, at stated L1 vs FP64"
UNIT = "DOF-updates/s"
N_CELLS = 256
DEGREES = (1, 2, 3)
WORKLOAD = "KPP 2D, f=(sin u, cos u), [-2,2]^2 periodic, 256x256 quads, DG Q1+Q2+Q3 (one SSP-RK3 step each), FP32"
SEED = 0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cfl_dt(p: int, n: int = N_CELLS) -> float:
    """CFL time step of the workload: dt = (0.3/(2p+1)) dx / (d lambda), lambda = 1."""
    return (0.3 / (2 * p + 1)) * (4.0 / n) / 2.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per cell and stage, sum-factorised FMA counts of the method's steps for
# 2D scalar DG Q_p with n = p+1 (stage d only in troubled cells):
#   (a) 8n^3 + 4n^2, (b) 4n^2, (c) 8n^3 + 6n^4, (d) 2n^5, (e) 14n^3 + 20n^2.
def fma_per_cell(p: int, troubled_fraction: float) -> float:
    n = p + 1
    return (8 * n**3 + 4 * n**2) + 4 * n**2 + (8 * n**3 + 6 * n**4) + troubled_fraction * 2 * n**5 + (14 * n**3 + 20 * n**2)


def bytes_per_dof_stage() -> float:
    """Algorithmic HBM bytes per DOF and stage in FP32: read u^(s-1), write u^(s), and
    read u^n in stages 2 and 3: (8 + 12 + 12) / 3."""
    return 32.0 / 3.0


KERNEL_SOURCES = ["dg_scalar_kernel.cuh", "dg_scalar_launch.cuh", "dg_scalar_2d.cu"]


def kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2601_16911_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the kernel
    source has changed since those counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("traffic_bytes_per_launch")


def run_reference(args):
    """The FP64 CPU oracle on the workload's arithmetic, bounded sample per step."""
    import numpy as np

    from oracle import oracle as O
    from paper_2601_16911_gb300 import inputs as I

    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = 64
    problems = []
    for p in DEGREES:
        d, ic = I.kpp(SEED, n=n, degree=p)
        problems.append((d, O.project(d, *ic).astype(np.float32).astype(np.float64)))
    units = sum(3 * d["nx"] * d["ny"] * (d["degree"] + 1) ** 2 for d, _ in problems)

    def step():
        for d, u in problems:
            O.ssprk3(d, u, cfl_dt(d["degree"], n), 1)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = units * args.steps / dt
    sample = f"one SSP-RK3 step of each of DG Q1, Q2, Q3 on the same KPP problem at 64x64 cells per benchmark step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (plain C, single thread)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample():
    """Oracle timed on a bounded sample of the workload: one SSP-RK3 step of each degree
    on the KPP problem at 128x128 cells (same arithmetic per cell as 256x256)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2601_16911_gb300 import inputs as I

    n = 128
    work = []
    for p in DEGREES:
        d, ic = I.kpp(SEED, n=n, degree=p)
        work.append((d, O.project(d, *ic)))
    t0 = time.perf_counter()
    units = 0
    for d, u in work:
        O.ssprk3(d, u, cfl_dt(d["degree"], n), 1)
        units += 3 * d["nx"] * d["ny"] * (d["degree"] + 1) ** 2
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one SSP-RK3 step of each of DG Q1, Q2, Q3 at 128x128 cells ({dt:.1f} s, 1 thread)"}


def l1_vs_fp64():
    """Final-time L1 difference of the FP32 GPU path against the FP64 oracle on a
    reduced mesh of the workload (32x32, 10 SSP-RK3 steps per degree)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2601_16911_gb300 import cvweno as cv
    from paper_2601_16911_gb300 import inputs as I

    out = {}
    for p in DEGREES:
        d, ic = I.kpp(SEED, n=32, degree=p)
        u = O.project(d, *ic).astype(np.float32).astype(np.float64)
        dt = cfl_dt(p, 32)
        ref = O.ssprk3(d, u, dt, 10)
        mesh = cv.Mesh(d)
        ug = torch.from_numpy(u.astype(np.float32)).cuda()
        mesh.advance(ug, dt, 10)
        mesh.status_check()
        got = ug.cpu().numpy().astype(np.float64)
        mesh.close()
        out[f"Q{p}"] = O.l1_diff(d, got, ref) / O.l1_diff(d, ref, np.zeros_like(ref))
    return out


def run_gpu(args):
    import torch

    from paper_2601_16911_gb300 import build as B
    from paper_2601_16911_gb300 import cvweno as cv
    from paper_2601_16911_gb300 import inputs as I

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if B.is_stale():
        if rank == 0:
            B.build()
        if ws > 1:
            torch.distributed.barrier()
    cv.load()

    meshes, states, dts, graphs, inits = [], [], [], [], []
    for p in DEGREES:
        d, ic = I.kpp(SEED, n=N_CELLS, degree=p)
        m = cv.Mesh(d)
        u = m.project(*ic)
        torch.cuda.synchronize()
        meshes.append(m)
        inits.append(u.clone())
        states.append(u)
        dts.append(cfl_dt(p))
    units_per_step = sum(3 * m.ncells * m.ndof * m.nvars for m in meshes)
    launches_per_step = 3 * len(meshes)

    # capture one SSP-RK3 step per degree in a CUDA graph (3 stage launches each)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for m, u, dt in zip(meshes, states, dts):
            m.advance(u, dt, 1)  # warm the kernels before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for m, u, dt in zip(meshes, states, dts):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            m.advance(u, dt, 1)
        graphs.append(g)
    for u, u0 in zip(states, inits):
        u.copy_(u0)
    torch.cuda.synchronize()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(ev):
        for k, g in enumerate(graphs):
            ev[k].record(stream)
            g.replay()
        ev[len(graphs)].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        one_step([torch.cuda.Event(enable_timing=True) for _ in range(len(graphs) + 1)])
    torch.cuda.synchronize()
    for m in meshes:
        m.status_check()

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(len(graphs) + 1)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # evicts the previous step's data from L2 (outside the events)
        one_step(events[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    for m in meshes:
        m.status_check()

    per_degree = [[events[i][k].elapsed_time(events[i][k + 1]) for i in range(args.steps)] for k in range(len(graphs))]
    step_ms = sum(sum(x) for x in per_degree) / args.steps
    t_local = step_ms * args.steps / 1000.0
    if ws > 1:
        t = torch.tensor([t_local], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    value = units_per_step * args.steps * ws / t_max

    # ---- end to end through the public API: pinned host -> device, step, device -> host ----
    host_in = [u0.cpu().pin_memory() for u0 in inits]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    h2d = sum(h.numel() * h.element_size() for h in host_in)
    d2h = h2d
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        for m, u, dt, hi, ho in zip(meshes, states, dts, host_in, host_out):
            u.copy_(hi, non_blocking=True)
            cv.cvweno_advance(m, u, dt, 1)
            ho.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_t = time.perf_counter() - e0
    e2e_value = units_per_step * e2e_steps / e2e_t

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel: the fused stage kernel at Q3 ----
    import numpy as np

    kq3 = DEGREES.index(3)
    q3_launch_ms = statistics.mean(per_degree[kq3]) / 3.0
    mq3 = meshes[kq3]
    out = mq3.residual_ex(states[kq3])
    troubled_frac = float(out["troubled"].float().mean().item())
    flops_q3 = 2.0 * fma_per_cell(3, troubled_frac) * mq3.ncells
    peaks, peak_kind = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved_tflops = flops_q3 / (q3_launch_ms * 1e-3) / 1e12
    hbm_bytes_q3 = bytes_per_dof_stage() * mq3.ncells * mq3.ndof
    hbm_gbs = hbm_bytes_q3 / (q3_launch_ms * 1e-3) / 1e9
    traffic = measured_traffic("dg_scalar_stage_q3_kpp256")
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / alu_peak_tflops, "traffic": traffic,
                "kernel": "dg_scalar_stage<2,3,KPP,16,8> (fused stages a-e + RK combine)",
                "launch_ms": q3_launch_ms,
                "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz ({peak_kind} sm_max_mhz)",
                "flops_per_launch": flops_q3, "troubled_fraction": troubled_frac,
                "hbm_algorithmic_gbs": hbm_gbs, "hbm_frac_of_measured": hbm_gbs / peaks.get("hbm_gbs", 6800.0)}

    cpu = None
    l1 = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_sample()
        l1 = l1_vs_fp64()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": N_CELLS * N_CELLS, "degrees": list(DEGREES),
                       "dofs_per_step_stage": units_per_step // 3, "units_per_step": units_per_step,
                       "l2": "flushed (512 MB write) between timed steps, outside the timed events",
                       "graphs": "one CUDA graph per degree (3 stage launches)",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single GPU",
                       "per_degree_ms": {f"Q{p}": statistics.mean(per_degree[k]) for k, p in enumerate(DEGREES)},
                       "wall_s_timed_region": wall,
                       "l1_rel_vs_fp64_32x32_10steps": l1},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "api": "cvweno_advance via the ctypes binding, pinned host buffers"},
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    for m in meshes:
        m.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
