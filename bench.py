"""Benchmark of the hot path: Fig. 1's time step on a virtual 2x2x2 topology
of 512x256x256 FP64 subdomains (overlap 2, periodic in x) held in one GPU,
with the halo update hidden behind the inner block (widths (16, 2, 2)).

One step = boundary slabs + halo update of T2 (high-priority stream) and the
inner block (low-priority stream), then the swap; K steps run as CUDA-graph
launches. Metric: T_eff = 3*N*s / t_step (read T and Ci, write T2, N all
points of all subdomains, s bytes per element) in GB/s, and cell updates/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank runs its own replica of the workload on its
GPU (weak scaling, no data-path collective); the timing is the maximum over
ranks. `--impl reference` times the FP64 CPU oracle on a bounded sample of the
same workload on this machine's host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "T_eff GB/s per step (3*N*s bytes / step time), stencil + halo, hidden communication"
WORKLOAD = "decomposed_2x2x2_512x256x256"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel_file: str, key: str):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[key]
        src = open(os.path.join(ROOT, "paper_2211_15716_gb300", "csrc", kernel_file), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None


def oracle_baseline(budget_s: float = 12.0):
    """FP64 CPU oracle, one 512x256x256 subdomain of the workload, repeated
    steps for about `budget_s` seconds on all host cores."""
    import oracle
    import synth

    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    n = (512, 256, 256)
    dims, periods, o = (2, 2, 2), (1, 0, 0), (2, 2, 2)
    ng = oracle.global_size(n, dims, o, periods)
    g = oracle.global_indices(n, dims, o, periods, 0)
    T = np.ascontiguousarray(synth.gaussian_bump(*g, ng) * np.ones((n[2], n[1], n[0])))
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(1, *g, ng))
    dd = [oracle.spacing(1.0, ng[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    T2 = T.copy()
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.step(T2, T, Ci, 1.0, dt, *dd)
        T, T2 = T2, T
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 2000:
            break
    npts = n[0] * n[1] * n[2]
    inner = (n[0] - 2) * (n[1] - 2) * (n[2] - 2)
    return {"value": 3 * npts * 8 * reps / el / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} steps of one 512x256x256 FP64 subdomain (of 8), no halo, {el:.1f} s",
            "cell_updates_per_s": inner * reps / el}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    cb = oracle_baseline(budget_s=max(5.0, min(60.0, 2.0 * (args.steps + args.warmup))))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="decomposed_2x2x2_512x256x256 (default) or a smaller case for profiling")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.warmup < 3:
        args.warmup = 3

    import paper_2211_15716_gb300 as igg
    from paper_2211_15716_gb300 import build as igg_build
    from paper_2211_15716_gb300 import workloads as wl

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    igg_build.build()

    w = wl.WORKLOADS[args.workload]
    tdtype = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[args.dtype]
    grid = igg.Grid(w.n, dims=w.dims, overlap=w.overlap, periods=w.periods)
    T, T2, Ci = wl.make_fields(w, grid, tdtype)
    if tdtype == torch.float64:
        dx, dy, dz, dt = wl.setup(w, grid, Ci)
    else:  # dt from the FP64 inputs, as for the FP64 form
        _, _, Ci64 = wl.make_fields(w, grid, torch.float64)
        dx, dy, dz, dt = wl.setup(w, grid, Ci64)
        del Ci64, _
    N = grid.nsub * grid.nloc
    inner = grid.nsub * (w.n[0] - 2) * (w.n[1] - 2) * (w.n[2] - 2)
    s = T.element_size()
    bytes_step = 3 * N * s
    stream = torch.cuda.current_stream()

    # warm-up (also captures the two-step CUDA graph)
    cur = grid.run(args.warmup, T, T2, Ci, w.lam, dt, dx, dy, dz, widths=w.widths)
    if cur is T2:
        T, T2 = T2, T
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- timed region: K hidden steps -----------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    cur = grid.run(args.steps, T, T2, Ci, w.lam, dt, dx, dy, dz, widths=w.widths)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    if cur is T2:
        T, T2 = T2, T
    ms_step = ms / args.steps

    # ---- dominant kernel: the full-step stencil kernel on this stream ----
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kreps = max(10, args.steps // 2)
    k0.record(stream)
    for _ in range(kreps):
        grid.step(T2, T, Ci, w.lam, dt, dx, dy, dz)
    k1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    k_ms = k0.elapsed_time(k1) / kreps

    # ---- end to end: host inputs -> K steps -> host result ----------------
    Th = torch.empty(T.shape, dtype=T.dtype, pin_memory=True)
    Ch = torch.empty(Ci.shape, dtype=Ci.dtype, pin_memory=True)
    Rh = torch.empty(T.shape, dtype=T.dtype, pin_memory=True)
    Th.copy_(T)
    Ch.copy_(Ci)
    torch.cuda.synchronize()
    barrier()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    T.copy_(Th, non_blocking=True)
    T2.copy_(Th, non_blocking=True)
    Ci.copy_(Ch, non_blocking=True)
    cur = grid.run(args.steps, T, T2, Ci, w.lam, dt, dx, dy, dz, widths=w.widths)
    Rh.copy_(cur, non_blocking=True)
    x1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = x0.elapsed_time(x1)
    if ws > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    assert torch.isfinite(Rh[0, 5, 5, :8].float()).all()

    hbm, hbm_kind = peaks()
    value = ws * bytes_step / (ms_step * 1e-3) / 1e9
    achieved = bytes_step / (k_ms * 1e-3) / 1e9
    traffic = traffic_for("stencil.cu", f"stencil {args.dtype} full step {args.workload}")
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic (seeded Gaussian bump T0, Ci = 1/U[1.5,2.5] on global indices)",
        "config": {"workload": args.workload, "subdomains": "x".join(map(str, w.dims)),
                   "local": "x".join(map(str, w.n)), "overlap": 2, "periods": "x",
                   "widths": list(w.widths), "nt_timed": args.steps,
                   "cells": N, "inner_cells": inner, "bytes_per_step": bytes_step,
                   "l2": f"inputs larger than L2 ({bytes_step / 1e9:.2f} GB moved per step vs 129 MB L2)",
                   "graph": "two steps per CUDA graph launch"},
        "cell_updates_per_s": ws * inner / (ms_step * 1e-3),
        "frac_of_8TBs": round(value / ws / 8000.0, 4),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": traffic,
                     "kernel": f"stencil kernel, {args.dtype} (full step, all subdomains)",
                     "peak_kind": hbm_kind, "kernel_ms": round(k_ms, 4)},
        "e2e": {"value": round(ws * bytes_step * args.steps / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": int(3 * N * s / args.steps),
                "d2h_bytes_per_step": int(N * s / args.steps),
                "note": "one job: H2D of T, T2 (= copy(T)) and Ci from pinned memory, K steps, D2H of T"},
        "gpu_launches": 5 * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        line["cpu_baseline"] = oracle_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    grid.finalize()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
