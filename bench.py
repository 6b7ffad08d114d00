"""Benchmark: S-model DVM cell x velocity-node updates per second on one GB300.

Default workload: the lid-driven cubic cavity, 16^3 = 4,096 hex cells, 32^3 velocity
nodes on [-6,6]^3, Kn = 0.1, diffuse walls at T = 1, lid speed 0.2 (synthetic, seeded).
A "step" is one explicit time step of the whole hot path over every cell: moments,
Shakhov equilibrium, boundary ghosts, upwind face fluxes and the Euler update (full
grid), plus Tucker rounding in the Tucker format.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--path full|tucker]
                    [--impl reference]

Prints one JSON line (rank 0).  With --impl reference the FP64 CPU oracle is timed on
the same workload instead (bounded sample per step).  N > 1 runs independent replicas
(one solve per GPU; the method has no data-path collective on one box).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DVM cell·velocity-node updates/s (Tucker vs full) at ≤1e-4 err; p99 solve latency"
UNIT = "updates/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--path", default="full", choices=["full", "tucker"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--rank-cap", type=int, default=None)
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--workload", default="cavity")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def make_workload(name):
    import workloads as W
    if name == "cavity":
        return W.cavity()
    if name == "cavity_small":
        return W.cavity(nside=8, N=24)
    if name == "sod":
        return W.sod_row()
    raise SystemExit(f"unknown workload {name}")


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel source is
    unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = os.path.join(ROOT, "paper_1912_04582_gb300", "csrc", "full_kernels.cu"
                       if kernel == "full" else "tucker_kernels.cu")
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for ln in open(p):
        t = ln.split()
        if len(t) >= 3 and not ln.startswith("#") and t[0] == kernel and t[1] == h:
            return float(t[2])
    return None


# --------------------------------------------------------------------------
def cpu_baseline(wl, budget_s=20.0):
    """The FP64 oracle (as it stands) on the host cores: full-workload steps until the
    budget is used (at least one)."""
    import oracle
    o = oracle.FullGridOracle(wl)
    dt = o.dt()
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step(1, dt)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": wl.n_cell * wl.nodes_per_cell * n / el, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{n} full step(s) of {wl.name} in {el:.1f} s (FP64 C oracle, OpenMP)"}


def run_reference(args, rank, world):
    wl = make_workload(args.workload)
    if rank != 0:
        return
    import oracle
    o = oracle.FullGridOracle(wl)
    dt = o.dt()
    for _ in range(args.warmup):
        o.step(1, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1, dt)
    el = time.perf_counter() - t0
    upd = wl.n_cell * wl.nodes_per_cell
    v = upd * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {**wl.describe(), "path": "full",
                                             "format": "full FP64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full step(s) of {wl.name}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    import paper_1912_04582_gb300 as P
    from paper_1912_04582_gb300 import _native as NAT

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    wl = make_workload(args.workload)
    fmt = NAT.DVM_FORMAT_TUCKER if args.path == "tucker" else NAT.DVM_FORMAT_FULL
    prec = NAT.DVM_PREC_MIXED if args.precision == "mixed" else NAT.DVM_PREC_FP64
    s = P.Solver(wl, format=fmt, precision=prec, stream=stream.cuda_stream,
                 rank_cap=args.rank_cap, tol=args.tol)
    upd = wl.n_cell * wl.nodes_per_cell

    for _ in range(args.warmup):
        s.step(1, residual=False)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        s.step(args.steps, residual=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    res = s.step(1)  # residual check after the timed region (state stays physical)
    value = world * upd * args.steps / (ms / 1e3)
    launches_per_step = 1 if args.path == "full" else None

    # roofline of the dominant kernel (the fused step: one launch per step)
    peaks, src = _peaks()
    kern_ms = ms / args.steps
    alg_bytes = 2 * 8 * upd                  # read f^n once, write f^{n+1} once (FP64)
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": _traffic("full"),
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
            "kernel": "full_step_kernel", "alg_bytes_per_launch": alg_bytes}

    # end-to-end through the C ABI with host buffers: H2D of f, one step, D2H of moments
    e2e = None
    if not args.no_e2e and rank == 0:
        f_host = torch.empty((wl.n_cell,) + tuple(wl.N), dtype=torch.float64, pin_memory=True)
        f_np = f_host.numpy()
        f_np[...] = s.f()
        k = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            P.dvm_init_f(s.h, f_np)
            s.step(1, residual=False)
            m = s.moments()
        el = time.perf_counter() - t0
        e2e = {"value": upd * k / el, "unit": UNIT, "h2d_bytes_per_step": int(f_np.nbytes),
               "d2h_bytes_per_step": int(m.nbytes),
               "note": "per step: dvm_init_f from pinned host f, dvm_step, dvm_moments to host"}

    line = None
    if rank == 0:
        cfg = {**wl.describe(), "path": args.path,
               "format": "full tensor FP64" if args.path == "full" else "Tucker",
               "l2": f"inputs larger than L2 ({8 * upd / 1e9:.2f} GB per copy of f)",
               "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}
        clocks = clk.summary()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": cfg, "roofline": roof,
                "gpu_launches": (launches_per_step * args.steps) if launches_per_step else None,
                "clocks": clocks, "residual_after": res}
        if e2e:
            line["e2e"] = e2e
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
