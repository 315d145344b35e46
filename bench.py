"""Benchmark of the split time step (HLLC sweeps + relaxations + Chebyshev
parabolic stages) of the two-temperature diffuse-interface model.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload impact]

One step = one full split step over the workload grid (CFL reduction, x and y
hyperbolic sweeps with pressure relaxation, viscous steps, temperature
relaxation and heat conduction).  Prints one JSON line on rank 0.

Timing: W untimed warm-up steps, then K steps timed one by one with CUDA events
on the solver's stream, a 256 MiB buffer write between steps flushing the L2
(129 MB), barrier + synchronize around the timed region, max over ranks.
Multi-GPU (torchrun): every rank advances its own replica of the workload
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per full split step (HLLC+Chebyshev) and % of HBM roofline"
UNIT = "cell-updates/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# FP64 rate of a GB300 (152 SMs x 2070 MHz x 4 FP64 FLOP/clk/SM, the nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="impact")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-bulk variant")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched configuration")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the gradient (dim_grad) measurement")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="run only the gradient measurement and print its JSON object (profiling)")
    ap.add_argument("--adjoint-steps", type=int, default=None, help="steps of the gradient problem (default 200)")
    ap.add_argument("--adjoint-ckpt", type=int, default=None, help="checkpoint spacing (default 20)")
    ap.add_argument("--batch-ninst", type=int, default=256, help="instances of the batched configuration")
    return ap.parse_args()


def workload_desc(wl):
    return {
        "workload": f"{wl.name} {wl.nx}x{wl.ny} FP64 (2D multiphase impact: solid projectile at 500 m/s on a "
                    f"solid slab in air, heat conduction and viscosity on)" if wl.name == "impact" else
        f"{wl.name} {wl.nx}x{wl.ny} FP64",
        "cells": wl.nx * wl.ny,
        "grid": [wl.nx, wl.ny],
        "precision": "fp64",
        "l2": "flushed between timed steps (256 MiB buffer write); state 33.6 MB < L2",
    }


def clocks_sampler_start(dev_index: int):
    try:
        f = open(os.devnull, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "-i", str(dev_index),
             "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE, stderr=f, text=True)
        return p
    except Exception:
        return None


def clocks_sampler_stop(p):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        return None
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for nm, v in zip(names, f[4:8]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def kernel_hash():
    h = hashlib.sha256()
    for fn in ("dim_device.cuh", "dim_sweep.cu", "dim_parabolic.cu"):
        with open(os.path.join(ROOT, "paper_2106_00282_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(PEAKS) as f:
            return json.load(f)
    except Exception:
        return {}


def flops_per_cell(kernel: str, wl) -> float:
    """Algorithmic FP64 operations per cell of one launch (+ - * / sqrt each
    one, as the plain FP64 statement of the stage performs them)."""
    from paper_2106_00282_gb300 import flops

    ndim = 2 if wl.nx > 1 and wl.ny > 1 else 1
    return flops.per_cell(kernel, wl.params, ndim=ndim)


def aggregate(ms_local: float, units_per_rank: float, world: int, dev):
    """Whole-job figures of `world` replicas: the slowest rank's time (max over
    ranks) and the units all ranks processed divided by that time (per second).
    With world > 1 every rank must call this (one all-reduce)."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def run_ours(args, rank, world, dev, precision=0, with_e2e=True):
    import torch

    from paper_2106_00282_gb300 import build as cuda_build, inputs as I
    from paper_2106_00282_gb300.api import Solver

    if rank == 0:
        cuda_build.build()
    if world > 1:
        torch.distributed.barrier()
    wl = I.bench_workload(args.workload)
    wl.params = wl.params.replace(precision=precision)
    ncell = wl.nx * wl.ny
    s = Solver(wl.params, wl.nx, wl.ny, wl.dx, wl.dy)
    U0 = s.from_primitive(torch.from_numpy(wl.prim).to(dev))
    U = U0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    W = max(3, args.warmup)
    K = args.steps
    s.step(U, W)
    torch.cuda.synchronize()
    st0 = s.status(reset=True)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sampler = clocks_sampler_start(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3)
    s.profile(True, reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record()
        s.step(U, 1, sync=False)
        ev[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clocks_sampler_stop(sampler)
    s.profile(False, reset=False)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate(ms, ncell * K, world, dev)
    st = s.status()
    if st & 3:
        raise RuntimeError(f"inadmissible state during the timed steps (status {st})")

    # per-kernel device times over the timed region
    kern = {}
    launches = 0
    for name in ("wave_max", "sweep_x", "sweep_y", "viscous_x", "viscous_y", "heat", "relax", "copy"):
        nl, kms = s.kernel_time(name)
        if nl:
            kern[name] = {"launches": nl, "ms": kms, "avg_us": 1e3 * kms / nl}
            if name != "copy":
                launches += nl
    dom = max((k for k in kern if k != "copy"), key=lambda k: kern[k]["ms"])
    peaks = measured_peak()
    fpc = flops_per_cell(dom, wl)
    achieved = fpc * ncell / (kern[dom]["avg_us"] * 1e-6) / 1e12
    traffic = None
    try:
        with open(TRAFFIC) as f:
            tr = json.load(f)
        e = tr.get(args.workload, {}).get(dom)
        if e and e.get("kernel_hash") == kernel_hash():
            traffic = e["bytes_per_launch"]
    except Exception:
        pass
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": dom,
                "flops_per_cell": fpc, "peak_source": "nominal FP64 rate (152 SMs x 2070 MHz x 4 FLOP/clk/SM)",
                "kernels": kern}
    hbm = peaks.get("hbm_gbs")
    alg_bytes = 128.0 * ncell  # the 8-plane FP64 state read and written once per step
    step_us = 1e3 * ms_max / K
    hbm_frac = (alg_bytes / (step_us * 1e-6) / 1e9) / hbm if hbm else None
    # DRAM bytes of a whole step from the recorded per-kernel traffic (ncu),
    # when every kernel of the step has a record for the current kernels
    dram_step = 0.0
    try:
        with open(TRAFFIC) as f:
            trw = json.load(f).get(args.workload, {})
        for name, v in kern.items():
            if name == "copy":
                continue
            e = trw.get(name)
            if not e or e.get("kernel_hash") != kernel_hash():
                dram_step = None
                break
            dram_step += e["bytes_per_launch"] * v["launches"] / K
    except Exception:
        dram_step = None
    hbm_obj = {"peak_gbs": hbm, "alg_bytes_per_step": alg_bytes,
               "eta_alg": hbm_frac,
               "dram_bytes_per_step": dram_step,
               "eta_dram": (dram_step / (step_us * 1e-6) / 1e9) / hbm if (hbm and dram_step) else None}

    # end to end: host buffers through dim_step_host (copies inside the timed region)
    e2e = None
    if with_e2e and not args.no_e2e:
        Uh = U0.cpu().pin_memory()
        Ke = max(3, min(K, 30))
        s.step_host(Uh, 1)
        tot = 0.0
        for k in range(Ke):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step_host(Uh, 1)
            tot += time.perf_counter() - t0
        _, e2e_value = aggregate(1e3 * tot, ncell * Ke, world, dev)
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(Uh.numel() * 8), "d2h_bytes_per_step": int(Uh.numel() * 8),
               "steps": Ke, "api": "dim_step_host (pinned host state, H2D + step + D2H per step)"}
    return dict(value=value, ms_per_step=step_us / 1e3, wl=wl, roofline=roofline, e2e=e2e, clocks=clocks,
                launches=launches, hbm_frac=hbm_frac, hbm=hbm_obj, status_warmup=st0)


def run_batched(dev, world=1, steps=10, warmup=3, ninst=256):
    """256 independent water/air problems of uneven sizes (FP32 bulk), one
    persistent launch per step replayed from a CUDA graph; the packed state
    (4.1 GB) is larger than the L2, so no flush is needed."""
    import torch

    from paper_2106_00282_gb300 import inputs as I
    from paper_2106_00282_gb300.api import Batch

    params, grids, prims = I.batch(ninst=ninst, seed=4)
    B = Batch(params, grids)
    U = B.from_primitive(B.pack_primitive(prims))
    del prims
    cfg = B.autotune(U)
    B.step(U, max(3, warmup))
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for a, e in ev:
        a.record()
        B.step(U, 1)
        e.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms, value = aggregate(sum(a.elapsed_time(e) for a, e in ev), B.ncell * steps, world, dev)
    flags, anyf = B.status()
    sizes = sorted({g[0] for g in grids} | {g[1] for g in grids})
    out = {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "instances": len(grids) * world,
           "cells": B.ncell, "sizes": sizes, "steps": steps, "status_or": anyf,
           "autotune": {"variant": cfg[0], "blocks": cfg[1], "x_tile": [cfg[2], cfg[3]], "y_tile": [cfg[4], cfg[5]]},
           "launch": "one persistent cooperative kernel per step, CUDA-graph replay",
           "precision": "fp32-bulk"}
    B.close()
    return out


def run_adjoint(dev, world=1, steps=None, ckpt=None):
    """The gradient problem on the conduction disc (512^2, FP64, 200 steps,
    checkpoints every 20): time of the forward run alone (dim_step) and of
    dim_grad (forward with checkpoints + reverse sweep with recomputation),
    each between device synchronizations, after one untimed call that
    allocates the workspace."""
    import torch

    from paper_2106_00282_gb300 import inputs as I
    from paper_2106_00282_gb300.api import Solver

    wl = I.disc_gradient()
    nsteps = steps or wl.steps
    ckpt = ckpt or wl.meta["ckpt"]
    s = Solver(wl.params, wl.nx, wl.ny, wl.dx, wl.dy)
    U0 = s.from_primitive(torch.from_numpy(wl.prim).to(dev))
    g = torch.randn(U0.shape, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(5))
    g /= U0.abs().reshape(8, -1).mean(1).clamp_min(1.0)[:, None, None]
    s.grad(U0, 4, g, 2)
    U = U0.clone()
    s.step(U, 2)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    U = U0.clone()
    s.step(U, nsteps)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    gU, gp = s.grad(U0, nsteps, g, ckpt)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    cells = wl.nx * wl.ny
    _, value = aggregate(1e3 * t_grad, cells * nsteps, world, dev)
    s.close()
    return {"workload": f"conduction-disc gradient problem {wl.nx}x{wl.ny}, {nsteps} steps, checkpoints every {ckpt}",
            "value": value, "unit": "cell-steps/s (forward + reverse)", "grad_s": t_grad, "forward_s": t_fwd,
            "grad_over_forward": t_grad / t_fwd, "precision": "fp64",
            "params_grad": [float(x) for x in gp]}


def host_cpu():
    """nproc and the CPU model of the host (from /proc/cpuinfo; Arm cores by implementer and part)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for line in info.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
        if model is None:
            imp = [l.split(":", 1)[1].strip() for l in info.splitlines() if l.startswith("CPU implementer")]
            part = [l.split(":", 1)[1].strip() for l in info.splitlines() if l.startswith("CPU part")]
            if imp and part:
                model = f"Arm implementer {imp[0]} part {part[0]}"
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_rate(wl, budget_s=10.0, max_steps=1000):
    """FP64 oracle (single-threaded C) on the same workload: steps until the budget."""
    from oracle import oracle as O

    U = O.from_primitive(wl.params, wl.prim)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps:
        U = O.step(wl.params, U, wl.dx, wl.dy, 1)[0]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return wl.nx * wl.ny * n / el, n, el


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return main_reference(args, rank, world)
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    if args.only_adjoint:
        from paper_2106_00282_gb300 import build as cuda_build

        cuda_build.build()
        ra = run_adjoint(dev, world, args.adjoint_steps, args.adjoint_ckpt)
        if rank == 0:
            print(json.dumps({"adjoint": ra}))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    r = run_ours(args, rank, world, dev)
    r32 = None if args.no_fp32 else run_ours(args, rank, world, dev, precision=1, with_e2e=False)
    rb = None if args.no_batch else run_batched(dev, world, ninst=args.batch_ninst)
    ra = None if args.no_adjoint else run_adjoint(dev, world, args.adjoint_steps, args.adjoint_ckpt)
    if rank == 0:
        wl = r["wl"]
        cpu = None
        if not args.no_cpu:
            from paper_2106_00282_gb300 import inputs as I

            rate, nst, el = oracle_rate(I.bench_workload(args.workload))
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{nst} oracle steps of the full {wl.nx}x{wl.ny} grid from the initial state "
                             f"({el:.1f} s, single-threaded C, -O2 -ffp-contract=off)",
                   "host": host_cpu()}
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload_desc(wl), parallelism=f"replicas{world}" if world > 1 else "single"),
                "hbm_roofline_frac_alg": r["hbm_frac"], "hbm": r["hbm"], "roofline": r["roofline"],
                "cpu_baseline": cpu,
                "e2e": r["e2e"], "clocks": r["clocks"], "gpu_launches": r["launches"]}
        if rb is not None:
            line["batched"] = rb
        if ra is not None:
            line["adjoint"] = ra
        if r32 is not None:
            line["fp32_bulk"] = {
                "value": r32["value"], "unit": UNIT, "ms_per_step": r32["ms_per_step"],
                "speedup_vs_fp64": r32["value"] / r["value"], "clocks": r32["clocks"],
                "kernels_us": {k: round(v["avg_us"], 1) for k, v in r32["roofline"]["kernels"].items()},
                "precision": "FP32 flux/stencil arithmetic; FP64 state accumulation, phase pressures, "
                             "volume-fraction transport, relaxation root solves, Chebyshev parameters",
                "accuracy": "relative L1 per conserved field vs the FP64 oracle <= 2e-5 after 100 steps "
                            "(tests/test_gpu_fp32.py)"}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_2106_00282_gb300 import inputs as I
    from oracle import oracle as O

    O.build()
    wl = I.bench_workload(args.workload)
    U = O.from_primitive(wl.params, wl.prim)
    for _ in range(max(3, args.warmup)):
        U = O.step(wl.params, U, wl.dx, wl.dy, 1)[0]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = O.step(wl.params, U, wl.dx, wl.dy, 1)[0]
    el = time.perf_counter() - t0
    value = wl.nx * wl.ny * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full oracle steps of the {wl.nx}x{wl.ny} grid after "
                                       f"{max(3, args.warmup)} warm-up steps",
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
