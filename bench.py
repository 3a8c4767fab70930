#!/usr/bin/env python3
"""Particle-steps/s of the per-step particle operator (collide + project), FP64.

Workload (default): 1,048,576 spheres, d ~ U[0.006, 0.008] (phi ~0.19), v ~ N(0,1),
e = 0.9, dt = 0.99 * 0.25 * d_min / max|v|, 32^3 hex mesh of degree 5 (6^3 Gauss
nodes per element), Gaussian sigma = 0.01 with a 3 sigma box cutoff, 4 N(0,1)
sources per particle. One step = pc_collide + pc_project over the whole state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0. Under torchrun each rank runs an independent
replica of the workload (seed = rank), weak scaling, no data-path collective.
"""
import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_05340_gb300 import inputs  # noqa: E402

METRIC = "particle-steps/s collide+project (FP64)"
UNIT = "particle-steps/s"
# FP64 pipe of a GB300: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (max SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# dram bytes per launch of the dominant kernel from the committed ncu capture
# (profiles/), or None when the kernel changed since that capture.
DEPOSIT_DRAM_BYTES = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def support_nodes(x, wl):
    """Gauss nodes inside each particle's box cutoff: sum_p n_x n_y n_z (exact, periodic)."""
    eta, _ = np.polynomial.legendre.leggauss(wl.degree + 1)
    h = 1.0 / wl.ne
    X = np.sort(((np.arange(wl.ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) * h).ravel())
    Xe = np.concatenate([X - 1.0, X, X + 1.0])
    rc = wl.cutoff_sigmas * wl.sigma
    tot = np.ones(x.shape[1], np.float64)
    for a in range(3):
        lo = np.searchsorted(Xe, x[a] - rc, side="left")
        hi = np.searchsorted(Xe, x[a] + rc, side="right")
        tot *= (hi - lo)
    return float(tot.sum())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc:
            return None
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_ours(args, ws, rank, local):
    import torch

    from paper_2501_05340_gb300 import pc

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    wl = inputs.WORKLOADS[args.workload]
    w = inputs.draw(args.workload, seed=rank)
    n, dt = w["x"].shape[1], w["dt"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = pc.State.from_arrays(w)
        b = pc.State.empty(n)
        ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt),
                         cutoff_sigmas=wl.cutoff_sigmas, stream=stream)
        field = ctx.new_field()
    torch.cuda.synchronize()

    def step(src, dst):
        ctx.collide(src, dst, dt)
        ctx.project(dst, field)

    for _ in range(args.warmup):
        step(a, b)
        a, b = b, a
    ctx.sync()
    ctx.set_timing(True)
    ctx.timing()
    l0 = ctx.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step(a, b)
            a, b = b, a
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = ev0.elapsed_time(ev1)
    phases = ctx.timing()
    ctx.set_timing(False)
    st = ctx.stats()
    launches = st["kernel_launches"] - l0
    if st["status"] != 0:
        raise RuntimeError("device status %d during the timed region" % st["status"])
    t_max = ms
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = n * args.steps * ws / (t_max / 1e3)

    # dominant kernel and its roofline
    dom = max(phases, key=lambda k: phases[k][0])
    dms, dcnt = phases[dom]
    roofline = None
    if dom == "deposit" and dcnt:
        nodes = support_nodes(a.x.cpu().numpy(), wl)
        flops = 8.0 * nodes  # 4 FMA (one per source component) per (particle, support node)
        achieved = flops / (dms / dcnt / 1e3) / 1e12
        roofline = {"kernel": "k_proj_gather", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": DEPOSIT_DRAM_BYTES,
                    "peak_source": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived, recipe unit counts)",
                    "algorithmic": "8 flop per (particle, Gauss node in its box support): %.4g flop per launch" % flops}
    phase_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in phases.items()}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(args, ctx, w, n, dt, stream, torch, pc, dist, ws)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, wl)
    clocks = clk.summary()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded random sequential addition, N(0,1) velocities and sources)",
        "config": {"workload": args.workload, "particles_per_gpu": n, "mesh": "%d^3 hex, degree %d" % (wl.ne, wl.degree),
                   "sigma": wl.sigma, "cutoff": "3 sigma box", "dt": dt, "restitution": w["e"],
                   "phi": round(w["phi"], 4), "l2": "inputs larger than L2 (state 105 MB + field 226 MB + scratch)",
                   "parallelism": "independent replica per GPU" if ws > 1 else "1 GPU"},
        "phase_ms_per_call": phase_ms, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks,
        "collide_stats": {k: st[k] for k in ("pairs", "candidates", "worklist", "rounds", "fp64_solves",
                                              "max_candidates", "cells_per_side", "stencil")},
    }


def e2e_run(args, ctx, w, n, dt, stream, torch, pc, dist, ws):
    """Same metric through the public API with host buffers: every step copies the
    input state from pinned host memory and reads the field back."""
    pin = lambda arr, dtp=torch.float64: torch.as_tensor(np.ascontiguousarray(arr)).to(dtp).pin_memory()
    host = dict(x=pin(w["x"]), v=pin(w["v"]), r=pin(w["r"]), m=pin(w["m"]), id=pin(w["id"], torch.int32),
                q=pin(w["q"]))
    dev = pc.State.empty(n)
    out = pc.State.empty(n)
    field = ctx.new_field()
    fhost = torch.empty(field.shape, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = field.numel() * 8

    def step():
        with torch.cuda.stream(stream):
            for k in ("x", "v", "r", "m", "id", "q"):
                getattr(dev, k).copy_(host[k], non_blocking=True)
            ctx.collide(dev, out, dt)
            ctx.project(out, field)
            fhost.copy_(field, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    stream.synchronize()
    el = time.perf_counter() - t0
    if dist:
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    return {"value": n * args.steps * ws / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


def cpu_sample(w, wl, frac_project=16):
    """Oracle time for one step over the workload: the full collide step, and the
    projection of every frac_project-th particle (scaled by frac_project)."""
    import oracle
    t0 = time.perf_counter()
    oracle.collide_step(w["x"], w["v"], w["r"], w["m"], w["id"], w["e"], w["dt"])
    t1 = time.perf_counter()
    sel = slice(0, None, frac_project)
    oracle.project(w["x"][:, sel], w["q"][:, sel], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    t2 = time.perf_counter()
    return (t1 - t0) + frac_project * (t2 - t1), t1 - t0, t2 - t1


def cpu_baseline(w, wl):
    n = w["x"].shape[1]
    tot, tc, tp = cpu_sample(w, wl)
    return {"value": n / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one full collide step over all %d particles (%.1f s) + projection of every 16th particle "
                      "(%.1f s, scaled x16), single thread, FP64 C oracle" % (n, tc, tp)}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    wl = inputs.WORKLOADS[args.workload]
    w = inputs.draw(args.workload, seed=0)
    n = w["x"].shape[1]
    for _ in range(args.warmup):
        cpu_sample(w, wl, frac_project=64)
    times = []
    for _ in range(args.steps):
        times.append(cpu_sample(w, wl, frac_project=64)[0])
    tot = float(np.sum(times))
    value = n * args.steps / tot
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "particles_per_gpu": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: one full collide step over all %d particles + projection of every "
                                       "64th particle scaled x64; single-thread FP64 C oracle" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
