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
# DRAM bytes (read + write) per launch of the dominant kernels at the bench workloads, from one
# ncu capture of each (dram__bytes_read.sum + dram__bytes_write.sum, summarised under profiles/);
# None once a kernel has changed since its capture.
DEPOSIT_KERNEL = "k_fx_deposit"
DEPOSIT_DRAM_BYTES = 751.2e6   # k_fx_deposit<6>, dense_1m
TC_DEPOSIT_DRAM_BYTES = 3.919e9  # k_tc_deposit<0, 8>, mixed_16m (8 workers)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-operators", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-curved", action="store_true",
                    help="skip the 67M-particle curved-mesh workload (its state takes minutes to draw on the host)")
    ap.add_argument("--mixed-steps", type=int, default=5)
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


def max_over_ranks(x, dist, device="cuda"):
    """The maximum of x over the ranks of the process group (x itself without one)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
    t_max = max_over_ranks(ms, dist)
    value = n * args.steps * ws / (t_max / 1e3)

    # dominant kernel and its roofline
    dom = max(phases, key=lambda k: phases[k][0])
    dms, dcnt = phases[dom]
    roofline = None
    if dom == "deposit" and dcnt:
        roofline = deposit_roofline(a.x.cpu().numpy(), wl, n, dms / dcnt, ms / args.steps)
    phase_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in phases.items()}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(args, ctx, w, n, dt, stream, torch, pc, dist, ws)

    operators = None
    if not args.no_operators:
        operators = operators_run(args, ctx, a, wl, stream, torch, pc, dt)

    ctx.close()
    del a, b, field
    adjoint = None
    if not args.no_adjoint and args.workload == "dense_1m":
        adjoint = adjoint_run(args, w, wl, stream, torch, pc)
    curved = None
    if not args.no_curved:
        try:
            curved = curved_run(args, rank, torch, pc, stream)
        except (RuntimeError, MemoryError, pc.PcError) as exc:  # keep the line; say why the leg is missing
            curved = {"workload": "curved_67m", "error": str(exc)[:300]}
    mixed = None
    if not args.no_mixed:
        mixed = mixed_run(args, rank, torch, pc, stream)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, wl)
    clocks = clk.summary()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded random sequential addition, N(0,1) velocities and sources)",
        "config": bench_config(args, w, ws),
        "phase_ms_per_call": phase_ms, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks, "mixed": mixed, "operators": operators, "adjoint": adjoint, "curved": curved,
        "collide_stats": {k: st[k] for k in ("pairs", "candidates", "worklist", "rounds", "fp64_solves",
                                              "max_candidates", "cells_per_side", "stencil")},
    }


def bench_config(args, w, ws):
    """The workload description both arms print."""
    wl = inputs.WORKLOADS[args.workload]
    return {"workload": args.workload, "particles_per_gpu": int(w["x"].shape[1]),
            "mesh": "%d^3 hex, degree %d" % (wl.ne, wl.degree), "sigma": wl.sigma,
            "cutoff": "%g sigma %s" % (wl.cutoff_sigmas, wl.cutoff), "dt": w["dt"], "restitution": w["e"],
            "phi": round(w["phi"], 4), "l2": "inputs larger than L2 (state 105 MB + field 226 MB + scratch)",
            "parallelism": "independent replica per GPU" if ws > 1 else "1 GPU"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth, else the fallback."""
    pk = measured_peaks().get("hbm_gbs")
    if pk:
        return float(pk), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return 6800.0, "fallback 6.8 TB/s (of fallback)"


def step_algorithmic_bytes(n, wl, per_particle=144):
    """Minimum HBM bytes of one FP64 step: read the state once (x, v, r, m, q: 144 B per
    particle), write x and v once, write the field once (8 B per node and component)."""
    return n * per_particle + wl.ne ** 3 * 4 * (wl.degree + 1) ** 3 * 8


def deposit_roofline(x, wl, n, dep_ms, step_ms):
    """HBM roofline of the FP64 deposit (the step's dominant kernel): algorithmic bytes per
    launch = particles x (x 24 B + q 32 B) read once + the field written once (8 B per node
    and component), over the kernel's mean CUDA-event duration, against the measured HBM
    copy bandwidth; the whole step beside it. What really bounds the kernel is stated too:
    the method's 8 flop (4 multiply-adds, one per source component) per (particle, Gauss
    node inside its box support), computed FP64-accurately as an exact fixed-point digit
    contraction on the tensor cores whose digit operands are built on the CUDA cores,
    against the FP64 pipe's derived peak."""
    peak, src = hbm_peak()
    nel, nodes = wl.ne ** 3, (wl.degree + 1) ** 3
    algo = n * 56 + nel * 4 * nodes * 8
    sec = dep_ms / 1e3
    achieved = algo / sec / 1e9
    step_algo = step_algorithmic_bytes(n, wl)
    step_gbs = step_algo / (step_ms / 1e3) / 1e9
    support = support_nodes(x, wl)
    traffic = DEPOSIT_DRAM_BYTES if (wl.name == "dense_1m" and DEPOSIT_DRAM_BYTES) else None
    return {"kernel": DEPOSIT_KERNEL if wl.degree + 1 <= 8 else "k_proj_deposit", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_over_algorithmic": (traffic / algo) if traffic else None,
            "peak_source": src, "algorithmic_bytes": algo,
            "algorithmic": "particles x (x 24 B + q 32 B) + field %d elements x 4 x %d nodes x 8 B, per launch"
                           % (nel, nodes),
            "kernel_ms": dep_ms,
            "step": {"algorithmic_bytes": step_algo, "achieved": step_gbs, "frac": step_gbs / peak,
                     "algorithmic": "144 B per particle (read x, v, r, m, q; write x, v) + the field"},
            "alu": {"bound_by": "digit operands of the FP64-accurate tensor-core contraction, built on the CUDA "
                                "cores, and the shared-memory pipe (ALU 48 %, FMA 41 %, LSU wavefronts 73 %, tensor "
                                "17 %: profiles/k_fx_deposit_dense_1m.md)",
                    "method_flop": 8.0 * support,
                    "method_flop_per_unit": "8 per (particle, Gauss node inside its box support)",
                    "achieved_fp64_equivalent_tflops": 8.0 * support / sec / 1e12,
                    "fp64_pipe_peak_tflops": FP64_PEAK_TFLOPS,
                    "frac_of_fp64_pipe": 8.0 * support / sec / 1e12 / FP64_PEAK_TFLOPS}}


def mixed_run(args, rank, torch, pc, stream, workload="mixed_16m"):
    """The mixed-precision path on its own workload (16,777,216 spheres, 64^3 mesh of
    degree 7): pc_collide_f32 + pc_project_f32 (FP16 split, tensor cores) per step,
    and the FP64 path timed on the same workload for comparison."""
    wl = inputs.WORKLOADS[workload]
    w = inputs.draw(workload, seed=rank)
    n, dt = w["x"].shape[1], w["dt"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    out = {"workload": workload, "particles": n, "dt": dt, "unit": UNIT, "tc": "f16"}
    with torch.cuda.stream(stream):
        s64 = pc.State.from_arrays(w)
        ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt),
                         cutoff_sigmas=wl.cutoff_sigmas, stream=stream)
        a = pc.StateF32.empty(n)
        b = pc.StateF32.empty(n)
        ctx.quantize(s64, a)
        f32 = ctx.new_field_f32()
    torch.cuda.synchronize()
    for _ in range(2):
        ctx.collide_f32(a, b, dt)
        ctx.project_f32(b, f32)
        a, b = b, a
    ctx.sync()
    ctx.set_timing(True)
    ctx.timing()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.mixed_steps):
        ctx.collide_f32(a, b, dt)
        ctx.project_f32(b, f32)
        a, b = b, a
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.mixed_steps
    ph = ctx.timing()
    ctx.set_timing(False)
    st = ctx.stats()
    if st["status"] != 0:
        raise RuntimeError("device status %d in the mixed run" % st["status"])
    out["ms_per_step"] = ms
    out["value"] = n / (ms / 1e3)
    out["phase_ms_per_call"] = {k: round(v[0] / max(v[1], 1), 4) for k, v in ph.items()}
    dep_ms = ph["deposit"][0] / max(ph["deposit"][1], 1)
    # tensor work issued: one M=128 N=64 K=16 MMA per 16 kept particles per element
    pairs = element_pairs(b.numpy(), ctx.cells_per_side, wl)
    flops = 2.0 * 128 * 64 * 16 * pairs["chunks"]
    peak = peaks.get("bf16_tflops", 1900.0)
    out["roofline"] = {"kernel": "k_tc_deposit", "bound": "tensor", "achieved": flops / (dep_ms / 1e3) / 1e12,
                       "peak": peak, "unit": "TFLOP/s", "frac": flops / (dep_ms / 1e3) / 1e12 / peak,
                       "traffic": TC_DEPOSIT_DRAM_BYTES if wl.name == "mixed_16m" else None,
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (fp16 has the same dense rate)",
                       "algorithmic": "2*128*64*16 flop per MMA, %d MMAs (16 kept particles each) per launch"
                                      % pairs["chunks"]}
    out["kept_particle_element_pairs"] = pairs["pairs"]
    # per-field error of the tensor-core fields (FP16 and BF16 splits) of the final mixed
    # state against the FP64 path's field of the same state (the FP64 path is held to
    # 1e-12 of the FP64 oracle by the parity tests; the sampled oracle comparison of the
    # FP32 fields at this size is in the tests too): normwise per component
    fbf = ctx.new_field_f32()
    ctx.project_f32(a, fbf, "bf16")
    nc = ctx.cells_per_side
    cell = a.cell.long()
    cx = torch.stack([cell % nc, (cell // nc) % nc, cell // (nc * nc)]).double()
    s_ref = pc.State(((cx + a.o.double()) / nc).contiguous(), a.v.double().contiguous(), a.r.double(),
                     a.m.double(), a.id.clone(), a.q.double().contiguous())
    fields32 = {"f16": f32, "bf16": fbf}
    torch.cuda.synchronize()
    ctx.close()
    del b
    # FP64 path on the same workload (one step after one warm-up)
    with torch.cuda.stream(stream):
        c64 = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt),
                         cutoff_sigmas=wl.cutoff_sigmas, stream=stream)
        t64 = pc.State.empty(n)
        f64 = c64.new_field()
    for rep in range(2):
        if rep == 1:
            ev0.record(stream)
        c64.collide(s64, t64, dt)
        c64.project(t64, f64)
        if rep == 1:
            ev1.record(stream)
    torch.cuda.synchronize()
    c64.sync()
    out["fp64_ms_per_step_same_workload"] = ev0.elapsed_time(ev1)
    out["speedup_vs_fp64"] = out["fp64_ms_per_step_same_workload"] / ms
    c64.project(s_ref, f64)
    c64.sync()
    den = f64.abs().amax(dim=(0, 2))
    out["field_error_vs_fp64_path"] = {
        tc: [float(v) for v in ((fl.double() - f64).abs().amax(dim=(0, 2)) / den).cpu()] for tc, fl in fields32.items()}
    out["field_error_metric"] = "max |F_tc - F_fp64| / max |F_fp64| per component (momentum x, y, z; energy)"
    c64.close()
    del fields32, fbf, f32, a, s_ref
    return out


def element_pairs(s32, nc, wl):
    """Kept (particle, element) pairs of the mixed deposit and its MMA count, from the
    particles' support boxes (every element gets ceil(kept / 16) MMAs)."""
    cell = s32["cell"].astype(np.int64)
    c = np.stack([cell % nc, (cell // nc) % nc, cell // (nc * nc)]).astype(np.float64)
    x = (c + s32["o"].astype(np.float64)) / nc
    eta, _ = np.polynomial.legendre.leggauss(wl.degree + 1)
    rc = wl.cutoff_sigmas * wl.sigma
    ne = wl.ne
    h = 1.0 / ne
    lo = np.floor((x - rc) * ne - 1e-9).astype(np.int64)
    counts = np.zeros(ne ** 3, np.int64)
    first = (eta[0] + 1) / 2 * h
    last = (eta[-1] + 1) / 2 * h
    n = x.shape[1]
    per_axis = []
    for a in range(3):
        es = []
        for o in range(3):
            e = lo[a] + o
            # element e holds a node within rc of x iff its node span [e h + first, e h + last] meets [x - rc, x + rc]
            ok = (e * h + first <= x[a] + rc) & (e * h + last >= x[a] - rc)
            es.append((np.mod(e, ne), ok))
        per_axis.append(es)
    pairs = 0
    for ox in range(3):
        for oy in range(3):
            for oz in range(3):
                ok = per_axis[0][ox][1] & per_axis[1][oy][1] & per_axis[2][oz][1]
                el = (per_axis[2][oz][0] * ne + per_axis[1][oy][0]) * ne + per_axis[0][ox][0]
                counts += np.bincount(el[ok], minlength=ne ** 3)
                pairs += int(ok.sum())
    return {"pairs": pairs, "chunks": int(np.ceil(counts / 16.0).sum())}


def e2e_run(args, ctx, w, n, dt, stream, torch, pc, dist, ws):
    """Same metric through the public API with host buffers: every step copies the
    input state from pinned host memory and reads the field back. The copies run on
    their own streams (host-to-device and device-to-host engines) with two input
    states and two fields, so step k's compute overlaps step k+1's upload and step
    k-1's download; events order each buffer's reuse."""
    pin = lambda arr, dtp=torch.float64: torch.as_tensor(np.ascontiguousarray(arr)).to(dtp).pin_memory()
    host = dict(x=pin(w["x"]), v=pin(w["v"]), r=pin(w["r"]), m=pin(w["m"]), id=pin(w["id"], torch.int32),
                q=pin(w["q"]))
    devs = [pc.State.empty(n), pc.State.empty(n)]
    out = pc.State.empty(n)
    fields = [ctx.new_field(), ctx.new_field()]
    fhost = [torch.empty(fields[0].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = fields[0].numel() * 8
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: [torch.cuda.Event(), torch.cuda.Event()]
    in_ready, in_free, f_ready, f_free = ev(), ev(), ev(), ev()
    for e_ in in_free + f_free:
        e_.record(stream)

    def step(k):
        b = k & 1
        s_in.wait_event(in_free[b])
        with torch.cuda.stream(s_in):
            for key in ("x", "v", "r", "m", "id", "q"):
                getattr(devs[b], key).copy_(host[key], non_blocking=True)
        in_ready[b].record(s_in)
        stream.wait_event(in_ready[b])
        ctx.collide(devs[b], out, dt)
        in_free[b].record(stream)
        stream.wait_event(f_free[b])
        ctx.project(out, fields[b])
        f_ready[b].record(stream)
        s_out.wait_event(f_ready[b])
        with torch.cuda.stream(s_out):
            fhost[b].copy_(fields[b], non_blocking=True)
        f_free[b].record(s_out)

    for k in range(max(1, args.warmup)):
        step(k)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    s_out.synchronize()
    stream.synchronize()
    s_in.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, dist)
    if not torch.equal(fhost[(args.steps - 1) & 1], fields[(args.steps - 1) & 1].cpu()):
        raise RuntimeError("the downloaded field differs from the device field")
    return {"value": n * args.steps * ws / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "overlap": "copies on separate streams, double-buffered"}


def curved_run(args, rank, torch, pc, stream, workload="curved_67m"):
    """The curved-mesh workload: 67,108,864 spheres on the 128^3 degree-3 mesh curved by
    the sine map, per step pc_collide_f32 + pc_project_curved_f32 (FP32 storage, spherical
    cutoff, Jacobian weights, Newton localisation). Drawing the state takes minutes on
    the host; --no-curved skips it."""
    wl = inputs.WORKLOADS[workload]
    w = inputs.draw(workload, seed=rank)
    n, dt = w["x"].shape[1], w["dt"]
    out = {"workload": workload, "particles": n, "dt": dt, "unit": UNIT, "phi": round(w["phi"], 4)}
    with torch.cuda.stream(stream):
        ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt),
                         cutoff_sigmas=wl.cutoff_sigmas, cutoff="sphere", amp=wl.amp, stream=stream)
        a, b = pc.StateF32.empty(n), pc.StateF32.empty(n)
        ctx.quantize(pc.State.from_arrays(w), a)
        field = ctx.new_field_f32()
    del w
    torch.cuda.synchronize()

    def step(src, dst):
        ctx.collide_f32(src, dst, dt)
        ctx.project_curved_f32(dst, field)

    for _ in range(args.warmup):
        step(a, b)
        a, b = b, a
    ctx.sync()
    ctx.set_timing(True)
    ctx.timing()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.mixed_steps):
        step(a, b)
        a, b = b, a
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.mixed_steps
    ph = ctx.timing()
    ctx.set_timing(False)
    if ctx.stats()["status"] != 0:
        raise RuntimeError("device status during the curved run")
    out.update({"ms_per_step": ms, "value": n / (ms / 1e3),
                "phase_ms_per_call": {k: round(v[0] / max(v[1], 1), 4) for k, v in ph.items() if v[1]}})
    ctx.close()
    return out


def adjoint_run(args, w, wl, stream, torch, pc, steps=50, every=10):
    """The differentiable rollout of the dense workload: loss 0.5 ||P(S_50(x, v), q) - T||^2
    with T the projection of a 1 % perturbed copy, forward (pair sets recorded,
    checkpoints every 10 steps) and backward (replays and step adjoints), FP64 (Rollout)
    and FP32 on the mixed path (Rollout32). Times include the library's host syncs."""
    from paper_2501_05340_gb300 import autograd

    n, dt = w["x"].shape[1], w["dt"]
    T = lambda a, dtp=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtp)
    rng = np.random.default_rng(11)
    xp = w["x"] + 0.01 * wl.sigma * rng.normal(size=w["x"].shape)
    xp -= np.floor(xp)
    pert = dict(w, x=xp, v=w["v"] * (1 + 0.01 * rng.normal(size=w["v"].shape)),
                q=w["q"] * (1 + 0.01 * rng.normal(size=w["q"].shape)))
    out = {"workload": args.workload, "steps": steps, "checkpoint_every": every}
    with torch.cuda.stream(stream):
        ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt) * 1.5,
                         stream=stream)
        r, m, ids = T(w["r"]), T(w["m"]), T(w["id"], torch.int32)
        for kind in ("fp64", "fp32"):
            if kind == "fp64":
                target = ctx.new_field()
                ctx.project(pc.State.from_arrays(pert), target)
                fn = autograd.rollout_loss
            else:
                p32 = pc.StateF32.empty(n)
                ctx.quantize(pc.State.from_arrays(pert), p32)
                target = ctx.new_field_f32()
                ctx.project_f32(p32, target)
                fn = autograd.rollout_loss_f32
            times = []
            for _ in range(2):  # the first pass warms up
                x0, v0, q = (T(w[k]).requires_grad_(True) for k in ("x", "v", "q"))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                loss = fn(x0, v0, q, r, m, ids, target, ctx, dt, steps, every)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                loss.backward()
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                times.append((t1 - t0, t2 - t1))
            if ctx.stats()["status"] != 0:
                raise RuntimeError("device status during the %s rollout" % kind)
            fwd, bwd = times[-1]
            out[kind] = {"forward_ms": round(1e3 * fwd, 2), "backward_ms": round(1e3 * bwd, 2),
                         "particle_steps_per_s": n * steps / (fwd + bwd)}
        ctx.close()
    return out


def operators_run(args, ctx, state, wl, stream, torch, pc, args_dt):
    """The corner-node (IDW) and nearest-DOF (Dirac) depositions of the same state, each
    timed alone over --steps calls after --warmup (CUDA events on the library's stream),
    with the achieved HBM bandwidth of their deposit kernels: algorithmic bytes per call
    = particles x (perm 4 + x 24 + q 32 B) + the field written once (+ the 8 x 4 corner
    sums and node densities written and read once for IDW) / the deposit phase's mean
    duration. Also the collision step with friction and rotation next to the
    frictionless one."""
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    n, nel, nodes = state.n, wl.ne ** 3, (wl.degree + 1) ** 3
    field = ctx.new_field()
    out = {"workload": args.workload, "peak_hbm_gbs": peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    # IDW also writes and reads its df32 corner sums (32 x 8 B per element) and node
    # densities (4 x 8 B per node) once
    for kind, extra in (("idw", 2 * (32 + 4) * 8 * nel), ("dirac", 0)):
        call = getattr(ctx, "project_" + kind)
        for _ in range(max(3, args.warmup)):
            call(state, field)
        ctx.sync()
        ctx.set_timing(True)
        ctx.timing()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            call(state, field)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        ph = ctx.timing()
        ctx.set_timing(False)
        if ctx.stats()["status"] != 0:
            raise RuntimeError("device status during the %s deposition" % kind)
        dep = ph["deposit"][0] / max(ph["deposit"][1], 1)
        algo = n * 60 + 4 * nodes * 8 * nel + extra
        out[kind] = {"ms_per_call": round(ms, 4), "particles_per_s": n / (ms / 1e3),
                     "phase_ms_per_call": {k: round(v[0] / max(v[1], 1), 4) for k, v in ph.items() if v[1]},
                     "deposit_algorithmic_bytes": algo, "deposit_hbm_gbs": algo / (dep / 1e3) / 1e9,
                     "deposit_frac": algo / (dep / 1e3) / 1e9 / peak}
    # the collision step with Coulomb friction and rotation (mu = 0.3, N(0, 50^2) spins)
    # next to the frictionless step, both from the same state into a scratch state
    dst = pc.State.empty(n)
    gen = torch.Generator(device="cuda").manual_seed(0)
    w_in = 50.0 * torch.randn(3, n, dtype=torch.float64, device="cuda", generator=gen)
    w_out = torch.empty_like(w_in)
    dt = args_dt
    res = {}
    def sfc_collide():
        ctx.set_pair_policy("sfc_first")
        ctx.collide(state, dst, dt)
        ctx.set_pair_policy("earliest")

    for kind, call in (("collide", lambda: ctx.collide(state, dst, dt)),
                       ("collide_rot", lambda: ctx.collide_rot(state, dst, w_in, w_out, 0.3, dt)),
                       ("collide_sfc", sfc_collide)):
        for _ in range(max(3, args.warmup)):
            call()
        ctx.sync()
        ctx.set_timing(True)
        ctx.timing()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            call()
        ev1.record(stream)
        torch.cuda.synchronize()
        ph = ctx.timing()
        ctx.set_timing(False)
        if ctx.stats()["status"] != 0:
            raise RuntimeError("device status during the %s step" % kind)
        res[kind] = {"ms_per_call": round(ev0.elapsed_time(ev1) / args.steps, 4),
                     "respond_ms": round(ph["respond"][0] / max(ph["respond"][1], 1), 4)}
    out["friction"] = dict(res["collide_rot"], mu=0.3, frictionless_ms_per_call=res["collide"]["ms_per_call"],
                           frictionless_respond_ms=res["collide"]["respond_ms"])
    out["sfc_first_pairs"] = {"ms_per_call": res["collide_sfc"]["ms_per_call"],
                              "earliest_contact_ms_per_call": res["collide"]["ms_per_call"]}
    # fluid -> particle coupling: a 4-variable field (rho, u) evaluated at every particle,
    # then the drag sources (the inputs of the projection in a two-way coupled step)
    fl = torch.randn(nel, 4, nodes, dtype=torch.float64, device="cuda", generator=gen)
    fluid = torch.empty(4, n, dtype=torch.float64, device="cuda")
    qd = torch.empty(4, n, dtype=torch.float64, device="cuda")
    for _ in range(max(3, args.warmup)):
        ctx.eval_field(state, fl, fluid)
        ctx.drag_sources(state, fluid, 1.8e-5, qd)
    ctx.sync()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    t_eval = t_drag = 0.0
    for _ in range(args.steps):
        evs[0].record(stream)
        ctx.eval_field(state, fl, fluid)
        evs[1].record(stream)
        ctx.drag_sources(state, fluid, 1.8e-5, qd)
        evs[2].record(stream)
        torch.cuda.synchronize()
        t_eval += evs[0].elapsed_time(evs[1])
        t_drag += evs[1].elapsed_time(evs[2])
    if ctx.stats()["status"] != 0:
        raise RuntimeError("device status during the field evaluation")
    out["coupling"] = {"eval_field_ms_per_call": round(t_eval / args.steps, 4), "nvar": 4,
                       "drag_sources_ms_per_call": round(t_drag / args.steps, 4)}
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_project_chunk(args):
    """Pool worker: the oracle's projection of one chunk of particles (returns a checksum
    so that the field is not shipped back)."""
    import oracle
    x, q, ne, degree, sigma, cutoff_sigmas = args
    F, _ = oracle.project(x, q, ne, degree, sigma, cutoff_sigmas)
    return float(F.sum())


class OraclePool:
    """A spawn-started process pool over the host's cores that runs the oracle's projection
    on disjoint chunks of a particle sample. The projection is a sum over particles, so the
    chunks are independent; the oracle itself is unchanged (single-threaded C)."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_project_chunk, [(np.full((3, 1), 0.5), np.ones((4, 1)), 3, 0, 0.05, 3.0)] * self.procs)

    def project(self, x, q, wl):
        chunks = np.array_split(np.arange(x.shape[1]), self.procs)
        jobs = [(np.ascontiguousarray(x[:, c]), np.ascontiguousarray(q[:, c]), wl.ne, wl.degree, wl.sigma,
                 wl.cutoff_sigmas) for c in chunks if len(c)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_project_chunk, jobs)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_sample(w, wl, pool, frac_project=16):
    """Oracle wall time for one step over the workload: the full collide step (the
    oracle's candidate search and global greedy matching, single thread), and the
    projection of every frac_project-th particle spread over the pool's processes,
    scaled by frac_project."""
    import oracle
    t0 = time.perf_counter()
    oracle.collide_step(w["x"], w["v"], w["r"], w["m"], w["id"], w["e"], w["dt"])
    t1 = time.perf_counter()
    sel = slice(0, None, frac_project)
    tp = pool.project(w["x"][:, sel], w["q"][:, sel], wl)
    return (t1 - t0) + frac_project * tp, t1 - t0, tp


def cpu_baseline(w, wl):
    n = w["x"].shape[1]
    pool = OraclePool()
    try:
        tot, tc, tp = cpu_sample(w, wl, pool)
    finally:
        pool.close()
    return {"value": n / tot, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "extrapolated": True,
            "sample_fraction_project": 1.0 / 16, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": "one full collide step over all %d particles (%.2f s, single thread: the oracle's greedy "
                      "matching is sequential) + projection of every 16th particle over %d processes (%.2f s wall, "
                      "scaled x16), FP64 C oracle" % (n, tc, pool.procs, tp)}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    wl = inputs.WORKLOADS[args.workload]
    w = inputs.draw(args.workload, seed=0)
    n = w["x"].shape[1]
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            cpu_sample(w, wl, pool, frac_project=64)
        times = []
        for _ in range(args.steps):
            times.append(cpu_sample(w, wl, pool, frac_project=64)[0])
    finally:
        pool.close()
    tot = float(np.sum(times))
    value = n * args.steps / tot
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(args, w, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "extrapolated": True, "sample_fraction_project": 1.0 / 64, "nproc": os.cpu_count(),
                             "cpu_model": cpu_model(),
                             "sample": "per step: one full collide step over all %d particles (single thread) + "
                                       "projection of every 64th particle over %d processes, its wall time "
                                       "scaled x64; FP64 C oracle" % (n, pool.procs)},
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
