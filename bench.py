#!/usr/bin/env python
"""Benchmark of the WU-VKLB step (weighted upwind vector kinetic lattice
Boltzmann, fused collide-and-stream) on B300.

Default workload: 2D Euler isentropic vortex (gamma 1.4, strength 5, background
rho = p = 1, velocity (1, 1)) on a periodic [0, 10]^2 grid of 1024^2 cells, D2Q5,
4 conserved fields, FP32 distributions, omega = 2, CFL 0.3, c = 0.05, k = 2.
A bench step is one time step of Fig. 5 (one kernel launch).  Each timed step is
bracketed by CUDA events on the simulation's stream, after an L2 flush (the
84 MB state would otherwise stay partly L2-resident): a 256 MiB write, then a
256 MiB read of another buffer, so that the flush's own dirty lines are written
back before the step starts rather than inside it.  Every
200 steps the state is re-initialised outside the timed events: at omega = 2 the
weighted set amplifies rounding (FP32 stays within 1 % of the FP64 error against
the exact solution to about 1,000 steps of this vortex, and one period takes
10^4), so the timed steps always advance a state of the paper's problem.

--impl reference times the FP64 CPU oracle (oracle/, test infrastructure) on the
host cores on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload euler_vortex_1024|mhd_orszag_tang_2048] [--no-extras] [--no-cpu-baseline]
       [--timed-only]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2608_04283_b300 import inputs  # noqa: E402

WORKLOADS = {
    "euler_vortex_1024": dict(
        system="euler", n=(1024, 1024), lo=(0.0, 0.0), hi=(10.0, 10.0),
        kw=dict(omega=2.0, cfl=0.3, c=0.05, k=2.0, gamma=1.4),
        ic=lambda: inputs.isentropic_vortex(1024),
        name="2D Euler isentropic vortex 1024x1024, periodic [0,10]^2, D2Q5, 4 fields, omega 2, CFL 0.3"),
    "mhd_orszag_tang_2048": dict(
        system="mhd_glm", n=(2048, 2048), lo=(0.0, 0.0), hi=(2 * np.pi, 2 * np.pi),
        kw=dict(omega=1.0, cfl=0.3, c=0.05, k=2.0, gamma=5.0 / 3.0, ch_factor=6.0),
        ic=lambda: inputs.orszag_tang(2048),
        name="2D ideal MHD-GLM Orszag-Tang 2048x2048, periodic [0,2pi]^2, D2Q5, 9 fields, omega 1, CFL 0.3"),
}
REINIT_EVERY = 200
FLUSH_BYTES = 256 << 20
NOMINAL_HBM_GBS = 8000.0   # nominal B300 HBM3e bandwidth (8 TB/s), beside the measured copy peak


# the device code the step kernels compile from: DRAM traffic recorded by a
# profile stays valid while these are unchanged (host files do not matter)
KERNEL_SOURCES = ("vk_ctl.cuh", "vk_kernels.cuh", "vk_math.cuh", "vk_systems.cuh")


def csrc_hash():
    """Hash of the kernel sources' code: comments and blank lines are left out,
    so editing a comment does not invalidate a recorded profile."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2608_04283_b300", "csrc")
    for f in KERNEL_SOURCES:
        for line in open(os.path.join(d, f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def tiling_for(system, precision, n):
    tab = json.load(open(os.path.join(ROOT, "paper_2608_04283_b300", "tuning.json")))
    ent = tab.get(f"{system}/{precision}")
    if not ent:
        return None
    side = max(n)
    best = min(ent.keys(), key=lambda k: abs(int(k) - side))
    return tuple(ent[best])


def launch_shape(system, precision, n):
    """(tile, (variant, stages)) the autotuner measured best for the nearest grid
    side, or None for the library's defaults."""
    tile = tiling_for(system, precision, n)
    if tile is None:
        return None
    tab = json.load(open(os.path.join(ROOT, "paper_2608_04283_b300", "tuning.json")))
    var = (0, 0)
    vt = {k: v for k, v in tab.get("_variants", {}).items() if k.startswith(f"{system}/{precision}/")}
    if vt:
        side = max(n)
        best = min(vt.keys(), key=lambda k: abs(int(k.rsplit("/", 1)[1]) - side))
        if int(best.rsplit("/", 1)[1]) == int(min(tab[f"{system}/{precision}"].keys(), key=lambda k: abs(int(k) - side))):
            var = tuple(vt[best])
    return tile, var


def configure(sim, shape):
    if shape is None:
        return
    tile, var = shape
    sim.set_tiling(64, 8)          # a shape every variant accepts
    sim.set_variant(*var)
    sim.set_tiling(*tile)          # the wave-fit height depends on the variant


# systems whose FP32-compute step kernel has a register-bounded instantiation
# (taken for blocks of at most 128 threads)
BOUNDED_STEP = ("mhd_glm", "euler")


def step_kernel_name(system, prec, tile_x, variant, form=0):
    """The step kernel the library launches: the bulk-copy variant, or the plain
    one (moment form: step2d_u_kernel), which FP32-compute MHD-GLM and Euler
    with blocks of at most 128 threads take in their register-bounded
    instantiation."""
    if variant == 1:
        return "step2d_tma_kernel"
    if system in BOUNDED_STEP and prec != "fp64" and tile_x <= 128:
        return "step2d_lb_kernel"
    return "step2d_u_kernel" if form == 1 else "step2d_kernel"


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def traffic_record(kernel_key):
    """Per-launch DRAM bytes of the step kernel from a committed ncu summary,
    valid only while the kernel sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel_key)
    if not e or e.get("csrc_hash") != csrc_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_throughput(torch, local_ms, cells, steps, world, device):
    """Whole-job MLUPS of `world` independent replicas (weak scaling: every rank
    steps its own copy of the workload): the slowest rank's timed region, taken
    by a MAX all-reduce, bounds the job.  Returns (MLUPS, max ms)."""
    ms = float(local_ms)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return world * cells * steps / (ms * 1e-3) / 1e6, ms


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- oracle arm
def blas_threads():
    """Threads numpy's BLAS may use for the oracle (its batched solves and
    products are the only multi-threaded parts)."""
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(var):
                return int(os.environ[var])
        return os.cpu_count() or 1

L2_NOTE = "GPU arm: L2 flushed before every timed step (256 MiB write, then 256 MiB read of another buffer)"


def workload_config(args, wl, world):
    """The workload both arms run, identical in their lines; each arm's own
    details (launch shape and precision, or the oracle's sample) sit beside it."""
    return {"workload": args.workload, "description": wl["name"], "cells": wl["n"][0] * wl["n"][1],
            "form": args.form, "l2": L2_NOTE, "reinit_every": REINIT_EVERY,
            "parallelism": "replicas" if world > 1 else "single"}


def oracle_mlups(wl, rows, steps, warmup):
    """The FP64 oracle as it stands on a bounded sample: a strip of ``rows`` rows
    of the workload grid (periodic), one oracle step per bench step."""
    from oracle import systems as osys
    from oracle import vklb as ovklb
    nx = wl["n"][0]
    U = np.ascontiguousarray(wl["ic"]()[:, :rows, :])
    dx = (wl["hi"][0] - wl["lo"][0]) / nx
    kw = wl["kw"]
    if wl["system"] == "euler":
        sysm = osys.Euler(kw["gamma"], 2)
    else:
        sysm = osys.MHDGLM(kw["gamma"])
    sim = ovklb.Sim(sysm, (nx, rows), (0.0, 0.0), (nx * dx, rows * dx), omega=kw["omega"], nu=kw["cfl"],
                    c=kw["c"], k=kw["k"], ch_factor=kw.get("ch_factor", 6.0))
    sim.set_state(U)
    sim.run(warmup)
    t0 = time.perf_counter()
    sim.run(steps)
    dt = time.perf_counter() - t0
    threads = blas_threads()
    return nx * rows * steps / dt / 1e6, dt, threads


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # strip height chosen so the whole run stays near 90 s of oracle work
    # (the oracle does about 1.1e-5 s per Euler cell update on one host)
    per_cell = 1.1e-5 if wl["system"] == "euler" else 2.5e-5
    rows = int(90.0 / (args.steps + args.warmup) / (wl["n"][0] * per_cell))
    rows = max(1, min(64, rows))
    val, dt, threads = oracle_mlups(wl, rows, args.steps, args.warmup)
    sample = f"{rows} x {wl['n'][0]} strip of the {wl['n'][0]}^2 grid per step, {args.steps} timed steps"
    line = {"metric": "MLUPS", "value": val, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args, wl, world),
            "launch": {"where": "host cores", "threads": threads, "precision": "fp64", "sample": sample},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- CUDA arm
class L2Flush:
    """Evicts L2 between timed steps: writes a buffer larger than L2, then reads
    a second one, leaving L2 full of clean lines the step does not use."""

    def __init__(self, torch, nbytes=FLUSH_BYTES):
        self.w = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
        self.acc = torch.zeros((), dtype=torch.float32, device="cuda")

    def __call__(self, i):
        self.w.fill_(i & 0xFF)
        self.acc.copy_(self.r.amax())


def timed_steps(torch, sim, stream, U0_dev, steps, warmup, flush, reinit_every=REINIT_EVERY):
    """Per-step event timing on the simulation's stream; L2 flushed before each step."""
    sim.set_state(U0_dev)
    with torch.cuda.stream(stream):
        for i in range(warmup):
            flush(i)
            sim.step(1)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            if i > 0 and i % reinit_every == 0:
                sim.set_state(U0_dev)
            flush(i)
            ev0[i].record(stream)
            sim.step(1)
            ev1[i].record(stream)
    torch.cuda.synchronize()
    durs = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])   # ms
    return durs


def run_ours(args, wl):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2608_04283_b300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2608_04283_b300 import vklb

    prec = args.precision
    stream = torch.cuda.Stream()
    sim = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision=prec, stream=stream, form=args.form,
                   **wl["kw"])
    tile = launch_shape(wl["system"], prec, wl["n"]) if args.form == "distributions" else None
    configure(sim, tile)
    U0 = wl["ic"]()
    U0_dev = torch.from_numpy(U0).cuda()
    flush_buf = L2Flush(torch)
    cells = wl["n"][0] * wl["n"][1]
    bpl = sim.info.bytes_per_lup

    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = vklb.launch_count()
    durs = timed_steps(torch, sim, stream, U0_dev, args.steps, args.warmup, flush_buf)
    l1 = vklb.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(durs.sum())
    value, total_ms = replica_throughput(torch, total_ms, cells, args.steps, world, "cuda")
    mean_ms = total_ms / args.steps
    achieved = bpl * cells / (mean_ms * 1e-3) / 1e9
    peaks, peak_src = measured_peaks()
    kname = step_kernel_name(wl["system"], prec, sim.info.tile_x, sim.info.variant, sim.info.form)
    key = f"{kname}/{wl['system']}/{prec}/{wl['n'][0]}x{wl['n'][1]}/{sim.info.tile_x}x{sim.info.tile_y}"
    traffic = traffic_record(key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peak_src + " (burst)",
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "algorithmic_bytes_per_lup": bpl, "kernel": kname}

    extras = {}
    acc = None
    acc_exact = None
    e2e = None
    cpu = None
    if rank == 0 and not args.timed_only:
        acc = accuracy_vs_fp64(torch, vklb, wl, prec, tile, steps=50, form=args.form)
        acc_exact = accuracy_vs_exact(vklb, prec) if prec != "fp64" else None
        e2e = end_to_end(torch, vklb, wl, prec, tile, steps=min(args.steps, REINIT_EVERY), U0=U0, form=args.form)
        if not args.no_extras:
            extras["copy_same_bytes"] = copy_same_bytes(torch, bpl * cells, flush_buf)
        if not args.no_extras and args.workload == "euler_vortex_1024":
            extras["mhd_orszag_tang_2048"] = secondary(torch, vklb, WORKLOADS["mhd_orszag_tang_2048"], prec,
                                                       flush_buf, steps=100)
            extras["moment_form"] = moment_form(torch, vklb, flush_buf)
            extras["batched_swe_256"] = batched_swe(torch, vklb)
            extras["batched_swe_256_moment_form"] = batched_swe(torch, vklb, form="moments")
            extras["served_mix"] = served_mix(args.served_requests)
            extras["served_paced"] = served_paced()
        if world == 1 and not args.no_cpu_baseline:
            v, dt, threads = oracle_mlups(wl, wl["n"][1], 1, 0)
            cpu = {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                   "sample": f"one oracle step of the full {wl['n'][0]}x{wl['n'][1]} grid ({dt:.1f} s)"}
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16-store/f32"}[prec],
                "data": "synthetic",
                "config": workload_config(args, wl, world),
                "launch": {"where": "cuda", "precision": prec, "tile": [sim.info.tile_x, sim.info.tile_y],
                           "variant": sim.info.variant},
                "hbm_gbs": achieved, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(l1 - l0), "clocks": clk, "accuracy_fp32_vs_fp64": acc,
                "accuracy_fp32_vs_exact": acc_exact,
                "step_ms": {"median": float(np.median(durs)), "p10": float(np.percentile(durs, 10)),
                            "p90": float(np.percentile(durs, 90))},
                "extras": extras}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def accuracy_vs_fp64(torch, vklb, wl, prec, tile, steps, form="distributions"):
    """L1 / Linf of the benchmarked precision against the FP64 CUDA path (which the
    parity tests tie to the oracle at <= 1e-11) after ``steps`` steps."""
    if prec == "fp64":
        return None
    U0 = wl["ic"]()
    out = {}
    res = []
    for p in (prec, "fp64"):
        s = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision=p, form=form, **wl["kw"])
        if p == prec:
            configure(s, tile)
        s.set_state(U0)
        s.step(steps)
        res.append(s.moments())
        s.close()
    a, b = res
    ch = None
    if wl["system"] == "mhd_glm":
        ch = wl["kw"]["ch_factor"] * mhd_max_fast_speed(b, wl["kw"]["gamma"])
    l1 = rel_norm(a, b, lambda x: np.abs(x).sum(), ch)
    linf = rel_norm(a, b, lambda x: np.abs(x).max(), ch)
    out["steps"] = steps
    out["rel_l1_per_field"] = [float(v) for v in l1]
    out["rel_linf_per_field"] = [float(v) for v in linf]
    out["rel_l1_max_field"] = float(l1.max())
    out["rel_linf_max_field"] = float(linf.max())
    out["rule"] = ("per field |a - b| / |b|; MHD-GLM's m_z, B_z and psi (zero or at rounding level in "
                   "Orszag-Tang) against the terms that carry them: |m|, |B| and c_h |B|")
    return out


def mhd_max_fast_speed(U, gamma):
    """Largest fast magnetosonic speed over the grid and both directions."""
    rho = U[0]
    bb = U[5] ** 2 + U[6] ** 2 + U[7] ** 2
    p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho - 0.5 * bb)
    a2, b2 = gamma * p / rho, bb / rho
    best = 0.0
    for d in (0, 1):
        bn2 = U[5 + d] ** 2 / rho
        cf = np.sqrt(0.5 * (a2 + b2 + np.sqrt(np.maximum((a2 + b2) ** 2 - 4.0 * a2 * bn2, 0.0))))
        best = max(best, float(cf.max()))
    return best


def rel_norm(a, b, norm, ch=None):
    """Per-field norm of a - b relative to b's.  For MHD-GLM (ch given) the
    fields Orszag-Tang keeps at zero or at rounding level take the scale of the
    terms that carry them: m_z that of |m|, B_z that of |B|, psi that of c_h |B|
    (its distribution components carry the cleaning waves' c_h B_n / 2)."""
    scale = [norm(b[k]) for k in range(b.shape[0])]
    if ch is not None:
        m = np.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2)
        B = np.sqrt(b[5] ** 2 + b[6] ** 2 + b[7] ** 2)
        scale[3] = max(scale[3], norm(m))
        scale[7] = max(scale[7], norm(B))
        scale[8] = max(scale[8], ch * norm(B))
    return np.array([norm(a[k] - b[k]) / scale[k] for k in range(b.shape[0])])


def accuracy_vs_exact(vklb, prec, n=128, T=2.0):
    """Error against the exact solution (the vortex translated by (T, T), Eq. 57)
    of the benchmarked precision and of the FP64 path, L1 and L-infinity per
    field, at the paper's vortex setting (omega 2, CFL 0.3, T = 2) and the
    largest side at which FP32 can meet 1 % of FP64's error (omega = 2 amplifies
    rounding; tests/test_gpu_accuracy_exact.py)."""
    wl = WORKLOADS["euler_vortex_1024"]
    ex = inputs.isentropic_vortex(n, shift=(T, T))
    out = {"workload": f"Euler vortex {n}x{n}, omega 2, CFL 0.3, T = {T}"}
    errs = {}
    for p in (prec, "fp64"):
        s = vklb.Sim("euler", (n, n), wl["lo"], wl["hi"], precision=p, **wl["kw"])
        s.set_state(inputs.isentropic_vortex(n))
        s.step_to(T)
        d = np.abs(s.moments() - ex).reshape(4, -1)
        s.close()
        errs[p] = (d.mean(axis=1), d.max(axis=1))
    out[f"{prec}_l1"] = [float(v) for v in errs[prec][0]]
    out[f"{prec}_linf"] = [float(v) for v in errs[prec][1]]
    out["fp64_l1"] = [float(v) for v in errs["fp64"][0]]
    out["fp64_linf"] = [float(v) for v in errs["fp64"][1]]
    out["max_rel_diff_l1"] = float(np.max(np.abs(errs[prec][0] - errs["fp64"][0]) / errs["fp64"][0]))
    out["max_rel_diff_linf"] = float(np.max(np.abs(errs[prec][1] - errs["fp64"][1]) / errs["fp64"][1]))
    out["within_1pct"] = bool(max(out["max_rel_diff_l1"], out["max_rel_diff_linf"]) <= 0.01)
    return out


def end_to_end(torch, vklb, wl, prec, tile, steps, U0, form="distributions", solves=8):
    """Through the public API with host buffers, wall clock.  A solve is the H2D
    of U0 from pinned memory, vklb_set_state, ``steps`` x vklb_step, vklb_moments
    and the D2H of U to pinned memory.

    value: a stream of ``solves`` solves in two slots (two simulations on their
    own streams, device staging buffers, copies on two copy streams), so that
    one slot's copies overlap the other's steps; every solve still moves its
    bytes across PCIe inside the timed region.  serial_value: one solve alone,
    host buffers passed to the API directly (nothing overlaps)."""
    pin_in = torch.empty(U0.shape, dtype=torch.float64, pin_memory=True)
    pin_in.numpy()[...] = U0
    host_in = pin_in.numpy()
    pin_out = [torch.empty(U0.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    cells = wl["n"][0] * wl["n"][1]

    # one solve alone
    s = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision=prec, form=form, **wl["kw"])
    configure(s, tile)
    s.set_state(host_in)
    s.step(2)
    s.moments(out=pin_out[0].numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(host_in)
    s.step(steps)
    s.moments(out=pin_out[0].numpy())
    serial = cells * steps / (time.perf_counter() - t0) / 1e6
    want = pin_out[0].numpy().copy()
    s.close()

    # a stream of solves in two slots
    streams = [torch.cuda.Stream() for _ in range(2)]
    cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
    sims = []
    for k in range(2):
        sk = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision=prec, form=form, stream=streams[k],
                      **wl["kw"])
        configure(sk, tile)
        sims.append(sk)
    dev_in = [torch.empty(U0.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    dev_out = [torch.empty(U0.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    ev = lambda: [torch.cuda.Event() for _ in range(2)]
    ev_in, ev_used, ev_done, ev_out = ev(), ev(), ev(), ev()

    def run(n_solves):
        for i in range(n_solves + 1):
            if i < n_solves:
                k = i % 2
                cin.wait_event(ev_used[k])            # set_state of solve i - 2 has read dev_in[k]
                with torch.cuda.stream(cin):
                    dev_in[k].copy_(pin_in, non_blocking=True)
                ev_in[k].record(cin)
                streams[k].wait_event(ev_in[k])
                sims[k].set_state(dev_in[k])
                ev_used[k].record(streams[k])
                sims[k].step(steps)
            if i >= 1:
                j = (i - 1) % 2
                streams[j].wait_event(ev_out[j])      # D2H of solve i - 3 has read dev_out[j]
                sims[j].moments(out=dev_out[j])       # waits for solve i - 1; solve i is queued
                ev_done[j].record(streams[j])
                cout.wait_event(ev_done[j])
                with torch.cuda.stream(cout):
                    pin_out[j].copy_(dev_out[j], non_blocking=True)
                ev_out[j].record(cout)
        torch.cuda.synchronize()

    run(2)
    t0 = time.perf_counter()
    run(solves)
    dt = time.perf_counter() - t0
    same = all(np.array_equal(pin_out[k].numpy(), want) for k in range(2))
    for sk in sims:
        sk.close()
    return {"value": solves * cells * steps / dt / 1e6, "unit": "MLUPS", "results_equal_serial": bool(same),
            "h2d_bytes_per_step": int(U0.nbytes / steps), "d2h_bytes_per_step": int(U0.nbytes / steps),
            "steps_per_solve": steps, "solves": solves, "serial_value": serial,
            "note": "one solve = H2D of U0 (pinned), set_state, the steps, moments, D2H of U (pinned); bytes "
                    "amortised per step; value: solves in two slots (copies of one overlap the steps of the "
                    "other); serial_value: one solve alone"}


def copy_same_bytes(torch, nbytes, flush_buf, reps=50):
    """A plain device copy moving the step's bytes (nbytes / 2 read, nbytes / 2
    written), L2 flushed before each copy as before each step: the bandwidth a
    streaming kernel of this size reaches, beside the large-copy peak."""
    n = nbytes // 2 // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    st = torch.cuda.current_stream()
    for i in range(5):
        b.copy_(a)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for i in range(reps):
        flush_buf(i)
        ev[i][0].record(st)
        b.copy_(a)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    ms = float(np.mean([x.elapsed_time(y) for x, y in ev]))
    return {"bytes": int(2 * n * 4), "ms": ms, "gbs": 2 * n * 4 / (ms * 1e-3) / 1e9,
            "note": "torch copy of the step's algorithmic bytes, L2 flushed before each copy"}


def moment_form(torch, vklb, flush_buf, steps=100):
    """omega = 1 workloads in both state forms (vklb_set_form), L2 flushed before
    every timed step: distributions at the autotuned launch shape, moments at
    128-cell rows of wave-fit height.  GB/s counts each form's own algorithmic
    bytes (2 x 5p x 4 B a cell for f, 2 x p x 4 B for U)."""
    out = {}
    cases = [("mhd_orszag_tang_2048", WORKLOADS["mhd_orszag_tang_2048"]),
             ("swe_hump_1024", dict(system="swe", n=(1024, 1024), lo=(0.0, 0.0), hi=(1.0, 1.0),
                                    kw=dict(omega=1.0, cfl=0.3, c=0.05, k=2.0),
                                    ic=lambda: inputs.swe_hump_2d(1024, 0.5, 0.5, 0.5, 0.08)))]
    peaks, _ = measured_peaks()
    for name, wl in cases:
        row = {}
        U0 = torch.from_numpy(wl["ic"]()).cuda()
        cells = wl["n"][0] * wl["n"][1]
        for form in ("distributions", "moments"):
            stream = torch.cuda.Stream()
            s = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision="fp32", stream=stream, form=form,
                         **wl["kw"])
            if form == "distributions":
                configure(s, launch_shape(wl["system"], "fp32", wl["n"]))
            ms = float(timed_steps(torch, s, stream, U0, steps, 5, flush_buf).mean())
            gbs = s.info.bytes_per_lup * cells / (ms * 1e-3) / 1e9
            row[form] = {"ms_per_step": ms, "MLUPS": cells / (ms * 1e-3) / 1e6, "hbm_gbs": gbs,
                         "frac_of_peak": gbs / peaks["hbm_gbs"], "bytes_per_lup": s.info.bytes_per_lup,
                         "tile": [s.info.tile_x, s.info.tile_y]}
            s.close()
        row["speedup"] = row["distributions"]["ms_per_step"] / row["moments"]["ms_per_step"]
        out[name] = row
    return out


def secondary(torch, vklb, wl, prec, flush_buf, steps):
    stream = torch.cuda.Stream()
    s = vklb.Sim(wl["system"], wl["n"], wl["lo"], wl["hi"], precision=prec, stream=stream, **wl["kw"])
    configure(s, launch_shape(wl["system"], prec, wl["n"]))
    U0 = torch.from_numpy(wl["ic"]()).cuda()
    durs = timed_steps(torch, s, stream, U0, steps, 5, flush_buf)
    cells = wl["n"][0] * wl["n"][1]
    mean_ms = float(durs.mean())
    bpl = s.info.bytes_per_lup
    peaks, src = measured_peaks()
    gbs = bpl * cells / (mean_ms * 1e-3) / 1e9
    s.close()
    return {"workload": wl["name"], "MLUPS": cells / (mean_ms * 1e-3) / 1e6, "ms_per_step": mean_ms,
            "hbm_gbs": gbs, "frac_of_peak": gbs / peaks["hbm_gbs"], "bytes_per_lup": bpl,
            "tile": [s.info.tile_x, s.info.tile_y], "variant": s.info.variant, "steps": steps}


# Launch shape of the batched shallow-water leg, measured on B300 over the
# 256-instance batch (sides 64..1024): distributions 128 x 8 (47.4 G cell
# updates/s; 64 x fitted: 36.8 G, its x-ring reads doubling the DRAM reads),
# moments 64 x fitted (98.1 G; 128 x 8: 83.5 G).
BATCH_TILES = {"distributions": (128, 8), "moments": (64, -1)}


def batched_swe(torch, vklb, count=256, steps=500, form="distributions"):
    """Batched form: 256 seeded SWE instances (sides 64..1024, Gaussian humps),
    500 steps each, one launch per step over all instances (CUDA graph), against
    the same instances launched one at a time, each at the autotuned tiling of
    its nearest grid side.  Reports solves/s."""
    specs = inputs.swe_humps_batch(count, seed=0)
    tile = BATCH_TILES[form]
    stream = torch.cuda.Stream()
    sims = []
    U0s = []
    for sp in specs:
        s = vklb.Sim("swe", (sp.n, sp.n), (0, 0), (1, 1), omega=1.0, cfl=0.3, precision="fp32", stream=stream,
                     form=form)
        s.set_tiling(*(tiling_for("swe", "fp32", (sp.n, sp.n)) or (128, -1)))
        U0 = torch.from_numpy(inputs.swe_hump_2d(sp.n, sp.amp, sp.x0, sp.y0, sp.sigma)).cuda()
        U0s.append(U0)
        sims.append(s)
    cells = sum(sp.n * sp.n for sp in specs)
    for s, U in zip(sims, U0s):
        s.set_state(U)
    b = vklb.Batch(sims, tile=tile)
    b.step(5, graph=True)          # warm-up (graph capture of 5 steps)
    torch.cuda.synchronize()
    for s, U in zip(sims, U0s):
        s.set_state(U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps, graph=True)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    batch_out = [sims[i].moments() for i in (0, count // 2, count - 1)]
    for s, U in zip(sims, U0s):
        s.set_state(U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in sims:
        s.step(steps)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    plain_out = [sims[i].moments() for i in (0, count // 2, count - 1)]
    # each instance alone takes its own wave-fit height, the batch one height
    # fitted to its whole work-list: the tilings differ, so the two agree to
    # FP32 rounding (the batch of one is bitwise equal to the batch of many,
    # which the GPU tests check)
    diff = max(float(np.abs(a - c).sum() / np.abs(c).sum()) for a, c in zip(batch_out, plain_out))
    b.close()
    for s in sims:
        s.close()
    return {"instances": count, "steps": steps, "cells_total": cells, "tile": list(tile),
            "plain_tiles": "autotuned per nearest grid side", "form": form,
            "batched_solves_per_s": count / tb, "plain_solves_per_s": count / tp,
            "batched_MLUPS": cells * steps / tb / 1e6, "plain_MLUPS": cells * steps / tp / 1e6,
            "speedup": tp / tb, "batched_vs_plain_rel_l1": diff,
            "note": "wall clock incl. launch; batched = one launch per step over all instances in one CUDA graph"}


def served_mix(count, budget=120e9):
    """Served form: the first ``count`` requests of the seeded serving trace
    (Poisson arrivals at 200/s; SWE / Euler / MHD-GLM; sides 128..2048; 100..2000
    steps; FP32) through the continuous-batching server under a 120 GB budget,
    against the same requests run one at a time (one launch per step).  Each
    request's analytic initial data (system, side, phases) is evaluated on the
    device in both runs (2,000 host-side states would hold about 130 GB)."""
    from paper_2608_04283_b300 import serve
    trace = inputs.serving_trace(count=count)
    srv = serve.Server(budget_bytes=budget, tick_steps=50, device_ic=True)
    # untimed warm-up of every family's kernels (the one-at-a-time run below
    # comes after the server's, so it is warm too)
    srv.run(inputs.serving_trace(count=6, seed=9, nmin=128, nmax=128, smin=10, smax=10), realtime=False)
    rep = srv.run(trace, realtime=True)
    out = rep.summary()
    out["peak_device_gb"] = rep.peak_bytes / 1e9
    out["budget_gb"] = budget / 1e9
    out["admitted_later_than_50ms"] = int(sum(j.t_admit - j.req.arrival > 0.05 for j in rep.jobs))
    plain = serve.run_plain(trace, device_ic=True)
    out["plain_solves_per_s"] = plain["solves_per_s"]
    out["plain_MLUPS"] = plain["MLUPS"]
    out["speedup_solves"] = out["solves_per_s"] / plain["solves_per_s"]
    out["note"] = ("latency = finish - arrival on the wall clock; initial states built on the device from the "
                   "request in both runs; results read back through pinned host buffers in both runs; the "
                   "200/s arrival rate overloads the GPU (about 1.5 G cell updates per request), so latency is "
                   "dominated by queueing (queue_* = admission - arrival)")
    return out


def served_paced(count=24, rate=3.0):
    """Served form below saturation: ``count`` requests of the same mix arriving
    at ``rate`` per second (Poisson, seed 1), so p50 / p99 are service latency
    rather than queueing."""
    from paper_2608_04283_b300 import serve
    trace = inputs.serving_trace(count=count, rate=rate, seed=1)
    payloads = {r.rid: inputs.request_initial_state(r) for r in trace}
    srv = serve.Server(budget_bytes=120e9, tick_steps=50)
    rep = srv.run(trace, realtime=True, payloads=payloads)
    out = rep.summary()
    out["arrival_rate_per_s"] = rate
    out["peak_device_gb"] = rep.peak_bytes / 1e9
    out["note"] = "latency = finish - arrival on the wall clock, arrivals paced below the GPU's capacity"
    return out


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="euler_vortex_1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="distributions", choices=["distributions", "moments"],
                    help="state form of the timed simulation (moments: omega = 1 workloads only)")
    ap.add_argument("--timed-only", action="store_true",
                    help="only the warm-up and timed steps (no accuracy check, end-to-end run, extras or CPU "
                         "baseline): the launch list of a profile then holds just the timed region's kernels")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="requests of the served-form leg (the serving trace has 2,000)")
    ap.add_argument("--only-batched", type=int, default=0, metavar="N",
                    help="run only the batched shallow-water leg with the first N instances (and --form), print "
                         "its JSON and exit: a case small enough to profile")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    return args


def main():
    args = parse_args()
    wl = WORKLOADS[args.workload]
    if args.only_batched > 0:
        import torch
        from paper_2608_04283_b300 import build
        build.build()
        from paper_2608_04283_b300 import vklb
        print(json.dumps(batched_swe(torch, vklb, count=args.only_batched, form=args.form)), flush=True)
    elif args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
