#!/usr/bin/env python3
"""Throughput of the P-LBM time step on GB300 (GLUPS and fraction of the HBM roofline).

Default workload: D3Q19 two-phase flow between parallel plates, 512 x 256 x 256 cells,
halfway bounce-back walls bounding y, periodic in x and z, liquid layers next to both
walls and a vapour core (flat interfaces at y = 63.5 and 191.5), body force 1e-7 along x,
Peng-Robinson EOS at T/Tc = 0.8, MRT collision, FP32 population storage.  Synthetic
seeded input; the populations (2.5 GB) are larger than L2, so no flush is needed.

One step = psi pass + fused force/collide/stream pass over the whole lattice.
Multi-GPU: independent replicas (the workload does not exchange data across GPUs),
weak scaling; value = cells * steps summed over ranks / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16s|fp64]
                  [--collision mrt|bgk] [--dims 512x256x256] [--impl reference] [--no-variants]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P-LBM GLUPS and % HBM roofline, FP32/FP16 vs FP64 at matched Laplace error"
PREC = {"fp64": 0, "fp32": 1, "fp16s": 2, "fp16s_sr": 2}
POP_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2, "fp16s_sr": 2}
PSI_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 4, "fp16s_sr": 4}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f16 storage / f32 arithmetic",
         "fp16s_sr": "f16 storage (stochastic rounding) / f32 arithmetic"}
T_RATIO, BODY_FORCE = 0.8, 1e-7
MRT_RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.4, s_m=1.98)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--precision", default="fp32", choices=list(PREC))
    ap.add_argument("--collision", default="mrt", choices=["mrt", "bgk"])
    ap.add_argument("--streaming", default="aa", choices=["aa", "fused"],
                    help="fused: one kernel per step, two population copies; aa: two kernels, in place")
    ap.add_argument("--dims", default="512x256x256")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="plates", choices=["plates", "batch96"],
                    help="plates: D3Q19 512x256x256 two-phase plates; batch96: 96 uneven D2Q9 instances")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-plan", action="store_true",
                    help="time the FP64 oracle alone on the host cores: D2Q9 BGK 256^2, D3Q19 BGK and MRT 96^3, "
                         "1 thread and all cores, median of 3 (prints one JSON line, no GPU work)")
    ap.add_argument("--cpu-plan-child", default="", help=argparse.SUPPRESS)
    ap.add_argument("--e2e-steps", type=int, default=100,
                    help="steps of the end-to-end run (init from host, steps, fields back to host)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(seconds: float, world: int, device) -> float:
    """The job time of a multi-rank run: the slowest rank's time (all_reduce MAX)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    tt = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_glups(cells_per_rank: int, steps: int, seconds: float, world: int) -> float:
    """Whole-job lattice updates per second (1e9): every rank advances its own replica of
    cells_per_rank cells by steps steps (weak scaling), timed by the slowest rank."""
    return world * cells_per_rank * steps / seconds / 1e9


def workload_name(dims, precision, collision):
    return f"d3q19_plates_{dims[0]}x{dims[1]}x{dims[2]}_{precision}_{collision}_pr0.8"


def bytes_per_cell(precision, q=19, streaming="aa"):
    """Algorithmic bytes per cell update.  Two-pass step: the psi pass reads Q populations and
    writes psi; the fused pass reads Q populations and psi, writes Q.  Single pass: Q
    populations read and Q written (psi stays on chip; halo re-reads are not algorithmic)."""
    sp, sq = POP_BYTES[precision], PSI_BYTES[precision]
    if streaming == "fused":
        return dict(psi_pass=0, fused_pass=2 * q * sp, step=2 * q * sp)
    return dict(psi_pass=q * sp + sq, fused_pass=2 * q * sp + sq, step=3 * q * sp + 2 * sq)


def initial_density(dims, rho_v, rho_l):
    from paper_2504_15018_gb300 import inputs
    return inputs.plates_d3q19(dims, rho_v, rho_l)[1]


def make_lattice(dims, precision, collision, streaming="aa"):
    import paper_2504_15018_gb300 as plb
    eos = plb.pr_eos(T_RATIO)
    opts = plb.make_opts(precision=PREC[precision], collision=plb.PLB_MRT if collision == "mrt" else plb.PLB_BGK,
                         wall_y=1, body_force=(BODY_FORCE, 0.0, 0.0), fp16_rounding=int(precision == "fp16s_sr"),
                         streaming=int(streaming == "fused"), **MRT_RATES)
    return plb.Lattice(plb.PLB_D3Q19, dims, eos, tau=1.0, G=-1.0, eps=2.0, opts=opts)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        # the timed region starts once the first sample is written
        t0 = time.time()
        while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

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
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        smax = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = sm[sm >= np.median(sm) * 0.5] if len(sm) else sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


KERNEL_SOURCES = ("plb_device.cuh", "plb_f2.cuh", "plb_fused.cuh", "plb_kernels.cuh", "plb_moment.cuh", "plb_pair.cuh",
                  "plb_plain.cuh", "plb_staged.cuh", "plb_step.cuh")


def kernel_source_sha():
    """Hash of the files that hold the step kernels' device code (k_psi_pair, k_psi_quad,
    k_collide_pair, k_collide_staged, k_collide_plain, k_fused_pair and everything they inline)
    and their launch shapes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_15018_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, kernel):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    sha = re.search(r"kernel_source_sha:\s*(\w+)", text)
    if not sha or sha.group(1) != kernel_source_sha():
        return None
    m = re.search(re.escape(workload) + r"\s*\|\s*" + re.escape(kernel) + r"\s*\|\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ GPU arm

def time_steps(lat, steps, torch):
    """Device time of `steps` steps with CUDA events on the lattice's stream."""
    st = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    lat.step(steps)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2504_15018_gb300 as plb

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dims = tuple(int(v) for v in args.dims.split("x"))
    ncell = dims[0] * dims[1] * dims[2]
    rho_v, rho_l, _ = plb.plb_solve_params(plb.pr_eos(T_RATIO))
    rho0 = initial_density(dims, rho_v, rho_l)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.precision == "fp64":
        args.streaming = "aa"            # the single pass needs FP32 arithmetic
    lat = make_lattice(dims, args.precision, args.collision, args.streaming)
    lat.init(rho0)
    lat.step(max(args.warmup, 3))
    lat.status()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    t = time_steps(lat, args.steps, torch)
    barrier()
    clocks = sampler.stop()
    lat.status()
    t = max_over_ranks(t, world, "cuda")
    value = job_glups(ncell, args.steps, t, world)

    # roofline of the dominant kernel (fused pass), per-launch events on the same stream
    nprof = min(args.steps, 20)
    ms_psi, ms_fused = lat.step_timed(nprof)
    bpc = bytes_per_cell(args.precision, streaming=args.streaming)
    fused_gbs = bpc["fused_pass"] * ncell * nprof / (ms_fused / 1e3) / 1e9
    peak, peak_kind = peak_hbm()
    wl = workload_name(dims, args.precision, args.collision)
    if args.streaming == "fused":
        kernel = "k_fused_pair (psi of tile + halo in shared memory, force, collide, push stream)"
    elif args.precision in ("fp16s", "fp16s_sr"):
        kernel = ("k_collide_staged (fused force + collide + stream, next plane staged in shared memory, "
                  "moment-space collision)")
    elif args.precision == "fp64":
        kernel = "k_collide_plain (fused force + collide + stream, FP64 in the equations' order)"
    else:
        kernel = "k_collide_pair (fused force + collide + stream)"
    traffic = recorded_traffic(wl, kernel.split()[0])
    roofline = {"bound": "hbm", "kernel": kernel,
                "achieved": round(fused_gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(fused_gbs / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": bpc["fused_pass"] * ncell,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "step_gbs": round(value / world * bpc["step"], 1),
                "step_frac": round(value / world * bpc["step"] / peak, 4),
                "time_share_fused": round(ms_fused / (ms_fused + ms_psi), 3)}
    if ms_psi > 0:
        psi_gbs = bpc["psi_pass"] * ncell * nprof / (ms_psi / 1e3) / 1e9
        roofline.update(psi_pass_gbs=round(psi_gbs, 1), psi_pass_frac=round(psi_gbs / peak, 4))

    # e2e through the public API with pinned host buffers: upload rho0, run, read fields back
    e2e = None
    if not args.no_e2e:
        rho_pin = torch.from_numpy(rho0).pin_memory()
        out_rho = torch.empty(ncell, dtype=torch.float64).pin_memory()
        out_u = torch.empty(3 * ncell, dtype=torch.float64).pin_memory()
        out_p = torch.empty(ncell, dtype=torch.float64).pin_memory()
        barrier()
        t0 = time.perf_counter()
        plb.plb_init(lat.h, rho_pin)
        t1 = time.perf_counter()
        lat.step(args.e2e_steps)
        mass = lat.reduce(plb.PLB_MASS)[0]
        t2 = time.perf_counter()
        plb.plb_moments(lat.h, out_rho, out_u, out_p)
        barrier()
        te = time.perf_counter() - t0
        parts = {"init_ms": round((t1 - t0) * 1e3, 3), "steps_and_mass_ms": round((t2 - t1) * 1e3, 3),
                 "moments_ms": round((t0 + te - t2) * 1e3, 3)}
        te = max_over_ranks(te, world, "cuda")
        h2d = rho_pin.numel() * 8
        d2h = (out_rho.numel() + out_u.numel() + out_p.numel()) * 8 + 8
        e2e = {"value": round(job_glups(ncell, args.e2e_steps, te, world), 4), "unit": "GLUPS",
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps,
               "what": "plb_init from pinned host rho0 + K steps + plb_reduce(mass) + plb_moments to pinned host",
               "mass": mass, "parts": parts}
    del lat
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants:
        combos = [("fp16s", "fused"), ("fp16s_sr", "fused"), ("fp32", "fused"), ("fp32", "aa"), ("fp16s", "aa"),
                  ("fp16s_sr", "aa"), ("fp64", "aa")]
        for prec, strm in combos:
            if (prec, strm) == (args.precision, args.streaming):
                continue
            lv = make_lattice(dims, prec, args.collision, strm)
            lv.init(rho0)
            lv.step(3)
            nst = 20 if prec != "fp64" else 6
            tv = time_steps(lv, nst, torch)
            lv.status()
            g = ncell * nst / tv / 1e9
            ms_p, ms_f = lv.step_timed(min(nst, 6))
            bpv = bytes_per_cell(prec, streaming=strm)
            variants[f"{prec}_{strm}"] = {
                "glups": round(g, 3), "step_frac_hbm": round(g * bpv["step"] / peak, 4),
                "dominant_kernel_frac_hbm": round(bpv["fused_pass"] * ncell * min(nst, 6) / (ms_f / 1e3) / 1e9 / peak, 4),
                "bytes_per_cell": bpv["step"]}
            del lv
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args, seconds=12.0)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": round(t / args.steps * 1e3, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
                "data": "synthetic (seeded tanh liquid-vapour layers, Maxwell densities of the PR EOS)",
                "config": {"workload": wl, "cells": ncell, "lattice": "D3Q19", "collision": args.collision,
                           "precision": args.precision, "streaming": args.streaming,
                           "bytes_per_cell": bpc["step"], "eos": "Peng-Robinson a=2/49 b=2/21 w=0.327 T/Tc=0.8",
                           "boundaries": "halfway bounce-back walls in y, periodic x and z",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (populations %.2f GB)" % (19 * POP_BYTES[args.precision] * ncell / 1e9)},
                "roofline": roofline, "clocks": clocks, "e2e": e2e,
                "gpu_launches": (1 if args.streaming == "fused" else 2) * args.steps,
                "cpu_baseline": cpu, "variants": variants or None}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------- CPU baseline

def oracle_sample_setup(dims_full, precision, collision, ny_sample=16, nz_sample=16):
    """Bounded sample of the plates workload for the FP64 oracle: a slab of the full
    x extent with ny_sample rows between the walls and nz_sample planes."""
    import oracle
    from oracle import params as pp
    a, b, om = 2.0 / 49.0, 2.0 / 21.0, 0.327
    T = T_RATIO * pp.pr_Tc(a, b)
    rv, rl, _ = pp.pr_maxwell(a, b, 1.0, om, T)
    dims = (dims_full[0], ny_sample, nz_sample)
    rho = initial_density(dims, rv, rl)
    P = oracle.make_params(oracle.D3Q19, dims, wall_y=True, eos=dict(kind="pr", a=a, b=b, R=1.0, omega=om, T=T),
                           tau=1.0, mrt=collision == "mrt", rates=MRT_RATES, fext=(BODY_FORCE, 0.0, 0.0))
    return P, oracle.init(P, rho), dims


def cpu_baseline_sample(args, seconds=12.0):
    import oracle
    dims_full = tuple(int(v) for v in args.dims.split("x"))
    P, f, dims = oracle_sample_setup(dims_full, args.precision, args.collision)
    n = dims[0] * dims[1] * dims[2]
    t0 = time.perf_counter()
    f = oracle.run(P, f, 1)
    one = time.perf_counter() - t0
    steps = max(2, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(P, f, steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(n * steps / dt / 1e9, 6), "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, D3Q19 {args.collision.upper()}, {dims[0]}x{dims[1]}x{dims[2]} slab of the "
                      f"plates workload (walls in y), {steps} steps, {dt:.1f} s, OpenMP over cells"}


# workload, lattice (0 D2Q9, 1 D3Q19), dims, MRT, steps with 1 thread, steps with all cores
CPU_PLAN = (("d2q9_bgk_256x256_droplet", 0, (256, 256, 1), False, 200, 2000),
            ("d3q19_bgk_96x96x96_droplet", 1, (96, 96, 96), False, 10, 100),
            ("d3q19_mrt_96x96x96_droplet", 1, (96, 96, 96), True, 10, 100))


def cpu_plan_child(spec):
    """One entry of the CPU plan in this process (OMP_NUM_THREADS set by the parent): three timed
    runs of the oracle after one warm-up step; prints their MLUPS."""
    import oracle
    from oracle import params as pp
    from paper_2504_15018_gb300 import inputs
    name, steps = spec.rsplit(":", 1)
    steps = int(steps)
    _, lattice, dims, mrt, _, _ = next(e for e in CPU_PLAN if e[0] == name)
    a, b, om = 2.0 / 49.0, 2.0 / 21.0, 0.327
    T = T_RATIO * pp.pr_Tc(a, b)
    rv, rl, _ = pp.pr_maxwell(a, b, 1.0, om, T)
    nd = 2 if lattice == 0 else 3
    center = tuple(d / 2 - 0.3 for d in dims[:nd])
    rho = inputs.droplet(dims, center, dims[0] / 4, rv, rl, 4.0)
    P = oracle.make_params(oracle.D2Q9 if lattice == 0 else oracle.D3Q19, dims,
                           eos=dict(kind="pr", a=a, b=b, R=1.0, omega=om, T=T), tau=1.0, mrt=mrt, rates=MRT_RATES)
    f = oracle.run(P, oracle.init(P, rho), 1)
    n = dims[0] * dims[1] * dims[2]
    out = []
    for _ in range(3):
        t0 = time.perf_counter()
        f = oracle.run(P, f, steps)
        out.append(n * steps / (time.perf_counter() - t0) / 1e6)
    print(json.dumps({"mlups": out}))


def run_cpu_plan(args):
    """The FP64 oracle on the host cores, 1 thread and all cores (one child process each, so
    OpenMP starts with that thread count); median of 3 runs."""
    ncores = os.cpu_count() or 1
    cpu = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                cpu = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    rows = []
    for name, _, dims, _, s1, sn in CPU_PLAN:
        for threads, steps in ((1, s1), (ncores, sn)):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-plan-child", f"{name}:{steps}"],
                               env=env, capture_output=True, text=True, check=True)
            mlups = json.loads(r.stdout.strip().splitlines()[-1])["mlups"]
            rows.append({"workload": name, "threads": threads, "steps": steps,
                         "mlups_median": round(float(np.median(mlups)), 3), "runs": [round(v, 3) for v in mlups]})
    print(json.dumps({"cpu_plan": rows, "kind": "oracle (plain FP64 C, OpenMP over cells)", "cores": ncores,
                      "cpu": cpu}))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    dims_full = tuple(int(v) for v in args.dims.split("x"))
    P, f, dims = oracle_sample_setup(dims_full, args.precision, args.collision)
    n = dims[0] * dims[1] * dims[2]
    for _ in range(max(args.warmup, 3)):
        f = oracle.run(P, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.run(P, f, 1)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    wl = workload_name(dims_full, args.precision, args.collision)
    sample = (f"FP64 C oracle on the host cores, D3Q19 {args.collision.upper()}, one step of a "
              f"{dims[0]}x{dims[1]}x{dims[2]} slab of the plates workload per timed step")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl, "cells_per_step": n, "sample": sample},
            "cpu_baseline": {"value": round(value, 6), "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------- batch workload

def batch96_instances(plb, precision, collision):
    """96 D2Q9 instances: sides in {64, ..., 512}, static / translating droplets and planar
    interfaces, T/Tc in [0.7, 0.9] (seeded); FP32, tau = 1, eps = 2, kappa = 1."""
    from paper_2504_15018_gb300 import inputs
    desc = inputs.batched_d2q9_instances(96)
    insts, fields = [], []
    for k, d in enumerate(desc):
        side = d["side"]
        eos = plb.pr_eos(d["T_over_Tc"])
        rv, rl, _ = plb.plb_solve_params(eos)
        opts = plb.make_opts(precision=PREC[precision], collision=plb.PLB_MRT if collision == "mrt" else plb.PLB_BGK,
                             **MRT_RATES)
        insts.append(plb.make_instance((side, side, 1), eos, tau=1.0, opts=opts))
        dims = (side, side, 1)
        u0 = None
        if d["kind"] == "planar":
            rho = inputs.slab(dims, 1, side // 4, 3 * side // 4, rl, rv, 4.0)
        else:
            rho = inputs.droplet(dims, (side / 2, side / 2), d["radius"], rv, rl, 4.0)
            if d["kind"] == "translating":
                u0 = np.zeros((2, side * side))
                u0[0], u0[1] = d["velocity"]
        fields.append((rho, u0))
    return insts, fields, desc


def run_batch(args):
    import torch

    import paper_2504_15018_gb300 as plb
    torch.cuda.set_device(0)
    prec = args.precision
    insts, fields, desc = batch96_instances(plb, prec, args.collision)
    cells = sum(i.dims[0] * i.dims[1] for i in insts)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    tile, bps, _ = b.autotune(3)
    b.step(max(args.warmup, 3))
    # one untimed call with the timed step count: plb_batch_step captures and instantiates a
    # CUDA graph for each new step count, which must not fall inside the timed region
    b.step(args.steps)
    b.status()
    st = b.stream
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step(args.steps)
    e1.record(st)
    e1.synchronize()
    clocks = sampler.stop()
    b.status()
    t = e0.elapsed_time(e1) / 1e3
    value = cells * args.steps / t / 1e9
    bpc = 3 * 9 * POP_BYTES[prec] + 2 * PSI_BYTES[prec]
    peak, peak_kind = peak_hbm()
    # the same instances stepped one lattice at a time (two launches per instance and step)
    lats = []
    for k, (rho, u0) in enumerate(fields):
        lat = plb.Lattice(plb.PLB_D2Q9, tuple(insts[k].dims), insts[k].eos, 1.0, -1.0, 2.0, opts=insts[k].opts)
        lat.init(rho, u0)
        lats.append(lat)
    nsep = min(args.steps, 50)
    for lat in lats:
        lat.step(2)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(nsep):
        for lat in lats:
            lat.step(1)
    e1.record()
    e1.synchronize()
    t_sep = e0.elapsed_time(e1) / 1e3
    sep_glups = cells * nsep / t_sep / 1e9
    del lats
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3) + args.steps, "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic (seeded)",
            "config": {"workload": f"d2q9_batch96_uneven_{prec}_{args.collision}", "instances": len(insts),
                       "cells": cells, "sides": sorted({d['side'] for d in desc}),
                       "kinds": {k: sum(1 for d in desc if d['kind'] == k) for k in ("static", "translating", "planar")},
                       "tile_cells": tile, "blocks_per_sm": bps,
                       "l2": "populations %.2f GB, larger than L2" % (9 * POP_BYTES[prec] * cells / 1e9)},
            "roofline": {"bound": "hbm", "kernel": "k_batch (persistent, all instances, graph-replayed)",
                         "achieved": round(value * bpc, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(value * bpc / peak, 4), "traffic": None,
                         "algorithmic_bytes_per_cell_step": bpc},
            "clocks": clocks, "gpu_launches": 1,
            "per_instance_launches": {"glups": round(sep_glups, 4), "launches_per_step": 2 * len(insts)}}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.cpu_plan_child:
        cpu_plan_child(args.cpu_plan_child)
    elif args.cpu_plan:
        run_cpu_plan(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch96":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
