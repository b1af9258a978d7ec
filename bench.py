#!/usr/bin/env python
"""Benchmark: seconds per implicit step of the multilevel-RAS Newton-Krylov
Peng-Robinson solver on GB300, with the RAS subdomain-solve kernel's HBM
roofline.

Workload (default): 3D 128 x 128 x 64 cell-centred grid (1,048,576 cells), seeded
log-normal permeability (sigma 1.5, correlated over 8 cells), methane PR-EOS,
corner-column injector/producer, dt = 0.1 day, BDF1 then BDF2; inexact Newton
to 1e-6 relative with FGMRES(30) (rtol 1e-6), two-level V-cycle RAS: 8 x 8 x 4
subdomains with overlap 2, ILU(0) factors in FP32, coarse grid coarsened 4x per
axis (32 x 32 x 16) solved by an FP32 dense block LU; Newton, residual,
Jacobian, SpMV and Krylov in FP64.

One step = one full implicit time step (all Newton iterations, every FGMRES
iteration, every preconditioner factorisation and application) on state that
is resident in HBM. `e2e` repeats the steps through the same public API with
the step's inputs copied from pinned host memory and the new state copied
back, inside the timed region.

`--workload c3` times the 60 x 220 x 85 channelised case with the three-level
V-cycle of Algorithm 1 instead (middle level 30 x 110 x 43, coarsest 15 x 55 x
22, ratio 2 per axis).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
path has no data exchange between them.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sec per implicit step and ras_apply HBM GB/s, FP32-RAS vs FP64, at 1e-6 rel residual"
WORKLOAD = ("3d 128x128x64 lognormal (1.05M cells), two-level V-cycle RAS 8x8x4 overlap 2, "
            "ILU(0) FP32 factors, coarse 4x (32x32x16) FP32 dense block LU, FP64 FGMRES(30) "
            "rtol 1e-6, Newton rtol 1e-6, dt 0.1 day")
WORKLOAD_C3 = ("3d 60x220x85 channelised (1.12M cells), three-level V-cycle RAS (Algorithm 1): "
               "4x11x5 subdomains overlap 2 on the fine grid, middle level 30x110x43 with 4x11x5 "
               "subdomains overlap 1 (ILU(0) on the Galerkin operator), coarsest 15x55x22 FP32 "
               "dense block LU, ratio 2 per axis, FP64 FGMRES(30) rtol 1e-6, Newton rtol 1e-6, "
               "dt 0.1 day")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--factor-prec", type=int, default=32)
    ap.add_argument("--coarse-prec", type=int, default=32)
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the all-FP64 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="32x32x16 case (profiling / smoke)")
    ap.add_argument("--workload", choices=["c2", "c3", "c4"], default="c2",
                    help="c2: 128x128x64 two-level (default); c3: 60x220x85 three-level; "
                         "c4: 64 independent reservoirs of 32^3..96^3 solved concurrently")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--kernel", choices=["ras_apply", "vcycle", "factor"], default=None,
                    help="kernel-only mode: factor once, then time REPS applications, or "
                         "(factor) REPS factorisations (used for the ncu captures)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--apply-kernel", type=int, choices=[0, 1], default=None,
                    help="fine subdomain-solve kernel: 0 level-scheduled, 1 pipelined "
                         "(default: the library's choice)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_reservoir(small=False, workload="c2"):
    from paper_2007_13966_gb300 import synthetic as syn
    if workload == "c3":
        return syn.channelised_reservoir()
    if small:
        return syn.lognormal_reservoir(32, 32, 16, 25.0, 25.0, 12.5, sigma=1.5, corr=8.0,
                                       seed_k=3, seed_phi=4, name="3d 32x32x16 lognormal")
    return syn.config_3d_1m()


def precond_opts(small=False, workload="c2"):
    if workload == "c3":
        return dict(parts=(4, 11, 5), overlap=2, nlevels=3, coarsen=(2, 2, 2), mlevel_type=0,
                    coarse_overlap=1)
    parts = (2, 2, 1) if small else (8, 8, 4)
    return dict(parts=parts, overlap=2, nlevels=2, coarsen=(4, 4, 4), mlevel_type=0,
                coarse_overlap=1)


def make_precond(ras, gp, po, factor_prec, coarse_prec, nlevels=None, apply_kernel=None):
    pc = ras.Precond(gp, po["parts"], po["overlap"], factor_prec=factor_prec,
                     nlevels=po["nlevels"] if nlevels is None else nlevels,
                     coarsen=po["coarsen"], mlevel_type=po["mlevel_type"],
                     coarse_prec=coarse_prec, coarse_overlap=po["coarse_overlap"])
    if apply_kernel is not None:
        pc.set_apply_kernel(apply_kernel)
    return pc


NEWTON = dict(rtol=1e-6, atol=1e-10, maxit=50, lin_rtol=1e-6, lin_atol=1e-8, restart=30,
              lin_maxit=3000)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, timeout=5.0):
        """Block until the sampler has printed its first sample (nvidia-smi's start-up,
        which initialises NVML, then falls before the timed region, not inside it)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------

def run_steps(gp, pc, res, state, nsteps, torch, stream_sync=True, e2e_host=None):
    """Advance `nsteps` implicit steps. state = dict(p_l, p_lm1, step)."""
    outs = []
    for _ in range(nsteps):
        order = 1 if state["step"] == 0 else 2
        if e2e_host is not None:
            # inputs from pinned host memory, result back to host
            state["p_l"].copy_(e2e_host["p_l"], non_blocking=True)
            state["p_lm1"].copy_(e2e_host["p_lm1"], non_blocking=True)
        p = state["p_l"].clone()
        out = gp.newton_step(pc, p, state["p_l"], state["p_lm1"], res.dt, order, **NEWTON)
        if out["status"] != 0:
            raise RuntimeError(f"newton_step status {out['status']}")
        if e2e_host is not None:
            e2e_host["p_lm1"].copy_(e2e_host["p_l"])
            e2e_host["p_l"].copy_(p, non_blocking=False)
        state["p_lm1"], state["p_l"] = state["p_l"], p
        state["step"] += 1
        outs.append(out)
    return outs


def timed(fn, torch, dist_on):
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3, r


def max_over_ranks(v, dist_on):
    if not dist_on:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(key):
    """Per-launch DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum)
    of the kernel from the committed profile summary, if the summary was taken
    on the current source of that kernel (its line records the source hash)."""
    import glob
    import re
    from paper_2007_13966_gb300 import build_lib
    cur = build_lib.source_hash(build_lib.RAS_APPLY_FILES)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = re.match(r"bench-traffic: (\S+) bytes_per_launch=(\d+) source_hash=(\w+)", line.strip())
                if m and m.group(1) == key and m.group(3) == cur:
                    return float(m.group(2))
    return None


def gb300_arm(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    dist_on = ws > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2007_13966_gb300 import ras

    res = make_reservoir(args.small, args.workload)
    N = res.grid.n
    gp = ras.Problem(res)
    po = precond_opts(args.small, args.workload)
    pc = make_precond(ras, gp, po, args.factor_prec, args.coarse_prec, apply_kernel=args.apply_kernel)
    p0 = torch.full((N,), res.p0, dtype=torch.float64, device="cuda")
    state = {"p_l": p0.clone(), "p_lm1": p0.clone(), "step": 0}

    # warm-up (also the first, BDF1, step)
    run_steps(gp, pc, res, state, args.warmup, torch)
    torch.cuda.synchronize()

    def clone(st):
        return {"p_l": st["p_l"].clone(), "p_lm1": st["p_lm1"].clone(), "step": st["step"]}

    s0 = clone(state)   # the state the timed steps start from
    # timed region: K implicit steps on resident state (no per-launch events inside)
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_ready()
    n0 = ras.kernel_launches()
    t, outs = timed(lambda: run_steps(gp, pc, res, state, args.steps, torch), torch, dist_on)
    launches = ras.kernel_launches() - n0
    clocks = sampler.stop()
    t = max_over_ranks(t, dist_on)
    sec_per_step = t / args.steps

    # e2e: the SAME K steps again from the same starting state, through the public
    # API with each step's inputs copied from pinned host memory and the new state
    # copied back inside the timed region
    se = clone(s0)
    pin = {"p_l": s0["p_l"].cpu().pin_memory(), "p_lm1": s0["p_lm1"].cpu().pin_memory()}
    te, outs_e = timed(lambda: run_steps(gp, pc, res, se, args.steps, torch, e2e_host=pin), torch,
                       dist_on)
    te = max_over_ranks(te, dist_on)

    # the subdomain-solve kernel's launch times: the same K steps a third time with
    # CUDA events recorded around every launch of it (kept out of the timed step)
    sa_ = clone(s0)
    pc.timing(True)
    pc.timing_read(reset=True)
    run_steps(gp, pc, res, sa_, args.steps, torch)
    torch.cuda.synchronize()
    apply_ms, apply_n = pc.timing_read(reset=True)
    pc.timing(False)

    # the all-FP64 form on the same step sequence, for the FP32-vs-FP64 comparison
    fp64 = None
    if not args.no_fp64_form and (args.factor_prec != 64 or args.coarse_prec != 64):
        pc64 = make_precond(ras, gp, po, 64, 64)
        run_steps(gp, pc64, res, clone(s0), 1, torch)   # warm-up of the FP64 handle
        k64 = max(1, min(args.steps, 3))
        # both forms timed on the same first k64 steps of the timed region
        sa, sb = clone(s0), clone(s0)
        t64, outs64 = timed(lambda: run_steps(gp, pc64, res, sa, k64, torch), torch, dist_on)
        tlo, _ = timed(lambda: run_steps(gp, pc, res, sb, k64, torch), torch, dist_on)
        t64 = max_over_ranks(t64, dist_on)
        tlo = max_over_ranks(tlo, dist_on)
        # one step of each form from the same FP64 state: max |p_lo - p_64| / max |p_64|
        diffs = []
        sx = clone(s0)
        for _ in range(k64):
            sy = clone(sx)
            run_steps(gp, pc64, res, sx, 1, torch)
            run_steps(gp, pc, res, sy, 1, torch)
            diffs.append(float((sy["p_l"] - sx["p_l"]).abs().max() / sx["p_l"].abs().max()))
        fp64 = {"sec_per_step": t64 / k64, "steps": k64,
                "newton_iters": [o["newton_iters"] for o in outs64],
                "fgmres_iters": [o["lin_total"] for o in outs64],
                "reduced_sec_per_step_same_steps": tlo / k64,
                "fp32_speedup": t64 / tlo,
                "state_rel_diff_per_step": diffs}
        del pc64

    if rank != 0:
        if dist_on:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    bytes_per_launch = pc.apply_bytes()
    avg_s = (apply_ms / 1e3) / max(apply_n, 1)
    achieved = bytes_per_launch / avg_s / 1e9 if apply_n else None
    traffic = None
    kname = "k_ras_pipe" if pc.apply_kernel() == 1 else "k_ras_apply"
    if args.workload == "c2" and not args.small:
        traffic = load_traffic(f"{kname}_fp{args.factor_prec}_1m")
    line = {
        "metric": METRIC,
        "value": sec_per_step,
        "unit": "s/step",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sec_per_step * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+f32",
        "data": "synthetic",
        "config": {
            "workload": (WORKLOAD_C3 if args.workload == "c3" else
                         WORKLOAD if not args.small else "3d 32x32x16 lognormal (profiling case)"),
            "cells": N, "subdomains": list(po["parts"]), "overlap": po["overlap"],
            "levels": po["nlevels"],
            "coarse": ([15, 55, 22] if args.workload == "c3" else
                       [32, 32, 16] if not args.small else [8, 8, 4]),
            "factor_prec": args.factor_prec, "coarse_prec": args.coarse_prec,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "working set ~1 GB > 129 MB L2 (no flush needed)",
        },
        "newton_iters": [o["newton_iters"] for o in outs],
        "fgmres_iters": [o["lin_total"] for o in outs],
        "clocks": clocks,
        "e2e": {"value": te / args.steps, "unit": "s/step",
                "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8,
                "same_steps_as_value": True,
                "newton_iters": [o["newton_iters"] for o in outs_e],
                "fgmres_iters": [o["lin_total"] for o in outs_e]},
        "gpu_launches": int(launches),
        "roofline": {
            "kernel": "%s (fine-level subdomain ILU(0) solves, %s factors)"
                      % (kname, {64: "FP64", 32: "FP32", 16: "BF16"}[args.factor_prec]),
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "peak_kind": peak_kind,
            "bytes_per_launch": bytes_per_launch,
            "avg_launch_us": avg_s * 1e6, "launches": int(apply_n),
            "launch_times": "CUDA events around every launch of the kernel, on its stream, in a "
                            "separate pass over the same K steps (not inside the timed steps)",
        },
        "fp64_form": fp64,
    }
    if ws == 1 and not args.no_cpu_baseline and args.workload == "c2":
        line["cpu_baseline"] = cpu_baseline_subprocess(args)
    print(json.dumps(line), flush=True)
    if dist_on:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# oracle on the host cores (CPU baseline leg and the reference arm)
# ---------------------------------------------------------------------------

SAMPLE = ("one implicit step (BDF1, Newton to 1e-6 with FGMRES(30) and the two-level V-cycle "
          "left-RAS / ILU(0) / dense coarse LU of the oracle) on a 32x32x16 sub-grid of the same "
          "recipe (2x2x1 subdomains of 16^3, overlap 2, coarse 8x8x4), scaled by the cell ratio "
          "1048576/16384 = 64")


def oracle_step_seconds():
    """Times the oracle (as it stands) on the bounded sample; returns scaled s/step."""
    import numpy as np
    from oracle import discretization as disc
    from oracle import multilevel as ml
    from oracle import newton, schwarz
    from paper_2007_13966_gb300 import synthetic as syn

    res = syn.lognormal_reservoir(32, 32, 16, 25.0, 25.0, 12.5, sigma=1.5, corr=8.0,
                                  seed_k=3, seed_phi=4)
    g = res.grid
    dims = (g.nx, g.ny, g.nz)
    prob = disc.Problem(res)
    P = ml.interpolation(dims, (4, 4, 4), 2)

    def fac(A, J):
        M = schwarz.Schwarz(A, dims, (2, 2, 1), 2)
        return ml.TwoLevel(A, M, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.VCYCLE)

    p0 = np.full(g.n, res.p0)
    t0 = time.perf_counter()
    newton.newton_solve(prob, fac, p0, p0, res.dt, 1, rtol=1e-6, atol=1e-10, lin_rtol=1e-6,
                        lin_atol=1e-8, restart=30)
    dt = time.perf_counter() - t0
    return dt * (1048576 / g.n), dt


def oracle_residual_anchor():
    """Times one oracle residual + Jacobian evaluation on the full 128x128x64 grid
    and on the 32x32x16 sample grid: a measured anchor for scaling the sample's
    step time by the cell ratio (returns both times and their ratio)."""
    import numpy as np
    from oracle import discretization as disc
    from paper_2007_13966_gb300 import synthetic as syn
    out = {}
    for name, res in (("1m", syn.config_3d_1m()),
                      ("sample", syn.lognormal_reservoir(32, 32, 16, 25.0, 25.0, 12.5, sigma=1.5,
                                                         corr=8.0, seed_k=3, seed_phi=4))):
        prob = disc.Problem(res)
        p = syn.random_pressure(res, 3, 1.0, 3.0)
        disc.residual(prob, p, 0.99 * p, 0.98 * p, res.dt, 2, want_jac=True)   # warm-up
        t0 = time.perf_counter()
        disc.residual(prob, p, 0.99 * p, 0.98 * p, res.dt, 2, want_jac=True)
        out[name] = time.perf_counter() - t0
    return {"residual_jacobian_1m_s": out["1m"], "residual_jacobian_sample_s": out["sample"],
            "measured_ratio": out["1m"] / out["sample"], "cell_ratio": 64}


def cpu_baseline_subprocess(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample"],
                           capture_output=True, text=True, env=env, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # the baseline is reported, never required
        return {"value": None, "unit": "s/step", "cores": 1, "kind": "oracle",
                "sample": SAMPLE, "error": str(e)[:200]}
    return {"value": d["value"], "unit": "s/step", "cores": 1, "kind": "oracle",
            "sample": SAMPLE, "sample_seconds": d["raw"], "host_cores": os.cpu_count(),
            "anchor": d.get("anchor")}


def cpu_sample_main():
    v, raw = oracle_step_seconds()
    print(json.dumps({"value": v, "raw": raw, "anchor": oracle_residual_anchor()}))


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_step_seconds()
    for _ in range(args.steps):
        v, _raw = oracle_step_seconds()
        vals.append(v)
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "s/step",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": value * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": 1048576},
        "cpu_baseline": {"value": value, "unit": "s/step", "cores": 1, "kind": "oracle",
                         "sample": SAMPLE},
        "e2e": {"value": value, "unit": "s/step", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_mode(args):
    """Set up the workload, factor once, time `reps` preconditioner applications."""
    import torch
    from paper_2007_13966_gb300 import ras
    res = make_reservoir(args.small, args.workload)
    N = res.grid.n
    gp = ras.Problem(res)
    po = precond_opts(args.small, args.workload)
    nl = 1 if args.kernel == "ras_apply" else po["nlevels"]
    pc = make_precond(ras, gp, po, args.factor_prec, args.coarse_prec, nlevels=nl,
                      apply_kernel=args.apply_kernel)
    from paper_2007_13966_gb300 import synthetic as syn
    p = torch.tensor(syn.random_pressure(res, 3, 1.0, 3.0), device="cuda")
    p0 = torch.full((N,), res.p0, dtype=torch.float64, device="cuda")
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    pc.factor(gp.J)
    if args.kernel == "factor":
        # ras_factor: fine ILU(0) factors (own stream), Galerkin product, block
        # assembly and the coarse block elimination; CUDA events, median of REPS
        for _ in range(2):
            pc.factor(gp.J)
        ts = sorted(timed(lambda: pc.factor(gp.J), torch, False)[0] for _ in range(args.reps))
        print(json.dumps({"kernel": "factor", "reps": args.reps, "factor_ms_median": ts[len(ts) // 2] * 1e3,
                          "factor_ms_min": ts[0] * 1e3}))
        return
    r = torch.randn(N, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    for _ in range(3):
        pc.apply(r, z)
    pc.timing(True)
    pc.timing_read(reset=True)
    t, _ = timed(lambda: [pc.apply(r, z) for _ in range(args.reps)], torch, False)
    ms, n = pc.timing_read(reset=True)
    B = pc.apply_bytes()
    print(json.dumps({"kernel": args.kernel, "apply_kernel": pc.apply_kernel(), "reps": args.reps,
                      "apply_us": t / args.reps * 1e6,
                      "subdomain_kernel_us": ms / max(n, 1) * 1e3, "bytes": B,
                      "GBps": B / (ms / max(n, 1) / 1e3) / 1e9 if n else None}))


WORKLOAD_C4 = ("64 independent 3d lognormal reservoirs, edges uniform in 32..96 (seed 7), "
               "per-instance seeds, two-level V-cycle: left-RAS ILU(0) with ~16^3 subdomains, overlap 1, "
               "exact coarse solve on the 4x coarsened grid, FP32 factors inside FP64 FGMRES(30), all "
               "reservoirs in one batch handle (one launch per fine-level FGMRES operation for the whole "
               "batch; coarse solves of all reservoirs in one cooperative launch, coarse block "
               "eliminations in waves of at least 16 CTAs per reservoir)")


def c4_arm(args):
    """One batch step = every reservoir of the batch advances one implicit step."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    dist_on = ws > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2007_13966_gb300 import batch
    from paper_2007_13966_gb300 import synthetic as syn

    def make(n, i):
        h = 100.0 / 128
        return syn.lognormal_reservoir(n, n, n, n * h, n * h, n * h, sigma=1.5, corr=8.0,
                                       seed_k=100 + i, seed_phi=200 + i)

    res = batch.random_batch(64, 32, 96, 7, make)
    opts = batch.BatchOpts(box=16, overlap=1, factor_prec=args.factor_prec, threads=16, fused=True,
                           nlevels=2, coarsen=(4, 4, 4), tune=True)
    b = batch.Batch(res, opts)
    tuned = {"chunk_cells": b.schedule, "table": b.tune_table}
    b.advance(max(args.warmup, 1))
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_ready()
    from paper_2007_13966_gb300 import ras
    n0 = ras.kernel_launches()
    t, _ = timed(lambda: b.advance(args.steps), torch, dist_on)
    launches = ras.kernel_launches() - n0
    clocks = sampler.stop()
    t = max_over_ranks(t, dist_on)
    iters = [it for i in b.inst for it in i.iters[-args.steps:]]
    cells = b.cells
    del b
    # the same reservoirs, one CUDA stream and host thread per reservoir, for context
    # (one BDF1 warm-up step, one timed BDF2 step)
    bs = batch.Batch(res, batch.BatchOpts(box=16, overlap=1, factor_prec=args.factor_prec, threads=16,
                                          fused=False, nlevels=2, coarsen=(4, 4, 4)))
    bs.advance(1)
    ts, _ = timed(lambda: bs.advance(1), torch, dist_on)
    del bs
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": t / args.steps, "unit": "s/step", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 1), "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_C4, "instances": len(res), "cells": cells,
                   "parallelism": "one batch handle: every FGMRES operation of all reservoirs in one launch"},
        "cell_steps_per_s": cells * args.steps / t,
        "newton_iters_mean": float(np.mean([a for a, _ in iters])),
        "fgmres_iters_mean": float(np.mean([c for _, c in iters])),
        "schedule_autotune": tuned,
        "streams_sec_per_step": ts,
        "fused_speedup_over_streams": ts / (t / args.steps),
        "clocks": clocks, "gpu_launches": int(launches), "e2e": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "c4" and args.impl != "reference" and not args.kernel:
        c4_arm(args)
        return
    if args.kernel:
        kernel_mode(args)
        return
    if args.cpu_sample:
        cpu_sample_main()
        return
    if args.impl == "reference":
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")
        reference_arm(args)
        return
    gb300_arm(args)


if __name__ == "__main__":
    main()
