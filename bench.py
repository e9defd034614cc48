"""Throughput benchmark of the fused MRT-LBKM step on GB300.

Workload: the 2-D periodic reactive field of 4096 x 4096 cells (32 random
Fourier modes in rho and T, solenoidal u of peak 0.1, lambda ~ U[0, 0.2],
S ~ U[1e4, 1e5], Q = 1, k = 2e4), FP32 state with FP64 conserved-moment
recovery and FP64 grid-wide TNE reductions on every step. A step is one launch
of the fused kernel over the whole grid (stencil, collision, reaction, Euler
update, TNE). The state (1.14 GB per copy) is larger than L2, so no flush is
needed between steps.

Prints one JSON line: Mcell-updates/s (cells x steps / time), the roofline of
the step kernel against the measured HBM copy bandwidth, an end-to-end figure
through the C ABI with host buffers, the CPU oracle timed on the host cores,
and SM clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the method has no other reference
implementation: the paper prints no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

import lbkm_inputs as li  # noqa: E402

N_CELLS_SIDE = 4096
BYTES_PER_CELL = {"f32": 136, "f64": 272}  # read + write of 16 f + lambda
# FP64 operations per cell update of the plain FP64 step kernel (step_kernel<double>, 2-D),
# from ncu's executed-instruction counters on a 1024 x 1024 grid: 2 per DFMA, 1 per DADD and
# DMUL (profiles/step_kernel_fp64_reactive2d.md)
F64_FLOP_PER_CELL = 911.5
F64_FLOP_SOURCE = ("ncu sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on on one step of "
                   "a 1024 x 1024 reactive field with TNE: 213.96 DFMA + 375.76 DADD + 107.87 DMUL "
                   "per cell")

METRIC = "Mcell-updates/s (16 f_i)"


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(ms, device, world):
    """The slowest rank's time: barrier, then an all-reduce (MAX) of the per-rank
    milliseconds; the replicas share no data, so this is the only collective."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the FP32 2-D step runs march_kernel (march.cu); FP64 and 1-D grids run step_kernel
STEP_KERNEL_SOURCES = {
    "march": ("march.cu", "pair.cuh", "vec2.cuh", "reduce.cuh", "cell.cuh", "kernels.cuh",
              "model.h"),
    "step": ("kernels.cu", "cell.cuh", "kernels.cuh", "model.h", "reduce.cuh"),
    "batch": ("batch.cu", "cell.cuh", "pair.cuh", "vec2.cuh", "kernels.cuh", "model.h"),
}
PROFILE = {"march": "march_kernel_reactive2d.md", "step": "step_kernel_fp64_reactive2d.md",
           "batch": "batch_kernel_batched.md"}


def step_kernel_digest(kernel="march"):
    """sha256 over the sources that define the step kernel."""
    import hashlib
    src = os.path.join(ROOT, "paper_1411_6697_gb300", "csrc")
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()


def profile_traffic(kernel, kernel_tag):
    """dram bytes per launch from the committed ncu summary, if it matches the current
    kernel source (sha256 line); else None."""
    prof = os.path.join(ROOT, "profiles", PROFILE[kernel])
    digest = step_kernel_digest(kernel)
    try:
        lines = open(prof).read().splitlines()
    except OSError:
        return None
    kv = {}
    for line in lines:
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("source_sha256") != digest:
        return None
    try:
        return float(kv.get(kernel_tag if kernel_tag.startswith("traffic_") else
                            "traffic_bytes_per_launch_%s" % kernel_tag))
    except (TypeError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

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
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_solver(cfg, precision, recovery, stream=None, tne_every=1, S=None, collision=0):
    from paper_1411_6697_gb300 import lbkm
    p = cfg["params"]
    return lbkm.Solver(nx=p["nx"], ny=p["ny"], precision=precision, recovery=recovery,
                       gamma=p["gamma"], orbit_kind=p["orbit_kind"], orbit_speed=p["orbit_speed"],
                       orbit_eta=p["orbit_eta"], S=p["S"] if S is None else S, Q=p["Q"],
                       omega1=p["omega1"], collision=collision,
                       omega2=p["omega2"], T_ig=p["T_ig"], dx=p["dx"], dy=p["dx"], dt=p["dt"],
                       bc=(p["bc_x"], p["bc_y"]), tne_every=tne_every,
                       tne_capacity=4096, stream=stream)


def time_steps(solver, stream, steps):
    """CUDA-event time of `steps` fused steps on the solver's stream (ms)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def cpu_oracle_rate(budget_s=12.0, side=1024):
    """The FP64 oracle, as it stands, on a side x side window generated with the same
    recipe; steps chosen to fill about budget_s seconds. Returns (Mcell/s, desc, cores)."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    cfg = li.reactive2d(n=side, steps=1)
    p = dict(cfg["params"])
    nx, ny = p.pop("nx"), p.pop("ny")
    ob = oracle.Oracle(nx, ny, **p)
    fl = cfg["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    t0 = time.perf_counter()
    f, lam = ob.run(f, fl["lam"], 1)
    one = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    ob.run(f, lam, steps)
    dt = time.perf_counter() - t0
    rate = nx * ny * steps / dt / 1e6
    desc = "FP64 C oracle (OpenMP, %d threads) on a %dx%d window of the same recipe, %d steps, " \
           "%.1f s" % (int(os.environ["OMP_NUM_THREADS"]), side, side, steps, dt)
    return rate, desc, int(os.environ["OMP_NUM_THREADS"])


def cpu_oracle_rate_single(budget_s=8.0, side=256):
    """The same oracle on one host core: a child process started with OMP_NUM_THREADS=1
    (OpenMP reads it when the oracle's first parallel region starts), a side x side window.
    Returns (Mcell/s, desc) or (None, why)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, bench; r = bench.cpu_oracle_rate(%r, %d); "
            "print(json.dumps(r))" % (budget_s, side))
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, check=True,
                             capture_output=True, text=True, timeout=300).stdout
        rate, desc, threads = json.loads(out.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return None, "single-thread run failed: %s" % e
    return (rate, desc) if threads == 1 else (None, "the child ran %d threads" % threads)


def cpu_oracle_rate_d2v24(budget_s=10.0, side=256):
    """The D2V24 FP64 oracle, as it stands, on a side x side window of the 2-D D2V24 field
    recipe; steps chosen to fill about budget_s seconds. Returns (Mcell/s, desc, cores)."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    cfg = li.d2v24_reactive2d(n=side, steps=1)
    p = dict(cfg["params"])
    nx, ny = p.pop("nx"), p.pop("ny")
    ob = oracle.Oracle(nx, ny, **p)
    fl = cfg["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    t0 = time.perf_counter()
    f, lam = ob.run(f, fl["lam"], 1)
    one = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    ob.run(f, lam, steps)
    dt = time.perf_counter() - t0
    rate = nx * ny * steps / dt / 1e6
    desc = ("FP64 C oracle with 24 velocities (OpenMP, %d threads) on a %dx%d D2V24 field, "
            "%d steps, %.1f s" % (int(os.environ["OMP_NUM_THREADS"]), side, side, steps, dt))
    return rate, desc, int(os.environ["OMP_NUM_THREADS"])


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, a bounded window per step."""
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    from oracle import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    side = 384
    cfg = li.reactive2d(n=side, steps=1)
    p = dict(cfg["params"])
    nx, ny = p.pop("nx"), p.pop("ny")
    ob = oracle.Oracle(nx, ny, **p)
    fl = cfg["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    lam = fl["lam"]
    for _ in range(args.warmup):
        f, lam = ob.run(f, lam, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, lam = ob.run(f, lam, 1)
    dt = time.perf_counter() - t0
    value = nx * ny * args.steps / dt / 1e6
    sample = "%dx%d window of the reactive2d recipe per step (FP64 oracle, %s threads)" % (
        side, side, os.environ["OMP_NUM_THREADS"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mcell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "reactive2d_4096x4096 (sampled window)", "window": side},
            "cpu_baseline": {"value": value, "unit": "Mcell-updates/s",
                             "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _shared_params(p0):
    return {k: p0[k] for k in ("gamma", "orbit_kind", "orbit_speed", "orbit_eta", "omega1",
                               "omega2", "T_ig", "dx", "dt")}


def measure_batched(steps, warmup, recovery="f64", plain_instances=24, plain_steps=64):
    """Config 4: 512 1-D detonations of uneven length, FP32, in one persistent launch per
    chunk of steps (CUDA graph), timed over `steps` steps; the plain single-instance FP64
    form timed on a seeded sample of the same instances, one after another."""
    import torch
    from paper_1411_6697_gb300 import lbkm
    rec = lbkm.RECOVER_F64 if recovery == "f64" else lbkm.RECOVER_DF32
    cfg = li.batched(n_instances=512, steps=5000)
    p0 = cfg["instances"][0]["params"]
    stream = torch.cuda.Stream()
    s = lbkm.Solver.batched(cfg["nx"], inst_S=cfg["S"], inst_Q=cfg["Q"], recovery=rec,
                            dy=p0["dx"], stream=stream, **_shared_params(p0))
    fields = {k: np.concatenate([d["fields"][k] for d in cfg["instances"]], axis=1)
              for k in ("rho", "ux", "uy", "T", "lam")}
    s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
    chosen = s.autotune(trial_steps=3)
    n = int(np.sum(cfg["nx"]))
    with torch.cuda.stream(stream):
        s.step(warmup)
        s.sync()
        ms = time_steps(s, stream, steps)
        s.sync()
    s.close()
    value = n * steps / (ms * 1e-3) / 1e6
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_CELL["f32"] * n / (ms / steps * 1e-3) / 1e9
    rng = np.random.default_rng(li.SEED_BASE + 40)
    sample = rng.choice(len(cfg["nx"]), plain_instances, replace=False)
    t64 = c64 = 0.0
    for i in sample:
        d = cfg["instances"][i]
        q = d["params"]
        one = lbkm.Solver(nx=q["nx"], ny=1, precision=lbkm.F64, S=q["S"], Q=q["Q"], bc=(1, 0),
                          dy=q["dx"], stream=stream, **_shared_params(q))
        fl = d["fields"]
        one.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
        with torch.cuda.stream(stream):
            one.step(3)
            t64 += time_steps(one, stream, plain_steps) * 1e-3
        c64 += q["nx"] * plain_steps
        one.close()
    plain = c64 / t64 / 1e6
    return {"workload": "batched_512x1d_detonations", "cells": n, "instances": len(cfg["nx"]),
            "steps_timed": steps, "ms_per_step": ms / steps, "mcell_per_s": value,
            "conserved_moment_recovery": recovery,
            "autotuned": {"threads": chosen[0], "blocks_per_sm": chosen[1], "blocks": chosen[2]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": profile_traffic("batch", "traffic_bytes_per_step_f32"), "peak_kind": peak_kind,
                         "kernel": "batch_kernel (f32)",
                         "algorithmic_bytes_per_step": BYTES_PER_CELL["f32"] * n},
            "plain_f64_single_instance_mcell_per_s": plain,
            "speedup_vs_plain_f64": value / plain,
            "plain_sample": "%d seeded instances, %d steps each, one after another" % (
                plain_instances, plain_steps),
            "accuracy": "per field <= 2e-5 against the FP64 oracle (6 uneven instances, 40 steps); "
                        "all 512 instances for 5000 steps within 4x the oracle's own FP32-storage "
                        "error (tests/test_gpu_batched.py)"}


def run_batched(args):
    """512 1-D detonations of uneven length in one persistent launch per chunk
    of steps, FP32; compared with the plain single-instance FP64 form on a sample of the
    same instances, run one after another."""
    import torch
    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        b = measure_batched(args.steps, args.warmup, args.recovery)
    line = {"metric": METRIC, "value": b["mcell_per_s"], "unit": "Mcell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": b["workload"], "cells": b["cells"], "instances": b["instances"],
                       "conserved_moment_recovery": b["conserved_moment_recovery"],
                       "autotuned": b["autotuned"],
                       "l2": "state %.2f GB per copy > L2: no flush" % (17 * b["cells"] * 4 / 1e9)},
            "roofline": b["roofline"],
            "plain_f64_single_instance_mcell_per_s": b["plain_f64_single_instance_mcell_per_s"],
            "speedup_vs_plain_f64": b["speedup_vs_plain_f64"], "plain_sample": b["plain_sample"],
            "gpu_launches": (args.steps + 31) // 32, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_detonation(args):
    """One 1-D detonation of 16384 cells, 20000 steps (L2-resident, latency-bound)."""
    import torch
    from paper_1411_6697_gb300 import lbkm
    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    cfg = li.detonation()
    fl = cfg["fields"]
    stream = torch.cuda.Stream()
    out = {}
    for name, prec in (("f64", lbkm.F64), ("f32", lbkm.F32)):
        q = cfg["params"]
        one = lbkm.Solver(nx=q["nx"], ny=1, precision=prec, S=q["S"], Q=q["Q"], bc=(1, 0),
                          dy=q["dx"], stream=stream, tne_every=1, tne_capacity=4096,
                          **_shared_params(q))
        one.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
        with torch.cuda.stream(stream):
            one.step(args.warmup)
            ms = time_steps(one, stream, args.steps)
        out[name] = q["nx"] * args.steps / (ms * 1e-3) / 1e6
        one.close()
    line = {"metric": METRIC, "value": out["f32"], "unit": "Mcell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "detonation_16384x1", "note": "2.2 MB state, L2-resident"},
            "f64_mcell_per_s": out["f64"]}
    print(json.dumps(line))
    return 0


def run_d2v24(args):
    """The paper's own D2V24 model: the steady-detonation run of Sec. IV.A (5000 cells,
    1 MB of state, L2-resident and latency-bound) and a 2-D reactive field of 2048^2
    cells (state > L2), each in FP64 and FP32, through lbkm24."""
    import torch
    from paper_1411_6697_gb300 import lbkm
    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    out = {}
    cases = (("detonation", li.d2v24_detonation(), args.steps),
             ("reactive2d", li.d2v24_reactive2d(n=2048, steps=args.steps), max(args.steps // 10, 5)))
    with ClockSampler(local) as clk:
        for name, cfg, steps in cases:
            fl = cfg["fields"]
            for tag, prec in (("f64", lbkm.F64), ("f32", lbkm.F32)):
                p = dict(cfg["lib_params"])
                bc = (p.pop("bc_x"), p.pop("bc_y"))
                s = lbkm.Solver24(precision=prec, bc=bc, stream=stream, **p)
                s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
                with torch.cuda.stream(stream):
                    s.step(args.warmup)
                    ms = time_steps(s, stream, steps)
                s.sync()
                n = p["nx"] * p["ny"]
                out["%s_%s" % (name, tag)] = dict(
                    mcell_per_s=n * steps / (ms * 1e-3) / 1e6, ms_per_step=ms / steps,
                    cells=n, steps=steps)
                s.close()
        # single- against multiple-relaxation-time cost (Sec. V, Table I: the paper's MRT
        # D2V24 takes 3 % longer than its SRT form on one CPU core): equal rates, no TNE,
        # the fast path (collision = 0) against the general kernel (collision = 1)
        cfg = cases[1][1]
        fl = cfg["fields"]
        steps = cases[1][2]
        for tag, prec in (("f64", lbkm.F64), ("f32", lbkm.F32)):
            for form, coll in (("srt", 0), ("mrt", 1)):
                p = dict(cfg["lib_params"])
                bc = (p.pop("bc_x"), p.pop("bc_y"))
                p["S"] = np.full(24, 5e4)
                s = lbkm.Solver24(precision=prec, bc=bc, stream=stream, collision=coll, **p)
                s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
                with torch.cuda.stream(stream):
                    s.step(args.warmup)
                    ms = time_steps(s, stream, steps)
                s.sync()
                n = p["nx"] * p["ny"]
                out["reactive2d_equal_rates_%s_%s" % (form, tag)] = dict(
                    mcell_per_s=n * steps / (ms * 1e-3) / 1e6, ms_per_step=ms / steps)
                s.close()
    peak, peak_kind = measured_peak()
    big = out["reactive2d_f32"]
    alg = 200 * big["cells"]  # 25 FP32 planes read and written per cell update
    achieved = alg / (big["ms_per_step"] * 1e-3) / 1e9
    line = {"metric": METRIC.replace("16 f_i", "24 f_i"), "value": out["detonation_f32"]["mcell_per_s"],
            "unit": "Mcell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "d2v24_detonation_5000x1",
                       "note": "the paper's D2V24 steady-detonation set (Sec. IV.A); 1 MB "
                               "state, L2-resident"},
            "cases": out,
            "cpu_baseline": dict(zip(("value", "sample", "cores"), cpu_oracle_rate_d2v24()),
                                 unit="Mcell-updates/s", kind="oracle"),
            "roofline_reactive2d_f32": {"bound": "alu", "achieved": achieved, "peak": peak,
                                        "unit": "GB/s", "frac": achieved / peak,
                                        "peak_kind": peak_kind,
                                        "note": "HBM fraction of the 2048^2 FP32 step; its "
                                                "FP64 conserved sums and recovery (1:58 FP64 "
                                                "rate) and the block transforms bound it"},
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def measure_adjoint(n_grad=1, steps=None):
    """Config 5: dJ/d(S, Q, omega1, omega2, rho0) of a 4000-step 1-D detonation of 8192
    cells (profile mismatch + integrated TNE), checkpoints every 64 steps, through
    lbkm_grad (host wall clock per gradient); against the plain FP64 forward run of the
    same length that central differences repeat twice per gradient entry. The same
    gradient with the FP32 forward (FP64 adjoint along the FP32 trajectory) beside it."""
    import torch
    from paper_1411_6697_gb300 import lbkm
    cfg = li.adjoint()
    base, tgt = cfg["base"], cfg["target"]
    q, fl = base["params"], base["fields"]
    steps = base["steps"] if steps is None else steps
    stream = torch.cuda.Stream()

    def solver(p, prec=lbkm.F64):
        s = lbkm.Solver(nx=p["nx"], ny=1, precision=prec, S=p["S"], Q=p["Q"], bc=(1, 0),
                        dy=p["dx"], stream=stream, **_shared_params(p))
        s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
        return s

    t = solver(tgt["params"])
    with torch.cuda.stream(stream):
        t.step(steps)
        t.sync()
    rho_t = t.macros()["rho"][0].copy()
    t.close()
    one = solver(q)
    with torch.cuda.stream(stream):
        one.step(3)
        one.sync()
        ms_fwd = time_steps(one, stream, steps)
    one.close()
    s = solver(q)
    g = s.grad(rho_t, steps, w_tne=cfg["w_tne"], checkpoint_every=cfg["checkpoint_every"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_grad):
        g = s.grad(rho_t, steps, w_tne=cfg["w_tne"], checkpoint_every=cfg["checkpoint_every"])
    sec = (time.perf_counter() - t0) / n_grad

    def objective_sec(sv):
        # J alone (lbkm_objective_value: the run and one d^2 reduction per state)
        sv.objective(rho_t, steps, w_tne=cfg["w_tne"], checkpoint_every=cfg["checkpoint_every"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        v = sv.objective(rho_t, steps, w_tne=cfg["w_tne"],
                         checkpoint_every=cfg["checkpoint_every"])
        return time.perf_counter() - t1, v["J"]

    sec_j, j_only = objective_sec(s)
    s.close()
    s32 = solver(q, lbkm.F32)
    g32 = s32.grad(rho_t, steps, w_tne=cfg["w_tne"], checkpoint_every=cfg["checkpoint_every"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_grad):
        g32 = s32.grad(rho_t, steps, w_tne=cfg["w_tne"],
                       checkpoint_every=cfg["checkpoint_every"])
    sec32 = (time.perf_counter() - t0) / n_grad
    sec32_j, j32_only = objective_sec(s32)
    s32.close()
    nx = q["nx"]
    n_scalar = 16 + 3               # S_1..S_16, Q, omega1, omega2
    n_entries = n_scalar + nx       # and the initial density field
    fd = 2 * ms_fwd * 1e-3          # one central difference = two forward runs
    return {"workload": "adjoint_%dx1_detonation_%d_steps" % (nx, steps), "checkpoint_every":
            cfg["checkpoint_every"], "w_tne": cfg["w_tne"], "J": g["J"],
            "gradient_ms": sec * 1e3, "plain_f64_forward_ms": ms_fwd,
            "objective_only_ms": sec_j * 1e3, "objective_only_J": j_only,
            "plain_f64_forward_mcell_per_s": nx * steps / (ms_fwd * 1e-3) / 1e6,
            "gradient_over_forward": sec / (ms_fwd * 1e-3),
            "speedup_vs_central_fd_scalars": n_scalar * fd / sec,
            "speedup_vs_central_fd_all_entries": n_entries * fd / sec,
            "gradient_entries": n_entries,
            "accuracy": "J, dJ/dS, dJ/dQ, dJ/domega1 within 1e-7 of the FP64 reverse-mode oracle "
                        "at this size, within 1e-5 of central differences "
                        "(tests/test_gpu_adjoint.py)",
            "fp32_forward": {
                "gradient_ms": sec32 * 1e3, "J": g32["J"],
                "objective_only_ms": sec32_j * 1e3, "objective_only_J": j32_only,
                "speedup_vs_f64_gradient": sec / sec32,
                "speedup_vs_central_fd_scalars": n_scalar * fd / sec32,
                "method": "FP32 forward run and checkpoints; each segment recomputed and "
                          "reversed in FP64 from its widened checkpoint",
                "accuracy": "equals the FP64 oracle restarted from the same FP32 checkpoints "
                            "to 1e-7; against the FP64 forward's gradient J, dJ/dQ, "
                            "dJ/domega1 within 3.3e-5, 4.8e-4, 1.0e-3, while dJ/dS and dJ/drho0 "
                            "are amplified by the linearisation about FP32 states over 4000 "
                            "steps (tests/test_gpu_adjoint.py::"
                            "test_adjoint_of_the_fp32_forward_full_config)"}}


def run_adjoint(args):
    """One lbkm_grad call per step (host wall clock) for config 5."""
    import torch
    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    n_grad = max(1, min(args.steps, 3))
    with ClockSampler(local) as clk:
        a = measure_adjoint(n_grad, args.adjoint_steps)
    nx, steps = 8192, args.adjoint_steps
    line = {"metric": METRIC, "value": nx * steps / (a["gradient_ms"] * 1e-3) / 1e6,
            "unit": "Mcell-updates/s (forward-equivalent, per gradient)", "n_gpus": 1,
            "steps": n_grad, "warmup": 1, "ms_per_step": a["gradient_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": a["workload"], "checkpoint_every": a["checkpoint_every"],
                       "w_tne": a["w_tne"],
                       "step": "one lbkm_grad call (forward with checkpoints, replay, "
                               "reverse sweep), host wall clock"},
            "clocks": clk.summary()}
    line.update({k: v for k, v in a.items() if k not in ("workload", "checkpoint_every", "w_tne")})
    print(json.dumps(line))
    return 0


def measure_reactive(side, precision, recovery, steps, T_ig=1.0):
    """Mcell-updates/s of `steps` steps of the reactive field (CUDA events)."""
    import torch
    from paper_1411_6697_gb300 import lbkm
    cfg = li.reactive2d(n=side, steps=1, T_ig=T_ig)
    stream = torch.cuda.Stream()
    s = make_solver(cfg, precision, recovery, stream=stream)
    fl = cfg["fields"]
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    with torch.cuda.stream(stream):
        s.step(3)
        ms = time_steps(s, stream, steps)
    s.close()
    return side * side * steps / (ms * 1e-3) / 1e6, ms / steps


def measured_f64_peak():
    """cuBLAS FP64 GEMM throughput on this GPU (4096^3, best of 3): the FP64 peak the plain
    FP64 step is reported against."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * 4096 ** 3 / (best * 1e-3) / 1e12


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--recovery", default="f64", choices=["f64", "df32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--side", type=int, default=N_CELLS_SIDE)
    ap.add_argument("--adjoint-steps", type=int, default=4000,
                    help="steps of the adjoint workload (4000; fewer only for profiling)")
    ap.add_argument("--workload", default="reactive2d",
                    choices=["reactive2d", "batched", "detonation", "adjoint", "d2v24"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "detonation":
        return run_detonation(args)
    if args.workload == "d2v24":
        return run_d2v24(args)

    import torch
    import torch.distributed as dist

    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_1411_6697_gb300 import lbkm
    prec = lbkm.F32 if args.precision == "f32" else lbkm.F64
    rec = lbkm.RECOVER_F64 if args.recovery == "f64" else lbkm.RECOVER_DF32
    cfg = li.reactive2d(n=args.side, steps=500)
    n = args.side * args.side
    stream = torch.cuda.Stream()
    solver = make_solver(cfg, prec, rec, stream=stream)
    fl = cfg["fields"]
    solver.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    with torch.cuda.stream(stream):
        if args.warmup:
            solver.step(args.warmup)
        solver.sync()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ms = time_steps(solver, stream, args.steps)
        solver.sync()
    ms_max = max_over_ranks(ms, "cuda", world)
    value = world * n * args.steps / (ms_max * 1e-3) / 1e6
    per_launch_ms = ms / args.steps
    tag = "f32" if prec == lbkm.F32 else "f64"
    alg_bytes = BYTES_PER_CELL[tag] * n
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    kernel = "march" if (prec == lbkm.F32 and args.side > 1) else "step"
    traffic = profile_traffic(kernel, tag + ("_df32" if rec == lbkm.RECOVER_DF32 else ""))

    # end to end through the C ABI with pinned host buffers: H2D of the initial fields,
    # the steps, D2H of the macroscopic fields and of the TNE history
    pinned = {k: torch.from_numpy(np.ascontiguousarray(
        np.broadcast_to(fl[k], (args.side, args.side)))).pin_memory() for k in fl}
    outs = {k: torch.empty((args.side, args.side), dtype=torch.float64).pin_memory()
            for k in ("rho", "ux", "uy", "T", "p", "lam")}
    e2e_steps = args.steps
    # one untimed pass first, as the device-timed steps have their warm-up: the first
    # touch of the pinned buffers and of the library's temporaries stays out of the timing
    with torch.cuda.stream(stream):
        solver.init_fields(pinned["rho"], pinned["ux"], pinned["uy"], pinned["T"],
                           pinned["lam"])
        solver.step(max(args.warmup, 1))
        solver.macros(out=outs)
        solver.tne_history(max_records=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        solver.init_fields(pinned["rho"], pinned["ux"], pinned["uy"], pinned["T"],
                           pinned["lam"])
        solver.step(e2e_steps)
        solver.macros(out=outs)
        hist = solver.tne_history(max_records=e2e_steps)
    t_e2e = time.perf_counter() - t0
    e2e_value = n * e2e_steps / t_e2e / 1e6
    h2d = 5 * n * 8
    d2h = 6 * n * 8 + len(hist) * 8 * 67

    line = {
        "metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": tag, "data": "synthetic",
        "config": {"workload": "reactive2d_%dx%d" % (args.side, args.side),
                   "cells_per_gpu": n, "precision": tag,
                   "conserved_moment_recovery": args.recovery,
                   "tne": "every step; per-thread sums of Delta_k, |Delta_k| exact, "
                          "FP64 across threads, blocks and the grid",
                   "l2": "state %.2f GB per copy > L2 (129 MB): no flush" % (
                       17 * n * (4 if tag == "f32" else 8) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": ("march_kernel<%d> (f32)" % rec) if kernel == "march"
                     else "step_kernel (%s)" % tag,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "duration": "CUDA events over the timed steps, each the step kernel "
                                 "and the few-microsecond TNE finish kernel"},
        "e2e": {"value": e2e_value, "unit": "Mcell-updates/s",
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "note": "init_fields from pinned host + %d steps + macros to pinned host + "
                        "TNE history" % e2e_steps},
        # per step: the fused step kernel and the TNE record finish
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }

    if rank == 0 and not args.no_variants:
        var = {}
        for name, pr, rc in (("f32_recover_f64", lbkm.F32, lbkm.RECOVER_F64),
                             ("f32_recover_df32", lbkm.F32, lbkm.RECOVER_DF32),
                             ("f64_plain", lbkm.F64, lbkm.RECOVER_F64)):
            if pr == prec and rc == rec:
                var[name] = value / world
                continue
            s2 = make_solver(cfg, pr, rc, stream=stream)
            s2.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
            with torch.cuda.stream(stream):
                s2.step(3)
                k = 20 if pr == lbkm.F32 else 4
                t = time_steps(s2, stream, k)
            var[name] = n * k / (t * 1e-3) / 1e6
            s2.close()
        line["variants_mcell_per_s"] = var
        # the same field at the paper's ignition threshold T_ig = 1.1 (T stays below 1.05:
        # nothing ignites; reported beside the T_ig = 1.0 workload)
        r11, ms11 = measure_reactive(args.side, lbkm.F32, lbkm.RECOVER_F64, 20, T_ig=1.1)
        line["reactive2d_tig_1_1"] = {"mcell_per_s": r11, "ms_per_step": ms11,
                                      "hbm_frac": BYTES_PER_CELL["f32"] * n / (ms11 * 1e-3) / 1e9 / peak}
        # the plain FP64 form: FP64 operations per cell counted by ncu on this kernel
        f64_peak = measured_f64_peak()
        flop = (var["f64_plain"] * 1e6 * F64_FLOP_PER_CELL / 1e12) if F64_FLOP_PER_CELL else None
        line["f64_plain"] = {"mcell_per_s": var["f64_plain"],
                             "fp64_flop_per_cell": F64_FLOP_PER_CELL,
                             "fp64_tflops": flop, "fp64_peak_tflops": f64_peak,
                             "peak_kind": "measured cuBLAS FP64 GEMM (4096^3)",
                             "frac": flop / f64_peak if flop else None,
                             "flop_count": F64_FLOP_SOURCE}
        # single- against multiple-relaxation-time cost (Sec. V, Table I: the paper's MRT
        # D2V24 takes 3 % longer than its SRT form on one CPU core): equal rates, no TNE,
        # the fast path (collision 0) against the moment-space kernel (collision 1)
        eq = {}
        for form, coll in (("srt", 0), ("mrt", 1)):
            s3 = make_solver(cfg, lbkm.F32, lbkm.RECOVER_F64, stream=stream, tne_every=0,
                             S=np.full(16, 5e4), collision=coll)
            s3.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
            with torch.cuda.stream(stream):
                s3.step(3)
                t3 = time_steps(s3, stream, 20)
            eq[form + "_mcell_per_s"] = n * 20 / (t3 * 1e-3) / 1e6
            s3.close()
        eq["mrt_over_srt_time"] = eq["srt_mcell_per_s"] / eq["mrt_mcell_per_s"]
        line["equal_rates_no_tne"] = eq
        # configs 4 and 5: speed-ups over the plain single-instance FP64 form
        line["batched"] = measure_batched(200, 5)
        line["adjoint"] = measure_adjoint(1)
    if rank == 0 and not args.no_cpu_baseline:
        rate, desc, cores = cpu_oracle_rate()
        rate1, desc1 = cpu_oracle_rate_single()
        line["cpu_baseline"] = {"value": rate, "unit": "Mcell-updates/s", "cores": cores,
                                "kind": "oracle", "sample": desc,
                                "single_thread": {"value": rate1, "sample": desc1}}
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
