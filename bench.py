#!/usr/bin/env python3
"""Throughput of the two-component D3Q19 multiscale LB step on GB300.

Workload: synthetic multiscale rock, 128^3 cells (20% solid Gaussian field,
~19% gray cells with Kozeny-Carman/Brooks-Corey/Corey curves, CSF
kappa = -0.045 in gray cells), component A driven from the x < 8 slab by a
body force 1e-5 into the wetting component B.  One benchmark step is one full
LB time step over the whole lattice (all kernels of the step).

Prints one JSON line (rank 0).  Metric: MLUPS over all N^3 cells, whole job.
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank advances its own replica (weak scaling); the
timed region is bracketed by barriers and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM-roofline % of 2-comp D3Q19 step; mixed/adjoint/batched vs plain FP32"
C_OBS_BYTES = 16 * 8  # the observables row read back per step
STORAGE_IDS = {"f32": 0, "f16": 1, "bf16": 2, "f16r": 3, "bf16r": 4}
WORKLOAD = "drainage in synthetic multiscale rock, 128^3, 2-component D3Q19, FP32"
EDGE = 128
FALLBACK_HBM_GBS = 6800.0


# --------------------------------------------------------------------- inputs
def workload_inputs(edge=EDGE):
    from paper_2512_21696_gb300 import synth
    cell, phi, ptype = synth.drainage_geometry(edge, synth.SEED_BASE + 1)
    rA, rB = synth.drainage_fields(cell, 1.0, 0.03)
    return dict(cell=cell, phi=phi.astype(np.float32), ptype=ptype, rhoA=rA.astype(np.float32),
                rhoB=rB.astype(np.float32))


SETTINGS = dict(G=1.1, kappa_csf=-0.045, body_accel=((1e-5, 0.0, 0.0), (0.0, 0.0, 0.0)), rho_wall=(0.03, 1.0),
                wet_idx=1)


def fiber_inputs(edge=192, axis=0):
    """Tensorial-resistivity fibre bundle: 400 seeded cylinders (r = 1.5, vMF
    kappa = 20 axes), gray where phi < 0.99, no solid; wetting B at rho_hi
    everywhere with A dissolved, body force 1e-5 on B along `axis`."""
    from paper_2512_21696_gb300 import synth
    cell, phi, ptype, _ = synth.fiber_bundle_geometry(edge, synth.SEED_BASE + 3)
    acc = [0.0, 0.0, 0.0]
    acc[axis] = 1e-5
    inp = dict(cell=cell, phi=phi.astype(np.float32), ptype=ptype,
               rhoA=np.full(cell.shape, 0.03, np.float32), rhoB=np.full(cell.shape, 1.0, np.float32))
    settings = dict(G=1.1, kappa_csf=-0.045, body_accel=((0.0, 0.0, 0.0), tuple(acc)), rho_wall=(0.03, 1.0),
                    wet_idx=1)
    return inp, settings, dict(aniso=10.0)


def algorithmic_bytes(cell):
    """Bytes each kernel must move per launch: 304 B per fluid cell (two
    components x 19 FP32 populations, read and written), 1 B cell type per
    cell and 25 B per gray cell (porosity, principal axis, residual state;
    the kernels' own gray record is 32 B, but the figure is the method's);
    the two-launch kernels add the 8 B of densities they exchange."""
    n = cell.size
    fluid = int((cell != 1).sum())
    gray = int((cell == 2).sum())
    step = fluid * 304 + n * 1 + gray * 25
    return dict(step=step,
                step_lp=fluid * 152 + n * 1 + gray * 25,
                step_r16=fluid * 160 + n * 1 + gray * 25,
                k_fused=fluid * 304 + n * 1 + gray * 25,
                k_march=fluid * 304 + n * 1 + gray * 25,
                k_fused_lp=fluid * 152 + n * 1 + gray * 25,
                k_collide=fluid * 304 + n * 1 + n * 8 + gray * 25,
                k_density=fluid * 152 + n * 1 + n * 8), fluid, gray


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources that define the fused step kernel, its launch configuration and
# the per-grid tile choice: a committed ncu summary's traffic figure is used
# only while these are unchanged since its capture.
KERNEL_SOURCES = ("lbm_cell.cuh", "lbm_common.cuh", "lbm_fused.cuh", "lbm_fused_launch.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2512_21696_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_drainage128.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha:\s*(\w+)", text)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return float(m.group(1))


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.samples = []
        self.proc = None
        self.dev = device_index
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return None
        t0, t1 = self.window or (0, float("inf"))
        inwin = [p for (t, p) in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [p for _, p in self.samples]
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in inwin if num(p[1]) is not None]
        mx = [num(p[2]) for p in inwin if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in inwin for k in range(4) if p[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inwin)}


# ------------------------------------------------------------ aggregation
def max_over_ranks(value, dist, device):
    """Largest per-rank value: the job ends with its slowest rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist, device):
    """Sum of a per-rank scalar (host-side reporting only)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_mlups(cells, steps, world, ms):
    """Whole-job throughput: every rank advances its own replica of `cells`."""
    return world * cells * steps / (ms * 1e-3) / 1e6


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2512_21696_gb300 import lbm
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.workload == "fiber":
        inp, settings, constitutive = fiber_inputs()
        workload = ("tensorial fibre bundle, 192^3, 400 cylinders, anisotropy 10, body force on B along x, "
                    "2-component D3Q19, FP32")
    else:
        inp, settings, constitutive, workload = workload_inputs(), SETTINGS, {}, WORKLOAD
    cell = inp["cell"]
    nz, ny, nx = cell.shape
    n = cell.size
    stream = torch.cuda.current_stream()
    p = lbm.lbm_default_params(nx, ny, nz, stream=stream.cuda_stream, storage=STORAGE_IDS[args.storage], **settings)
    ctx = lbm.lbm_create(p)
    lbm.lbm_set_kernel(ctx, args.path, args.tile)
    _, tile_used = lbm.lbm_get_kernel(ctx)
    lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive(**constitutive))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in inp.items()}
    lbm.lbm_set_geometry(ctx, dev["cell"], dev["phi"], dev["ptype"])
    lbm.lbm_init_fields(ctx, dev["rhoA"], dev["rhoB"])

    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        lbm.lbm_step(ctx, 1)
    torch.cuda.synchronize()

    launches0 = lbm.lbm_launch_count(ctx)
    lbm.lbm_profile(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    lbm.lbm_step(ctx, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if dist:
        dist.barrier()
    clocks.mark(t_wall0, t_wall1)
    ms = ev0.elapsed_time(ev1)
    prof = lbm.lbm_profile_read(ctx)
    lbm.lbm_profile(ctx, False)
    launches = lbm.lbm_launch_count(ctx) - launches0
    ms = max_over_ranks(ms, dist, "cuda")
    obs = lbm.lbm_observables(ctx, check=False)

    # end-to-end through the public API with pinned host buffers
    host = {k: torch.from_numpy(np.ascontiguousarray(inp[k])).pin_memory() for k in ("rhoA", "rhoB")}
    outs = [torch.empty(s, dtype=torch.float32).pin_memory() for s in ((nz, ny, nx), (nz, ny, nx), (3, nz, ny, nx),
                                                                       (nz, ny, nx))]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the initial fields go up from pinned host memory; every step then reads
    # its result (the observables: masses, saturation, fluxes) back into its
    # own slot of pinned host memory, as a monitoring loop does, without
    # stalling the stream; the final fields come down at the end
    raw = torch.zeros((args.steps, lbm.LBM_OBS_RAW), dtype=torch.float64).pin_memory()
    row = raw.stride(0) * raw.element_size()
    e0 = time.perf_counter()
    lbm.lbm_init_fields(ctx, host["rhoA"].numpy(), host["rhoB"].numpy())
    for k in range(args.steps):
        lbm.lbm_step(ctx, 1)
        lbm.lbm_observables_async(ctx, raw.data_ptr() + k * row)
    lbm.lbm_get_fields(ctx, *[o.numpy() for o in outs])  # synchronises the stream
    obs_all = [lbm.lbm_obs_decode(ctx, raw.data_ptr() + k * row, check=False) for k in range(args.steps)]
    e_ms = (time.perf_counter() - e0) * 1e3
    obs_e2e = obs_all[-1]
    assert [o["step"] for o in obs_all] == list(range(1, args.steps + 1))
    e_ms = max_over_ranks(e_ms, dist, "cuda")
    clocks.stop()
    ctx.close()

    if obs["nan_count"] or obs_e2e["nan_count"]:
        # a step whose fields went non-finite has no throughput to report
        raise SystemExit(f"bench: non-finite fields after the timed steps ({obs['nan_count']} cells)")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    alg, fluid, gray = algorithmic_bytes(cell)
    mlups = job_mlups(n, args.steps, world, ms)
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("k_collide", (args.steps, ms))
    dname, (dlaunch, dtotal) = dom
    avg_s = dtotal / max(dlaunch, 1) * 1e-3
    peak, peak_kind = measured_peak()
    step_key = {"f32": "step", "f16": "step_lp", "bf16": "step_lp"}.get(args.storage, "step_r16")
    dkey = dname if args.storage in ("f32", "f16", "bf16") else "step_r16"
    achieved = alg.get(dkey, alg[step_key]) / avg_s / 1e9
    step_gbs = alg[step_key] * args.steps / (ms * 1e-3) / 1e9
    h2d = 2 * n * 4
    d2h = 6 * n * 4 + args.steps * C_OBS_BYTES
    out = {
        "metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded multiscale-rock recipe)",
        "config": {"workload": workload if args.storage == "f32" else workload.replace("FP32", f"{args.storage.upper()} storage, FP32 arithmetic"),
                   "storage": args.storage, "cells": n, "fluid_frac": round(fluid / n, 4),
                   "gray_frac": round(gray / n, 4), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (2 x 319 MB population buffers)",
                   "kernels_per_step": round(launches / args.steps, 3),
                   "path": args.path, "tile": {"requested": args.tile, "in_use": tile_used}},
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "frac_of_nominal_8tbs": round(achieved / 8000.0, 4),
                     # the committed capture is of the F32 drainage launch with the default tile
                     "traffic": ncu_traffic(dname) if (args.storage == "f32" and args.workload == "drainage"
                                                       and args.path == 0 and args.tile == 8) else None,
                     "alg_bytes_per_launch": alg.get(dkey, alg[step_key]),
                     "avg_launch_ms": round(avg_s * 1e3, 5)},
        "mflups": round(job_mlups(fluid, args.steps, world, ms), 2),  # non-solid cells only
        "step_roofline": {"alg_bytes_per_cell": round(alg[step_key] / n, 2), "achieved_gbs": round(step_gbs, 1),
                          "frac": round(step_gbs / peak, 4)},
        "kernels": {k: {"launches": v[0], "avg_ms": round(v[1] / max(v[0], 1), 5)} for k, v in prof.items()},
        "e2e": {"value": round(job_mlups(n, args.steps, world, e_ms), 2), "unit": "MLUPS",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "ms_total": round(e_ms, 3)},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "observables": {"mass": obs["mass"], "sat": obs["sat"], "nan_count": obs["nan_count"],
                        "e2e_nan_count": obs_e2e["nan_count"]},
    }
    if args.workload == "fiber":
        # Darcy: K_x = <u_x> nu / g over all cells (tau = 1), at the step reached
        out["permeability_x_at_step"] = {"K": obs["flux_vol"][0] * (0.5 / 3.0) / 1e-5, "step": obs["step"]}
    if world == 1 and not args.no_cpu_baseline and args.workload == "drainage":
        out["cpu_baseline"] = cpu_baseline(inp, budget_s=args.cpu_budget)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------ oracle timing
def _oracle_slab(inp, nzs):
    """Oracle on the first nzs z-planes of the workload (a bounded sample)."""
    import oracle as O
    from paper_2512_21696_gb300 import synth
    cell = np.ascontiguousarray(inp["cell"][:nzs])
    shape = cell.shape
    p = O.make_params(shape, G=SETTINGS["G"], kappa=SETTINGS["kappa_csf"], accel=SETTINGS["body_accel"],
                      rho_wall=SETTINGS["rho_wall"], wet=SETTINGS["wet_idx"])
    o = O.Oracle(p, cell, inp["phi"][:nzs].astype(np.float64), ptype=inp["ptype"][:nzs], curves=[O.make_curve()])
    o.init_fields(inp["rhoA"][:nzs].astype(np.float64), inp["rhoB"][:nzs].astype(np.float64))
    return o, int(np.prod(shape))


def cpu_baseline(inp, budget_s=15.0):
    import oracle as O
    O.build()
    o, cells = _oracle_slab(inp, inp["cell"].shape[0])
    t = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t
    k = max(1, int(budget_s / max(one, 1e-3)))
    t = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t
    cores = O.max_threads()
    # the same oracle on one core, on a slab of 8 planes (a few seconds)
    o1, cells1 = _oracle_slab(inp, 8)
    O.set_threads(1)
    try:
        o1.step(1)
        t = time.perf_counter()
        o1.step(2)
        dt1 = time.perf_counter() - t
    finally:
        O.set_threads(cores)
    return {"value": round(cells * k / dt / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"full 128^3 workload, {k} timed FP64 steps after 1 untimed ({dt:.1f} s)",
            "one_core": {"value": round(cells1 * 2 / dt1 / 1e6, 3), "unit": "MLUPS",
                         "sample": "8 of 128 z-planes, 2 timed steps after 1 untimed"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    O.build()
    inp = workload_inputs()
    nz = inp["cell"].shape[0]
    budget = 150.0 / max(args.steps + args.warmup, 1)
    probe, _ = _oracle_slab(inp, 8)
    t = time.perf_counter()
    probe.step(1)
    per_plane = (time.perf_counter() - t) / 8
    nzs = int(min(nz, max(1, budget / max(per_plane, 1e-6))))
    o, cells = _oracle_slab(inp, nzs)
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    mlups = cells * args.steps / dt / 1e6
    sample = f"first {nzs} of {nz} z-planes of the 128^3 workload per step"
    out = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded multiscale-rock recipe)",
           "config": {"workload": WORKLOAD, "cells": cells, "sample": sample},
           "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": O.max_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------- batched REV library
REV_KINDS = ("spheres", "grf", "fibers", "slits")


def rev_library(nruns, seed, first=0):
    """Fully resolved REV runs first .. first + nruns - 1 of one seeded
    library: edge ~ U{24..64}, pore type round robin (the same run index
    gives the same REV whatever slice it is generated in)."""
    from paper_2512_21696_gb300 import synth
    rng = np.random.default_rng(seed)
    edges = rng.integers(24, 65, size=first + nruns)
    return [(int(edges[r]), REV_KINDS[r % 4]) + synth.rev_geometry(int(edges[r]), REV_KINDS[r % 4],
                                                                   seed + 1000 * (r + 1))[:2]
            for r in range(first, first + nruns)]


def rev_slice(runs_per_rank, rank):
    """The library runs of one rank: each rank advances its own runs_per_rank
    REVs (weak scaling over independent problems, no data-path collective)."""
    return rank * runs_per_rank, runs_per_rank


def run_rev(args, rank=0, world=1, local_rank=0):
    """Single-phase permeability runs of a REV library (wetting B at rho_hi,
    A dissolved at rho_lo, g = 1e-4 on B along x, nu = 0.012): all runs in one
    batch (persistent launch per step, CUDA-graph replay, tuned tiles) against
    the same runs stepped one after another.  Under torchrun every rank runs
    its own --rev-runs REVs of the library (weak scaling; the time is the
    slowest rank's, the cells are summed)."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    first, count = rev_slice(args.rev_runs, rank)
    lib = rev_library(count, synth.SEED_BASE + 5, first)
    stream = torch.cuda.current_stream()
    tau = 3 * 0.012 + 0.5
    g = 1e-4
    runs = [lbm.lbm_default_params(e, e, e, stream=stream.cuda_stream, storage=STORAGE_IDS[args.storage],
                                   G=1.1, tau=(tau, tau), rho_wall=(0.03, 1.0), wet_idx=1,
                                   body_accel=((0, 0, 0), (g, 0, 0))) for e, _, _, _ in lib]
    b = lbm.lbm_batch_create(runs)
    views = [lbm.lbm_batch_run(b, r) for r in range(len(lib))]
    for v, (e, kind, cell, phi) in zip(views, lib):
        lbm.lbm_set_geometry(v, cell, phi.astype(np.float32))
        lbm.lbm_init_fields(v, np.full(cell.shape, 0.03, np.float32), np.full(cell.shape, 1.0, np.float32))
    cells = sum(c.size for _, _, c, _ in lib)
    fluid = sum(int((c != 1).sum()) for _, _, c, _ in lib)
    t0 = time.time()
    tiles = lbm.lbm_batch_tune(b, 6)
    tune_s = time.time() - t0
    lbm.lbm_batch_step(b, args.warmup + (args.warmup & 1))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = args.steps + (args.steps & 1)
    lbm.lbm_batch_step(b, steps)  # captures the graph
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0.record(stream)
    lbm.lbm_batch_step(b, steps)  # replays it
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_batch = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    cells_all = sum_over_ranks(sum(c.size for _, _, c, _ in lib), dist, "cuda")
    info = lbm.lbm_batch_info(b)
    # the same runs one after another (each its own single-lattice launches)
    ev0.record(stream)
    for v in views:
        lbm.lbm_step(v, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    nu = (tau - 0.5) / 3.0
    kperm = {}
    taken = 0
    for v, (e, kind, cell, phi) in zip(views, lib):
        o = lbm.lbm_observables(v, check=False)
        kperm.setdefault(kind, []).append(o["flux_vol"][0] * nu / g)
        taken = o["step"]
    steady = None
    if args.steady_max > 0:
        # continue every run to steady flow (mean velocity changing by at most
        # 1e-5 of itself over 500 steps), untimed; K is then the Darcy value
        t0 = time.time()
        ok, done = lbm.lbm_batch_step_to_steady(b, 500, 1e-5, args.steady_max)
        wall = time.time() - t0
        ks = {}
        for o, (e, kind, cell, phi) in zip(lbm.lbm_batch_observables(b), lib):
            ks.setdefault(kind, []).append(o["flux_vol"][0] * nu / g)
        steady = {"reached": bool(ok), "extra_steps": done, "wall_s": round(wall, 2),
                  "K": {k: round(float(np.mean(v)), 6) for k, v in ks.items()}}
    b.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    mlups = cells_all * steps / (ms_batch * 1e-3) / 1e6
    out = {"metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": ms_batch / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded REV pore types)",
           "config": {"workload": f"batched REV library: {len(lib)} single-phase runs per GPU, edge U{{24..64}}, "
                                  "pore types spheres/grf/fibers/slits round robin",
                      "storage": args.storage, "cells": int(cells_all), "fluid_frac": round(fluid / cells, 4),
                      "parallelism": f"runs split x{world}", "l2": "inputs larger than L2"},
           "sequential": {"value": round(cells_all * steps / (ms_seq * 1e-3) / 1e6, 2), "unit": "MLUPS",
                          "ms_per_step": ms_seq / steps},
           "batched_over_sequential": round(ms_seq / ms_batch, 3),
           "gpu_launches": info["groups"] * steps, "launches_per_step": info["groups"],
           "tiles": {t: tiles.count(t) for t in sorted(set(tiles))}, "tune_s": round(tune_s, 2),
           "permeability_at_step": {k: round(float(np.mean(v)), 6) for k, v in kperm.items()},
           "steps_taken": taken}
    if steady is not None:
        out["steady_state"] = steady
    print(json.dumps(out), flush=True)


def run_revlib(args):
    """REV library generation (the workflow's step ii) on a subset: for each of
    --rev-runs REVs (pore types round robin) one single-phase run and eight
    two-phase runs at Sw = 0.2 ... 0.9, all in one batch.  In a periodic REV
    each component's mass is conserved, so the saturation set at t = 0 holds;
    both components feel the same acceleration g along x.  With
    --steady-max, the mass-sink-source controller first brings every two-phase
    run to its target Sw (the fill only approximates it) and the batch then
    steps to steady flow (the Appendix's controller and MSS).  After --steps:
    K = <u_x> nu / g (single phase), Kr_a = q_a / q_single with
    q_a = <(rho_a/rho) u_x>, Pc = mean p of non-wetting-rich cells minus
    mean p of wetting-rich cells, p = (rhoA + rhoB)/3 + G rhoA rhoB."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    seed = synth.SEED_BASE + 5
    lib = rev_library(args.rev_runs, seed)
    stream = torch.cuda.current_stream()
    # tau = 1 for every run: at the paper's Kr viscosity (tau 0.51) and at
    # nu = 0.012 (tau 0.536) many two-phase runs of this step turn non-finite;
    # Kr = q_a / q_single and K = <u> nu / g do not depend on nu in the Darcy
    # regime, and the viscous time scale is shorter at tau = 1
    tau, g, G = 1.0, 1e-4, 1.1
    sws = [0.2 + 0.1 * k for k in range(8)]
    runs, inits = [], []
    for r, (e, kind, cell, phi) in enumerate(lib):
        for k, sw in enumerate([None] + sws):
            runs.append(lbm.lbm_default_params(e, e, e, stream=stream.cuda_stream, G=G, tau=(tau, tau),
                                               rho_wall=(0.03, 1.0), wet_idx=1,
                                               body_accel=((g, 0, 0), (g, 0, 0)) if sw else ((0, 0, 0), (g, 0, 0))))
            if sw is None:
                rA, rB = np.full(cell.shape, 0.03), np.full(cell.shape, 1.0)
            else:
                # wetting B on the lowest-ranked fraction sw of the pore cells of a smooth field
                fld = synth.gaussian_random_field(cell.shape, max(2.0, e / 8.0), synth.rng_for(seed + 77 * r + k))
                pore = cell != synth.SOLID
                cut = np.quantile(fld[pore], sw)
                wet = pore & (fld <= cut)
                rA, rB = np.where(wet, 0.03, 1.0), np.where(wet, 1.0, 0.03)
            inits.append((cell, phi, rA.astype(np.float32), rB.astype(np.float32)))
    b = lbm.lbm_batch_create(runs)
    views = [lbm.lbm_batch_run(b, r) for r in range(len(runs))]
    for v, (cell, phi, rA, rB) in zip(views, inits):
        lbm.lbm_set_geometry(v, cell, phi.astype(np.float32))
        lbm.lbm_init_fields(v, rA, rB)
    cells = sum(int(np.prod(c.shape)) for c, _, _, _ in inits)
    tiles = lbm.lbm_batch_tune(b, 6)
    steps = args.steps + (args.steps & 1)
    control = None
    if args.steady_max > 0:
        # the fill only approximates each stage's saturation: the mass-sink-
        # source controller brings every two-phase run to its target Sw
        # (single-phase runs keep theirs), then all runs go to steady flow
        t0 = time.time()
        lbm.lbm_batch_step(b, 200)
        now = [o["sat"] for o in lbm.lbm_batch_observables(b, check=False)]
        targets = [now[r] if r % 9 == 0 else sws[r % 9 - 1] for r in range(len(runs))]
        hit, k_mss = lbm.lbm_batch_mss_to_saturation(b, targets, 0.05, 5e-3, 2e-3, 50, args.steady_max)
        steady, k_st = lbm.lbm_batch_step_to_steady(b, 500, 1e-4, args.steady_max)
        obs = lbm.lbm_batch_observables(b, check=False)
        bad = [r for r, o in enumerate(obs) if o["nan_count"] > 0]
        control = {"targets_reached": bool(hit), "mss_steps": k_mss, "steady": bool(steady), "steady_steps": k_st,
                   "wall_s": round(time.time() - t0, 2),
                   "sat_error_max": max((abs(o["sat"] - t) for r, (o, t) in enumerate(zip(obs, targets))
                                         if r not in bad), default=None),
                   "non_finite_runs": [{"run": r, "kind": lib[r // 9][1], "edge": lib[r // 9][0],
                                        "sw_target": None if r % 9 == 0 else sws[r % 9 - 1]} for r in bad]}
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lbm.lbm_batch_step(b, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    nu = (tau - 0.5) / 3.0
    curves = {}
    for r, (e, kind, cell, phi) in enumerate(lib):
        base = r * 9
        ra, rb, u, swf = lbm.lbm_get_fields(views[base])
        q1 = float(u[0].mean())
        ent = curves.setdefault(kind, dict(K=[], Sw=[], Krw=[], Krn=[], Pc=[]))
        ent["K"].append(q1 * nu / g)
        row = dict(Sw=[], Krw=[], Krn=[], Pc=[])
        for k in range(8):
            ra, rb, u, swf = lbm.lbm_get_fields(views[base + 1 + k])
            pore = cell != synth.SOLID
            rt = np.where(pore, ra + rb, 1.0)
            qw, qn = float((rb / rt * u[0])[pore].sum() / cell.size), float((ra / rt * u[0])[pore].sum() / cell.size)
            p = (ra + rb) / 3.0 + G * ra * rb
            nrich, wrich = pore & (ra > rb), pore & (rb > ra)
            row["Sw"].append(float(swf[pore].mean()))
            row["Krw"].append(qw / q1 if q1 else np.nan)
            row["Krn"].append(qn / q1 if q1 else np.nan)
            row["Pc"].append(float(p[nrich].mean() - p[wrich].mean()) if nrich.any() and wrich.any() else np.nan)
        for key in row:
            ent[key].append(row[key])
    b.close()
    def avg(rows, nd):
        with np.errstate(all="ignore"):
            m = np.nanmean(np.asarray(rows, dtype=np.float64), axis=0)
        return [round(float(x), nd) if np.isfinite(x) else None for x in np.atleast_1d(m)]

    summary = {kind: {"K": avg(v["K"], 6)[0], "Sw": avg(v["Sw"], 3), "Krw": avg(v["Krw"], 4),
                      "Krn": avg(v["Krn"], 4), "Pc": avg(v["Pc"], 6)} for kind, v in curves.items()}
    out = {"metric": METRIC, "value": round(cells * steps / (ms * 1e-3) / 1e6, 2), "unit": "MLUPS", "n_gpus": 1,
           "steps": steps, "warmup": 0, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded REV pore types)",
           "config": {"workload": f"REV library: {len(lib)} REVs x (single phase + 8 saturations) = {len(runs)} "
                                  "runs in one batch", "cells": cells, "storage": "f32"},
           "tiles": {t: tiles.count(t) for t in sorted(set(tiles))}, "library_at_step": summary,
           "saturation_control": control}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------ stepped-pressure imbibition
def run_imbibition(args):
    """Stepped-pressure imbibition (Sec. I; Pc(Sw) in the Appendix) on the
    96^3 multiscale-rock recipe: a wetting-B inlet reservoir plane at z = 0,
    a non-wetting-A outlet plane at z = 95 (z not periodic), the rock filled
    with A except a B slab at the inlet.  The outlet holds p_out; the inlet
    pressure is raised level by level, Pc = p_out - p_in from +0.04 to -0.02
    (p = (rhoA + rhoB)/3 + G rhoA rhoB), each level stepped to steady
    saturation (check every 500 steps, |dS| <= 1e-4, at most --level-max
    steps).  Reports the Pc-Sw pairs and MLUPS over the whole protocol."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    n, G, lo = 96, 1.1, 0.03
    cell, phi, ptype = synth.drainage_geometry(n, synth.SEED_BASE + 4)
    cell = cell.copy()
    cell[0], cell[-1] = synth.INLET, synth.OUTLET
    zz = np.arange(n)[:, None, None] + np.zeros(cell.shape, np.int64)
    rA = np.where(zz < 4, lo, 1.0).astype(np.float32)
    rB = np.where(zz < 4, 1.0, lo).astype(np.float32)
    stream = torch.cuda.current_stream()
    p = lbm.lbm_default_params(n, n, n, stream=stream.cuda_stream, G=G, kappa_csf=-0.045,
                               rho_wall=(lo, 1.0), wet_idx=1, periodic=(1, 1, 0), storage=STORAGE_IDS[args.storage])
    ctx = lbm.lbm_create(p)
    lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive())
    lbm.lbm_set_geometry(ctx, cell, phi.astype(np.float32), ptype)
    lbm.lbm_init_fields(ctx, rA, rB)
    pres = lambda major, minor: (major + minor) / 3.0 + G * major * minor
    p_out = pres(1.0, lo)
    pcs = [0.04, 0.03, 0.02, 0.01, 0.0, -0.01, -0.02]
    # inlet wetting density giving p_in = p_out - Pc with the minority at lo
    levels = [((lo, (p_out - pc - lo / 3.0) / (1.0 / 3.0 + G * lo)), (1.0, lo)) for pc in pcs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, sat, steps = lbm.lbm_pressure_levels(ctx, levels, 500, 1e-4, args.level_max)
    wall = time.perf_counter() - t0
    obs = lbm.lbm_observables(ctx, check=False)
    ctx.close()
    total = int(sum(steps))
    out = {"metric": METRIC, "value": round(cell.size * total / wall / 1e6, 2), "unit": "MLUPS", "n_gpus": 1,
           "steps": total, "warmup": 0, "ms_per_step": wall * 1e3 / total, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else args.storage,
           "data": "synthetic (seeded multiscale-rock recipe)",
           "config": {"workload": "stepped-pressure imbibition, 96^3 multiscale rock between reservoir planes, "
                                  f"{len(pcs)} levels, at most {args.level_max} steps each",
                      "cells": int(cell.size), "storage": args.storage,
                      "timing": "host wall clock around the protocol (steps + saturation checks)"},
           "all_levels_steady": bool(ok),
           "pc_sw": [{"Pc": pc, "rho_in_B": round(lv[0][1], 6), "Sw": round(s, 5), "steps": int(k)}
                     for pc, lv, s, k in zip(pcs, levels, sat, steps)],
           "nan_count": obs["nan_count"]}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------- 2-D droplet (D2Q9)
def run_droplet2d(args):
    """Sec. III.A on D2Q9: an oil droplet of radius 40 in water on a 100^2
    periodic plane (rho 1.0 / 0.03, G = 1.1, tau = 1), Eq. 4 off (kappa = 0)
    and on (kappa = -0.045, everywhere), --steps steps each.  Reports
    sigma = dp R (2-D Laplace law; R the mass-equivalent radius), the maximum
    |u_x| (the paper's spurious-current measure), the 10-90 % interface
    width on the centre line and the step rate; the paper's printed values
    are context (its G and psi are not given)."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    n, R = 100, 40
    shape = (1, n, n)
    rA, rB = synth.cylinder_droplet_fields(shape, R, (n // 2, n // 2), 1.0, 0.03)
    stream = torch.cuda.current_stream()
    rows = {}
    total_ms = 0.0
    for kappa in (0.0, -0.045):
        p = lbm.lbm_default_params(n, n, 1, stream=stream.cuda_stream, G=1.1, kappa_csf=kappa, csf_everywhere=1,
                                   lattice=1, probe_center=(n // 2, n // 2, 0), probe_r_in=R - 4.0,
                                   probe_r_out=R + 4.0)
        ctx = lbm.lbm_create(p)
        lbm.lbm_set_geometry(ctx, np.zeros(shape, np.uint8), np.ones(shape, np.float32))
        lbm.lbm_init_fields(ctx, rA.astype(np.float32), rB.astype(np.float32))
        lbm.lbm_step(ctx, args.warmup)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lbm.lbm_step(ctx, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        total_ms += ms
        obs = lbm.lbm_observables(ctx, check=False)
        a, b, u, sw = lbm.lbm_get_fields(ctx)
        ctx.close()
        lo, hi = float(a.min()), float(a.max())
        r_eq = float(np.sqrt((a.sum() - lo * a.size) / (hi - lo) / np.pi))
        line = a[0, n // 2, n // 2:]  # centre line, droplet centre outwards
        frac = (line - lo) / (hi - lo)
        width = float(np.count_nonzero((frac > 0.1) & (frac < 0.9)))
        rows[str(kappa)] = {"sigma": obs["dp"] * r_eq, "dp": obs["dp"], "R_eq": round(r_eq, 3),
                            "max_abs_ux": float(np.abs(u[0]).max()), "max_u": obs["max_u"],
                            "interface_width_10_90": width, "ms_per_step": ms / args.steps}
    ratio = rows["0.0"]["sigma"] / rows["-0.045"]["sigma"]
    cells = n * n
    out = {"metric": METRIC, "value": round(cells * 2 * args.steps / (total_ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "n_gpus": 1, "steps": 2 * args.steps, "warmup": args.warmup, "ms_per_step": total_ms / (2 * args.steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Sec. III.A droplet on D2Q9: R = 40 on 100^2, kappa 0 and -0.045",
                      "cells": cells, "l2": "fits in L2 (launch-bound)"},
           "gpu_launches": 2 * 2 * args.steps, "droplet": rows, "sigma_ratio_kappa0_over_kappa": round(ratio, 3),
           "paper_context": {"sigma": {"0": 0.026, "-0.045": 7.43e-4}, "max_ux": {"0": 6.43e-3, "-0.045": 6.45e-3}}}
    print(json.dumps(out), flush=True)


# --------------------------------------- 2-D imbibition, random porosity (D2Q9)
def run_imbibition2d(args):
    """Sec. III.B on D2Q9: water imbibition into a 100 x 100 under-resolved
    medium whose porosity is normally distributed about 0.5 (std 0.1 here,
    clipped to [0.1, 0.9]; the paper gives the mean only), walls left and
    right, a water inlet row on top and an oil outlet row at the bottom, Eq. 4
    with kappa = -0.045 in the gray cells.  Both viscosities are 1.66e-2
    (tau = 0.55, the paper's Sec. I.B value): at the Sec. III.B value 1.66e-3
    (tau = 0.505) this two-component step diverged within the first level.  The outlet pressure starts 10 % above the inlet's and is lowered
    in ten equal levels of --steps / 10 steps each (the paper's protocol).
    Reports the water saturation per level and the step rate."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    nx, ny, G, lo = 100, 102, 1.1, 0.03
    rng = synth.rng_for(synth.SEED_BASE + 10)
    phi = np.clip(0.5 + 0.1 * rng.standard_normal((1, ny, nx)), 0.1, 0.9).astype(np.float32)
    cell = np.full((1, ny, nx), synth.GRAY, np.uint8)
    cell[0, -1, :], cell[0, 0, :] = synth.INLET, synth.OUTLET  # water on top (y = ny - 1), oil below
    rA = np.where(cell == synth.INLET, lo, 1.0).astype(np.float32)
    rB = np.where(cell == synth.INLET, 1.0, lo).astype(np.float32)
    tau = 3 * 1.66e-2 + 0.5
    stream = torch.cuda.current_stream()
    p = lbm.lbm_default_params(nx, ny, 1, stream=stream.cuda_stream, G=G, kappa_csf=-0.045, tau=(tau, tau),
                               rho_wall=(lo, 1.0), wet_idx=1, periodic=(0, 0, 1), lattice=1)
    ctx = lbm.lbm_create(p)
    lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive())
    lbm.lbm_set_geometry(ctx, cell, phi)
    lbm.lbm_init_fields(ctx, rA, rB)
    pres = lambda major, minor: (major + minor) / 3.0 + G * major * minor
    p_in = pres(1.0, lo)
    # outlet oil density giving p_out = f p_in with the minority at lo
    levels = [((lo, 1.0), ((f * p_in - lo / 3.0) / (1.0 / 3.0 + G * lo), lo)) for f in np.linspace(1.10, 1.0, 10)]
    per = max(1, args.steps // 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, sat, steps = lbm.lbm_pressure_levels(ctx, levels, per, 1.0, per)  # a fixed number of steps per level
    wall = time.perf_counter() - t0
    obs = lbm.lbm_observables(ctx, check=False)
    a, b, u, sw = lbm.lbm_get_fields(ctx)
    ctx.close()
    inner = cell[0] == synth.GRAY
    speed = float(np.sqrt(u[0, 0] ** 2 + u[1, 0] ** 2)[inner].mean())
    total = int(sum(steps))
    out = {"metric": METRIC, "value": round(nx * ny * total / wall / 1e6, 2), "unit": "MLUPS", "n_gpus": 1,
           "steps": total, "warmup": 0, "ms_per_step": wall * 1e3 / total, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (normal porosity, seeded)",
           "config": {"workload": "Sec. III.B imbibition on D2Q9: 100 x 100 gray medium between reservoir rows, "
                                  "outlet pressure lowered from 1.10 to 1.00 of the inlet's in 10 levels",
                      "cells": nx * ny, "tau": tau, "timing": "host wall clock (steps + saturation checks)"},
           "levels": [{"p_out_over_p_in": round(float(f), 4), "Sw": round(s, 5)}
                      for f, s in zip(np.linspace(1.10, 1.0, 10), sat)],
           "mean_speed_gray": speed, "nan_count": obs["nan_count"]}
    print(json.dumps(out), flush=True)


# ------------------------------------------------- 2-D fibre zigzag (D2Q9)
def run_zigzag2d(args):
    """Single-phase flow through the zigzag pathway between two wavy-fibre
    bundles (Sec. I.B, Sec. III.E) on D2Q9: the pathway is open pore
    (phi = 1), the bundles gray with phi = 0.95; pressure rows on top and
    bottom in the paper's ratio 0.740 : 0.733 (p = rho_B / 3, component B
    alone: a dissolved A at rho_lo would bring the Eq. 1 drag of a component
    whose relative permeability is floored at kr_min), walls left and right,
    nu = 1.66e-2 (tau = 0.55), 120 x 180 cells between the pressure rows.
    Isotropic resistivity from K0(phi) against the tensorial one whose least
    component is 1e-4 K0 (Eq. 7).  Reports the fraction of the flux carried
    inside the pathway (mean over the rows), both runs, and the step rate."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    nx, ny, lo, hi = 120, 180, 0.03, 1.0
    cell, phi_all, path_all = synth.zigzag_pathway_geometry(nx, ny)
    path = path_all[:, 1:-1, :]
    rho_in = hi * 0.740 / 0.733
    stream = torch.cuda.current_stream()
    res, total_ms = {}, 0.0
    for aniso in (1.0, 1e4):
        p = lbm.lbm_default_params(nx, ny + 2, 1, stream=stream.cuda_stream, G=1.1, tau=(0.55, 0.55),
                                   rho_wall=(lo, hi), wet_idx=1, periodic=(0, 0, 1), lattice=1)
        ctx = lbm.lbm_create(p)
        lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive(aniso=aniso))
        lbm.lbm_set_geometry(ctx, cell, phi_all)
        lbm.lbm_init_fields(ctx, np.zeros(cell.shape, np.float32), np.full(cell.shape, hi, np.float32))
        lbm.lbm_set_pressure(ctx, (0.0, rho_in), (0.0, hi))
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lbm.lbm_step(ctx, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        obs = lbm.lbm_observables(ctx, check=False)
        a, b, u, sw = lbm.lbm_get_fields(ctx)
        ctx.close()
        uy = -u[1, 0, 1:-1, :]  # flow runs from the top row down
        inside = (uy * path[0]).sum(axis=1) / uy.sum(axis=1)
        res["tensorial" if aniso > 1 else "isotropic"] = {
            "pathway_flux_fraction": round(float(inside.mean()), 4),
            "pathway_width_fraction": round(float(path.mean()), 4),
            "flux_per_row": float(uy.sum(axis=1).mean()), "nan_count": obs["nan_count"]}
    cells = nx * (ny + 2)
    out = {"metric": METRIC, "value": round(cells * 2 * args.steps / (total_ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "n_gpus": 1, "steps": 2 * args.steps, "warmup": 0, "ms_per_step": total_ms / (2 * args.steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (zigzag pathway between gray fibre bundles)",
           "config": {"workload": "Sec. I.B / III.E zigzag pathway on D2Q9: 120 x 180, open pathway between "
                                  "phi = 0.95 fibre bundles, pressure rows, isotropic vs tensorial resistivity",
                      "cells": cells},
           "gpu_launches": 2 * 2 * args.steps, "zigzag": res}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ static droplet
def run_droplet(args):
    """32^3 static droplet (R = 8, rho 1.0/0.03, G = 1.1, tau = 1): the state
    fits in L2, so the step is launch-bound; it runs as a one-lattice batch,
    whose steps are replayed from a CUDA graph.  Reported as us per step."""
    import torch
    from paper_2512_21696_gb300 import lbm, synth
    torch.cuda.set_device(0)
    shape = (32, 32, 32)
    rA, rB = synth.droplet_fields(shape, 8, (16, 16, 16), 1.0, 0.03)
    stream = torch.cuda.current_stream()
    p = lbm.lbm_default_params(32, 32, 32, stream=stream.cuda_stream, G=1.1, probe_center=(16.0, 16.0, 16.0),
                               probe_r_in=4.0, probe_r_out=12.0, storage=STORAGE_IDS[args.storage])
    b = lbm.lbm_batch_create([p])
    v = lbm.lbm_batch_run(b, 0)
    lbm.lbm_set_geometry(v, np.zeros(shape, np.uint8), np.ones(shape, np.float32))
    lbm.lbm_init_fields(v, rA.astype(np.float32), rB.astype(np.float32))
    steps = args.steps + (args.steps & 1)
    lbm.lbm_batch_step(b, steps)  # capture + warm-up
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lbm.lbm_batch_step(b, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    o = lbm.lbm_observables(v, check=False)
    b.close()
    out = {"metric": METRIC, "value": round(32 ** 3 * steps / (ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "n_gpus": 1, "steps": steps, "warmup": steps, "ms_per_step": ms / steps, "us_per_step": 1e3 * ms / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (droplet)",
           "config": {"workload": "static droplet 32^3, R = 8, G = 1.1, tau = 1 (fits in L2: launch-bound)",
                      "storage": args.storage, "graph": True},
           "observables": {"mass": o["mass"], "dp": o["dp"], "max_u": o["max_u"], "step": o["step"]}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------- porosity gradient
def run_adjoint(args):
    """dL/dphi of the outlet-flux/saturation loss on the 96^3 multiscale-rock
    recipe (A driven by the body force), hand-written adjoint with checkpoints
    every --ckpt steps, against the forward alone."""
    import torch
    from paper_2512_21696_gb300 import lbm
    torch.cuda.set_device(0)
    inp = workload_inputs(96)
    cell = inp["cell"]
    nz, ny, nx = cell.shape
    stream = torch.cuda.current_stream()
    p = lbm.lbm_default_params(nx, ny, nz, stream=stream.cuda_stream, **SETTINGS)
    ctx = lbm.lbm_create(p)
    lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive())
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in inp.items()}
    lbm.lbm_set_geometry(ctx, dev["cell"], dev["phi"], dev["ptype"])
    lbm.lbm_init_fields(ctx, dev["rhoA"], dev["rhoB"])
    lbm.lbm_step(ctx, args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lbm.lbm_init_fields(ctx, dev["rhoA"], dev["rhoB"])
    ev0.record(stream)
    lbm.lbm_step(ctx, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = ev0.elapsed_time(ev1)
    obs = lbm.lbm_observables(ctx, check=False)
    q_t, s_t = 0.5 * obs["flux_out"] if obs["flux_out"] != 0 else 1e-6, obs["sat"] - 0.02
    lbm.lbm_init_fields(ctx, dev["rhoA"], dev["rhoB"])
    grad = torch.empty(cell.shape, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, q, S, _ = lbm.lbm_adjoint_run(ctx, q_t, s_t, args.steps, args.ckpt, grad)
    torch.cuda.synchronize()
    ms_adj = (time.perf_counter() - t0) * 1e3
    g = grad.cpu().numpy()
    ctx.close()
    n = cell.size
    out = {"metric": METRIC, "value": round(n * args.steps / (ms_adj * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_adj / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded multiscale-rock recipe)",
           "config": {"workload": f"porosity gradient (forward + checkpointed adjoint), 96^3 multiscale rock, "
                                  f"{args.steps} steps, checkpoint every {args.ckpt}",
                      "cells": n, "gray_cells": int((cell == 2).sum())},
           "forward_ms": round(ms_fwd, 3), "forward_plus_adjoint_ms": round(ms_adj, 3),
           "adjoint_over_forward": round(ms_adj / ms_fwd, 2),
           "loss": {"L": L, "q": q, "S": S, "q_target": q_t, "s_target": s_t},
           "grad": {"max_abs": float(np.abs(g).max()), "nonzero": int(np.count_nonzero(g))}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", type=int, default=0, help="0 fused single launch, 1 two launches")
    ap.add_argument("--storage", choices=list(STORAGE_IDS), default="f32",
                    help="population storage: f32; f16 / bf16 globally shifted; f16r / bf16r rest-referenced (FP32 arithmetic)")
    ap.add_argument("--workload", choices=("drainage", "fiber", "droplet", "rev", "revlib", "adjoint", "imbibition",
                                           "droplet2d", "imbibition2d", "zigzag2d"),
                    default="drainage",
                    help="drainage: the 128^3 multiscale-rock step; fiber: the 192^3 tensorial fibre bundle; "
                         "droplet: the 32^3 static droplet (CUDA-graph replay); rev: the batched REV library; "
                         "revlib: K, Kr and Pc at 8 saturations for a REV subset; "
                         "adjoint: the porosity gradient on the 96^3 recipe; "
                         "imbibition: the stepped-pressure Pc-Sw protocol between reservoir planes; "
                         "droplet2d: the Sec. III.A droplet on D2Q9; "
                         "imbibition2d: the Sec. III.B random-porosity imbibition on D2Q9; "
                         "zigzag2d: the zigzag pathway between fibre bundles of Sec. I.B / III.E on D2Q9")
    ap.add_argument("--level-max", type=int, default=10000, help="imbibition: most steps per pressure level")
    ap.add_argument("--ckpt", type=int, default=100, help="adjoint checkpoint interval")
    ap.add_argument("--rev-runs", type=int, default=256)
    ap.add_argument("--steady-max", type=int, default=0,
                    help="rev: after timing, step every run to steady flow (at most this many steps); revlib: drive "
                         "every two-phase run to its target Sw with the mass-sink-source controller, then to steady "
                         "flow, before the timed steps (at most this many steps each)")
    ap.add_argument("--tile", type=int, default=8,
                    help="fused tile: 0 = 32x8, 1 = 32x16, 2 = 32x8 two CTAs/SM, 3 = 32x12, 4 = 64x8, "
                         "5 / 6 = published-density march 32x8 / 32x7, 7 = 64x7, "
                         "8 = chosen per grid among 2, 4, 7 (default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "rev":
        run_rev(args, rank, world, local_rank)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "droplet":
        run_droplet(args)
    elif args.workload == "revlib":
        run_revlib(args)
    elif args.workload == "imbibition":
        run_imbibition(args)
    elif args.workload == "droplet2d":
        run_droplet2d(args)
    elif args.workload == "imbibition2d":
        run_imbibition2d(args)
    elif args.workload == "zigzag2d":
        run_zigzag2d(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
