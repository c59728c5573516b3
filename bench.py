#!/usr/bin/env python
"""SRD (MPCD) step throughput on GB300: particle-steps/s and HBM roofline.

Default workload: the 250 x 250 x 250-cell SRD solvent at 5 particles per
cell (7.8 * 10^7 particles) in mixed precision (FP32 particles, int64
fixed-point cell sums, FP64 thermostat factor) with the cell-level
Maxwell-Boltzmann thermostat at kT = 1 and 2000 chains of 50 beads (mass 5,
harmonic bonds k = 1000, r0 = 0.5, 10 velocity-Verlet substeps per
collision), alpha = 130 deg, dt = 0.1, grid shift every step, 500 steps.
Synthetic, seeded inputs (uniform positions, zero-momentum Maxwell-Boltzmann
velocities, random-walk chains).

One JSON line on rank 0:
  value     particle-steps/s of the whole job, state resident in HBM, timed with
            CUDA events on the stream the kernels run on
  e2e       same metric through the C ABI with host arrays (set_state, K steps,
            get_state), wall clock
  roofline  dominant kernel: algorithmic bytes / its event-timed duration
  cpu_baseline  the CPU oracle, single thread, on a bounded sample
  extra     (N = 1, default workload) the 10^7-particle SRD box, the 64-box
            ensemble batched against per-box launches (a short run), and a
            short served sweep below saturation with p50/p99 job latency
--impl reference times the CPU oracle (the reference of this build) instead.
Multi-GPU (torchrun): independent replica boxes per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1801_10187_gb300 import inputs  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 1.25          # GB300 nominal FP64 (non-tensor) rate
# FP64 flops per particle-step of the collide + stream/bin pass (FMA = 2, no
# compares): cell sum 3, v - u 3, rotation about the cell axis 30, u + R d 3,
# r + v dt 6, r - s 3.  The per-cell work (u, the axis) is not counted.
FP64_FLOPS_PER_PARTICLE = 48
METRIC = "MPCD particle-steps/s"
# the 50M+ particle mixed-precision box: 7.8e7 particles, thermostat, solute
DEFAULT_WORKLOAD = "srd-250c-rho5-mixed-solute"
UNIT = "particle-steps/s"
# kernels launched per step: the fused cell kernel and the record update; the
# solute adds MD + bead grouping, 3 bead-scan phases and the bead scatter
LAUNCHES_PER_STEP = 2
LAUNCHES_PER_STEP_SOLUTE = 7


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def workload_cfg(name):
    if name not in inputs.WORKLOADS:
        raise SystemExit(f"unknown workload {name}; choose from {sorted(inputs.WORKLOADS)}")
    return dict(inputs.WORKLOADS[name])


def box_kwargs(cfg):
    kw = dict(n=cfg["n"], dt=cfg["dt"], alpha_deg=cfg["alpha_deg"], kT=cfg["kT"],
              seed=cfg["seed"], thermostat=cfg["thermostat"], precision=cfg["precision"],
              sort_period=cfg.get("sort_period", 0), collision=cfg.get("collision", "srd"),
              angular=cfg.get("angular", False))
    if cfg.get("n_chains"):
        kw.update(chain_len=cfg["chain_len"], md_substeps=cfg["md_substeps"],
                  solute_mass=cfg["bead_mass"], bond_k=cfg["bond_k"], bond_r0=cfg["bond_r0"],
                  lj_epsilon=cfg.get("lj_epsilon", 0.0), lj_sigma=cfg.get("lj_sigma", 0.0))
    return kw


def make_chains(cfg, n, n_chains, seed):
    if cfg.get("lj_epsilon"):  # beads that repel start apart
        return inputs.avoiding_chains(n, n_chains, cfg["chain_len"], cfg["bond_r0"],
                                      0.9 * cfg["lj_sigma"], kT=cfg["kT"],
                                      bead_mass=cfg["bead_mass"], seed=seed)
    return inputs.chains(n, n_chains, cfg["chain_len"], cfg["bond_r0"], kT=cfg["kT"],
                         bead_mass=cfg["bead_mass"], seed=seed)


def make_state(cfg, n=None, seed_offset=0, with_chains=True):
    n = n or cfg["n"]
    s = inputs.solvent(n, cfg["density"], kT=cfg["kT"], seed=cfg["seed"] + seed_offset,
                       mixed=cfg["precision"] == "mixed")
    sp = sv = None
    if cfg.get("n_chains") and with_chains:
        sp, sv = make_chains(cfg, n, cfg["n_chains"], cfg["seed"] + 1000 + seed_offset)
    return s, sp, sv


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing
def oracle_rate(cfg, budget_s, steps=None, warmup=0):
    """Time the CPU oracle (as it stands, one thread) on the workload.  The box
    is the full workload box when it fits the budget, else a cube of the same
    density, parameters and precision scaled down so that (warmup + steps)
    oracle steps take about budget_s."""
    import oracle
    oracle.build()
    full_cells = int(np.prod(cfg["n"]))
    ns_per_ps = 170.0  # rough oracle cost per particle-step, for sizing only
    nsteps = steps if steps else 3
    want_ps = budget_s * 1e9 / ns_per_ps / max(1, nsteps + warmup)
    cells = min(full_cells, max(27, int(want_ps / cfg["density"])))
    if cfg.get("lj_epsilon"):
        # the oracle's pair repulsion visits every pair of beads in every MD
        # substep: keep the sample's beads (at the workload's bead density)
        # within the budget, about 10 ns per pair visit
        nb_max = math.sqrt(budget_s / max(1, nsteps + warmup) / cfg["md_substeps"] / 1e-8)
        nb_full = cfg["n_chains"] * cfg["chain_len"]
        cells = min(cells, max(27, int(full_cells * nb_max / nb_full)))
    if cells < full_cells:
        edge = max(3, int(round(cells ** (1 / 3))))
        n = (edge, edge, edge)
    else:
        n = tuple(cfg["n"])
    s, sp, sv = make_state(cfg, n=n, with_chains=False)
    prec = oracle.MIXED if cfg["precision"] == "mixed" else oracle.FP64
    okw = dict(n=n, dt=cfg["dt"], alpha_deg=cfg["alpha_deg"], kT=cfg["kT"], seed=cfg["seed"],
               thermostat=cfg["thermostat"], precision=prec,
               collision=oracle.AT if cfg.get("collision") == "at" else oracle.SRD,
               angular=bool(cfg.get("angular", False)))
    if cfg.get("n_chains"):
        nch = max(1, int(round(cfg["n_chains"] * np.prod(n) / full_cells)))
        sp, sv = make_chains(cfg, n, nch, cfg["seed"] + 1000)
        okw.update(chain_len=cfg["chain_len"], md_substeps=cfg["md_substeps"],
                   solute_mass=cfg["bead_mass"], bond_k=cfg["bond_k"], bond_r0=cfg["bond_r0"],
                   lj_epsilon=cfg.get("lj_epsilon", 0.0), lj_sigma=cfg.get("lj_sigma", 0.0))
    p = oracle.Params(**okw)
    st = oracle.State(s.pos, s.vel, sp if sp is not None else np.zeros((0, 3)),
                      sv if sv is not None else np.zeros((0, 3)))
    if warmup:
        oracle.step(p, st, warmup)
    t0 = time.perf_counter()
    oracle.step(p, st, nsteps)
    dt = time.perf_counter() - t0
    npart = st.pos.shape[0] + st.spos.shape[0]
    rate = npart * nsteps / dt
    sample = (f"{nsteps} steps of a {n[0]}x{n[1]}x{n[2]}-cell box ({npart} particles), same "
              f"density/parameters/precision as the workload")
    return rate, sample, dt, nsteps


# ------------------------------------------------------------------ traffic record
def kernel_traffic(kernel, workload):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary
    record, if it was taken on the current sources of that kernel (their
    combined hash matches), else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    ent = rec.get(f"{kernel}/{workload}")
    if not ent:
        return None
    if sources_hash(ent["sources"]) != ent.get("sources_sha256_16"):
        return None
    return ent["dram_bytes_per_launch"] * ent.get("scale_to_workload", 1.0)


def _code_only(text):
    """Source text without comments and blank lines: what the compiled kernel
    depends on (an edit of a comment does not change the counters)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def sources_hash(paths):
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process
    group): each rank's elapsed time is reduced to the job's wall time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed units_per_rank (replicas, weak
    scaling) within the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra figures (10^7 box, batched ratio, served sweep)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--jobs", type=int, default=None, help="served workload: number of jobs")
    ap.add_argument("--no-sweep", action="store_true", help="served workload: skip the rate sweep")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the launch tuner: the engine's default launch (blocks per SM at "
                         "the occupancy limit, pass-2 chunks of 3, 32 cells per warp); for "
                         "profiling a fixed configuration")
    args = ap.parse_args()
    cfg = workload_cfg(args.workload)
    kind = cfg.get("kind", "box")
    K = args.steps if args.steps is not None else cfg.get("steps", 0)
    W = max(3, args.warmup)
    if kind != "box":
        return run_fleet(args, cfg, kind, K, W)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    config = {"workload": args.workload, "cells": list(cfg["n"]), "density": cfg["density"],
              "precision": cfg["precision"], "thermostat": cfg["thermostat"],
              "alpha_deg": cfg["alpha_deg"], "dt": cfg["dt"], "kT": cfg["kT"],
              "particles_per_gpu": int(round(cfg["density"] * np.prod(cfg["n"]))),
              "parallelism": f"replicas{world}" if world > 1 else "single"}
    if cfg.get("n_chains"):
        config["solute"] = {"chains": cfg["n_chains"], "beads_per_chain": cfg["chain_len"]}

    if args.impl == "reference":
        if rank != 0:
            return
        budget = 150.0
        rate, sample, dt, nsteps = oracle_rate(cfg, budget, steps=K, warmup=W)
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
                "n_gpus": args.gpus, "steps": K, "warmup": W,
                "ms_per_step": 1e3 * dt / nsteps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if cfg["precision"] == "fp64"
                else "f32+i64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    import paper_1801_10187_gb300 as pkg

    s, sp, sv = make_state(cfg, seed_offset=rank)
    N = s.pos.shape[0] + (sp.shape[0] if sp is not None else 0)
    # a dedicated (non-default) stream: the library orders all its work on it
    # and the CUDA events below are recorded on the same stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    box = pkg.Box(stream=stream.cuda_stream, **box_kwargs(cfg))
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(W)
    # launch tuner on real warm-up steps (grid of the fused pass), then the
    # re-captured step graph warms up again
    if args.no_tune:
        config["launch"] = {"blocks_per_sm": "occupancy limit", "pass2_chunk": 3,
                            "cells_per_warp": 32, "tuner": "off"}
    else:
        tuned_bps, tuned_ms, _, tuned_chunk, tuned_cpw = box.tune(2)
        config["launch"] = {"blocks_per_sm": tuned_bps if tuned_bps > 0 else "one per span part",
                            "pass2_chunk": tuned_chunk, "cells_per_warp": tuned_cpw,
                            "tuner_ms_per_step": tuned_ms}
    box.step(2)
    torch.cuda.synchronize()

    # ---- device-resident throughput ----
    sampler = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    value = job_rate(N * K, world, ms * 1e-3)

    # ---- per-phase times (event-timed eager steps, same stream) ----
    phases = box.phase_times(min(K, 50))
    hbm_peak, peak_src = load_peaks()
    es = 4 if cfg["precision"] == "mixed" else 8
    # the fused kernel performs the whole step: its algorithmic bytes are the
    # step's, 2 s_r + 3 s_v per particle (read r, write r, read v twice, write v)
    step_bytes = 2 * 3 * es + 3 * 3 * es
    dom = "fused_step"
    dom_ms = phases[dom]
    achieved = step_bytes * s.pos.shape[0] / (dom_ms * 1e-3) / 1e9
    # the warp-spread kernel runs mixed-model boxes without walls
    if cfg.get("angular") and not (cfg["precision"] == "mixed"
                                   and cfg.get("collision", "srd") == "srd"):
        kname = "k_cells"  # one thread per cell
    else:
        kname = "k_cells_warp" if cfg["precision"] == "mixed" else "k_cells_warp_d"
    traffic = kernel_traffic(kname, args.workload)
    roofline = {"bound": "hbm", "kernel": f"{kname} (collide t + stream/bin t+1)",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "frac_of_8tbs": achieved / 8000.0,
                "traffic": traffic, "peak_source": peak_src,
                "alg_bytes_per_particle": step_bytes,
                "kernel_ms": dom_ms, "particles": int(s.pos.shape[0])}
    if cfg["precision"] == "fp64":
        # The FP64 model is bound by the FP64 pipe, not by HBM: on GB300 FP64
        # runs at 1/64 of the FP32 rate.  Algorithmic FP64 flops per particle
        # and step: collide 36 (difference, Rodrigues rotation, sum), cell sums
        # 6, stream 12, wrap 6, binning 6 (an FMA counts two).
        flops = FP64_FLOPS_PER_PARTICLE * s.pos.shape[0] / (dom_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": f"{kname} (collide t + stream/bin t+1)",
                    "achieved": flops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": flops / FP64_PEAK_TFLOPS, "traffic": traffic,
                    "peak_source": "nominal: GB300 FP64 (non-tensor) rate from the "
                                   "data sheet, not measured",
                    "alg_flops_per_particle": FP64_FLOPS_PER_PARTICLE,
                    "hbm_frac": achieved / hbm_peak}
    step_gbs = step_bytes * N * K / (ms * 1e-3) / 1e9 / world
    hbm_step = {"bytes_per_particle_step": step_bytes, "achieved_gbs": step_gbs,
                "frac_of_peak": step_gbs / hbm_peak, "frac_of_8tbs": step_gbs / 8000.0,
                "phase_ms": phases}

    # ---- end to end through the C ABI with host arrays ----
    e2e = None
    if not args.no_e2e:
        Ke = K
        box2 = pkg.Box(stream=stream.cuda_stream, **box_kwargs(cfg))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        box2.set_state(s.pos, s.vel, sp, sv)
        box2.step(Ke)
        out = box2.get_state()
        t1 = time.perf_counter()
        wall = t1 - t0
        if dist:
            t = torch.tensor([wall], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            wall = float(t.item())
        assert out[4] == Ke
        h2d = s.pos.shape[0] * 2 * 3 * es + (0 if sp is None else sp.shape[0] * 48)
        e2e = {"value": N * Ke * world / wall, "unit": UNIT,
               "h2d_bytes_per_step": h2d / Ke, "d2h_bytes_per_step": h2d / Ke,
               "steps_per_job": Ke, "wall_s": wall}
        box2.close()

    # ---- CPU baseline (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sample, dt, nsteps = oracle_rate(cfg, 20.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    per_step = LAUNCHES_PER_STEP_SOLUTE if cfg.get("n_chains") else LAUNCHES_PER_STEP
    if cfg.get("lj_epsilon"):  # neighbour-list build (3), first force, 3 per MD substep
        per_step += 4 + 3 * cfg["md_substeps"]
    launches = per_step * K
    config["l2"] = (f"state {s.pos.shape[0] * 6 * es / 1e6:.0f} MB > 129 MB L2 (inputs larger "
                    "than L2; no flush)")
    config["device_bytes"] = box.footprint_bytes()
    config["bytes_per_particle"] = box.footprint_bytes() / N
    box.close()

    # ---- extra figures (N = 1, default workload) ----
    extra = None
    if world == 1 and not args.no_extra and args.workload == DEFAULT_WORKLOAD:
        extra = run_extra(pkg, torch, stream, hbm_peak)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64" if cfg["precision"] == "fp64" else "f32+i64",
                "data": "synthetic", "config": config, "clocks": clocks, "e2e": e2e,
                "gpu_launches": launches, "roofline": roofline, "hbm_step": hbm_step,
                "cpu_baseline": cpu, "extra": extra}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ extra figures
def run_extra(pkg, torch, stream, hbm_peak):
    """Short runs of the other measured forms, for the default line: the
    10^7-particle SRD box (device-resident rate and the fused kernel's
    roofline), the 64-box ensemble batched against per-box plain launches,
    and the served workload at two arrival rates below saturation."""
    out = {}
    # 10^7-particle SRD box, mixed, no thermostat
    name = "srd-100c-rho10-mixed"
    cfg = workload_cfg(name)
    s, _, _ = make_state(cfg)
    box = pkg.Box(stream=stream.cuda_stream, **box_kwargs(cfg))
    box.set_state(s.pos, s.vel)
    box.step(10)
    box.tune(2)
    box.step(2)
    torch.cuda.synchronize()
    K = 500
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    phases = box.phase_times(50)
    n = s.pos.shape[0]
    gbs = 60 * n / (phases["fused_step"] * 1e-3) / 1e9
    out[name] = {"particles": n, "steps": K, "ms_per_step": ms / K,
                 "value": n * K / (ms * 1e-3), "unit": UNIT,
                 "fused_kernel_ms": phases["fused_step"], "achieved_gbs": gbs,
                 "frac": gbs / hbm_peak, "frac_of_8tbs": gbs / 8000.0,
                 "bytes_per_particle": box.footprint_bytes() / n}
    box.close()
    del s
    # 64-box ensemble: one batch against per-box plain launches
    bcfg = workload_cfg("srd-batch64-mixed")
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    args = argparse.Namespace(workload="srd-batch64-mixed")
    b = _run_batch(pkg, torch, stream, sampler, args, bcfg, 50, 5, 0, 1, None)
    out["srd-batch64-mixed"] = {
        "boxes": b["config"]["boxes"], "particles": b["config"]["particles"], "steps": 50,
        "batched": b["value"], "per_box_plain_launches": b["per_box_plain_launches"]["value"],
        "ratio_batched_over_per_box": b["per_box_plain_launches"]["ratio_batched_over_per_box"],
        "unit": UNIT}
    # served workload below saturation: two arrival rates, 60 jobs each
    from paper_1801_10187_gb300 import serve
    scfg = workload_cfg("srd-served-poisson")
    free, _total = torch.cuda.mem_get_info()
    sweep = []
    for rate in (5.0, 10.0):
        jobs = serve.poisson_jobs(60, rate, seed=scfg["jobs_seed"] + 200, l_min=scfg["l_min"],
                                  l_max=scfg["l_max"], density=scfg["density"],
                                  steps_min=scfg["steps_min"], steps_max=scfg["steps_max"],
                                  alpha_deg=scfg["alpha_deg"])
        srv = serve.Server(precision=scfg["precision"], max_bytes=int(free * 0.8),
                           stream=stream.cuda_stream)
        st = srv.run(jobs, realtime=True)
        srv.close()
        d = st.as_dict()
        d["rate_jobs_per_s"] = rate
        sweep.append(d)
    # the same 60 jobs all due at once (closed loop): the server saturated,
    # its capacity beside the batched ensemble's
    jobs = serve.poisson_jobs(60, 10.0, seed=scfg["jobs_seed"] + 200, l_min=scfg["l_min"],
                              l_max=scfg["l_max"], density=scfg["density"],
                              steps_min=scfg["steps_min"], steps_max=scfg["steps_max"],
                              alpha_deg=scfg["alpha_deg"])
    srv = serve.Server(precision=scfg["precision"], max_bytes=int(free * 0.8),
                       stream=stream.cuda_stream)
    st = srv.run(jobs, realtime=False)
    srv.close()
    saturated = st.as_dict()
    out["srd-served-poisson"] = {"recipe": "serve.poisson_jobs, 60 jobs per rate: L "
                                           "log-uniform [10,160], density 5, steps "
                                           "U[100,5000], 130 deg, thermostat every other job",
                                 "sweep": sweep, "saturated_closed_loop": saturated}
    return out


# ------------------------------------------------------------------ batched / served
def _fleet_reference(args, cfg, kind, K, W):
    """Oracle timing for the batch and served workloads: one of their boxes
    (a 16^3-cell box at density 5, the smallest ensemble member) as the
    bounded sample."""
    sub = dict(n=(16, 16, 16), density=5, dt=cfg["dt"] if "dt" in cfg else 0.1, kT=1.0,
               alpha_deg=130.0, seed=1000, thermostat=False, precision=cfg["precision"])
    rate, sample, dt, nsteps = oracle_rate(sub, 150.0, steps=max(1, min(K or 5, 20)), warmup=0)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
            "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / nsteps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i64", "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_fleet(args, cfg, kind, K, W):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            _fleet_reference(args, cfg, kind, K, W)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    import paper_1801_10187_gb300 as pkg
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sampler = ClockSampler(local_rank)
    if kind == "batch":
        line = _run_batch(pkg, torch, stream, sampler, args, cfg, K, W, rank, world, dist)
    else:
        line = _run_serve(pkg, torch, stream, sampler, args, cfg, rank, world, dist)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _run_batch(pkg, torch, stream, sampler, args, cfg, K, W, rank, world, dist):
    """All boxes of the ensemble in one batch (one fused launch per step for
    every box), against the same boxes stepped one after another as plain
    single-box contexts.  Thermal initial states are drawn on the device."""
    specs = inputs.ensemble(cfg["n_boxes"], seed=cfg["ensemble_seed"])
    common = dict(dt=cfg["dt"], kT=cfg["kT"], thermostat=cfg["thermostat"],
                  precision=cfg["precision"])
    counts = [int(round(s["density"] * np.prod(s["n"]))) for s in specs]
    N = sum(counts)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # ---- batched ----
    batch = pkg.Batch(cfg["precision"], stream=stream.cuda_stream)
    t0 = time.perf_counter()
    for s, n in zip(specs, counts):
        batch.add_thermal(n, init_seed=s["seed"] + rank * 100000, n=s["n"],
                          alpha_deg=s["alpha_deg"], seed=s["seed"] + rank * 100000, **common)
    batch.step(W)
    batch.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0, e1 = ev(), ev()
    e0.record(stream)
    batch.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    obs = [batch.observables(i) for i in range(len(specs))]
    wall = time.perf_counter() - t0
    if dist:
        t = torch.tensor([ms, wall], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, wall = float(t[0].item()), float(t[1].item())
    batched = N * K * world / (ms * 1e-3)
    assert all(o["step"] == W + K for o in obs)
    batch.close()

    # ---- per-box plain launches, one box after another ----
    per_ms = 0.0
    for s, n in zip(specs, counts):
        box = pkg.Box(stream=stream.cuda_stream, n=s["n"], alpha_deg=s["alpha_deg"],
                      seed=s["seed"] + rank * 100000, **common)
        box.set_state_thermal(n, init_seed=s["seed"] + rank * 100000)
        box.step(W)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        box.step(K)
        b.record(stream)
        torch.cuda.synchronize()
        per_ms += a.elapsed_time(b)
        box.close()
    if dist:
        t = torch.tensor([per_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        per_ms = float(t.item())
    per_box = N * K * world / (per_ms * 1e-3)
    es = 4 if cfg["precision"] == "mixed" else 8
    step_bytes = 2 * 3 * es + 3 * 3 * es
    peak, src = load_peaks()
    gbs = step_bytes * N * K / (ms * 1e-3) / 1e9
    return {"metric": METRIC, "value": batched, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i64" if cfg["precision"] == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "boxes": len(specs), "particles": N,
                       "recipe": "inputs.ensemble(64, seed=4): L in U{16..96}, density 5|10, "
                                 "angle 90|120|130 deg, seeds 1000+i, thermal states on device",
                       "l2": f"state {N * 6 * es / 1e9:.1f} GB > 129 MB L2 (no flush)"},
            "clocks": clocks,
            "per_box_plain_launches": {"value": per_box, "unit": UNIT, "ms_total": per_ms,
                                       "ratio_batched_over_per_box": batched / per_box},
            "e2e": {"value": N * K * world / wall, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": len(specs) * 96 / K,
                    "note": "add_thermal (states drawn on device) + warm-up + K steps + "
                            "observables of every box, wall clock"},
            "gpu_launches": 2 * K,
            "roofline": {"bound": "hbm", "kernel": "k_cells_warp (all boxes in one launch)",
                         "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": None, "peak_source": src,
                         "alg_bytes_per_particle": step_bytes},
            "cpu_baseline": None}


def _run_serve(pkg, torch, stream, sampler, args, cfg, rank, world, dist):
    """The served workload: Poisson job arrivals, admission by device-memory
    footprint, every resident job advanced in one batch; p50/p99 latency and
    aggregate throughput, then a sweep of arrival rates below saturation."""
    from paper_1801_10187_gb300 import serve
    n_jobs = args.jobs if args.jobs is not None else cfg["n_jobs"]
    free, _total = torch.cuda.mem_get_info()
    budget = int(free * 0.8)

    def one(rate, nj, seed):
        jobs = serve.poisson_jobs(nj, rate, seed=seed, l_min=cfg["l_min"], l_max=cfg["l_max"],
                                  density=cfg["density"], steps_min=cfg["steps_min"],
                                  steps_max=cfg["steps_max"], alpha_deg=cfg["alpha_deg"])
        srv = serve.Server(precision=cfg["precision"], max_bytes=budget,
                           stream=stream.cuda_stream)
        st = srv.run(jobs, realtime=True)
        srv.close()
        d = st.as_dict()
        d["rate_jobs_per_s"] = rate
        return d

    if dist:
        dist.barrier()
    sampler.start()
    main_run = one(cfg["rate"], n_jobs, cfg["jobs_seed"] + rank)
    clocks = sampler.stop()
    sweep = []
    if not args.no_sweep:
        for r in cfg["sweep_rates"]:
            sweep.append(one(r, cfg["sweep_jobs"], cfg["jobs_seed"] + 100 + rank))
    value = main_run["particle_steps_per_s"]
    if dist:
        t = torch.tensor([main_run["makespan_s"]], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        value = main_run["particle_steps"] * world / float(t.item())
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
            "config": {"workload": args.workload, "jobs": n_jobs, "rate_jobs_per_s": cfg["rate"],
                       "recipe": "serve.poisson_jobs: L log-uniform [10,160], density 5, steps "
                                 "U[100,5000], 130 deg, thermostat on every other job",
                       "admission_bytes": budget},
            "clocks": clocks, "served": main_run, "sweep": sweep,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "note": "wall clock of the whole served run through the public API"},
            "gpu_launches": None, "roofline": None, "cpu_baseline": None}


if __name__ == "__main__":
    main()
