#!/usr/bin/env python
"""Throughput of the split 6D Vlasov step (Eq. 5, SL-MPP5 sweeps + rho_nu moment).

Workload (default): 64^3 spatial x 32^3 velocity cells, FP32 f (8.59e9 cells,
34.4 GB), |u| <= 5 u_T, f0 = (1 + delta) F_FD with delta rms 0.05 (P ~ k^-2), a fixed
CDM background of contrast rms 1.0 and neutrino fraction 0.03, 4 pi G = 1,
self-consistent steps (moment -> Poisson -> second kick), a from 0.5 to 0.6 over
10 steps, each step's dt set by a seeded Courant number in [0.5, 0.9].

One "step" = one vlasov_step: 9 directional sweeps of all cells, the moment, the
Poisson solve and the velocity-sweep constants.  metric = cell updates per second
per sweep = 9 x cells x steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload on its own GPU (the
path has no exchange on one GPU: "replicas only"); value sums the ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "6D cell-updates/s per sweep"
UNIT = "cell-updates/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # HBM3e specification, for context beside the measured copy peak
# algorithmic bytes of one FP32 cell update: one 4-byte read and one 4-byte write of f
BYTES_PER_UPDATE = 8.0
# cell updates per cell that one launch of each sweep kind makes (the fused kick tail
# runs D_uy and D_uz in one pass over f)
UPDATES_PER_PASS = {"sweep_uyuz": 2, "kick": 3}

WORKLOAD = dict(name="fp32_64x32", n=64, nu=32, V=5.0, L=1.0, delta_rms=0.05, cdm_rms=1.0,
                f_nu=0.03, four_pi_G=1.0, a0=0.5, a1=0.6, cfl=(0.5, 0.9), seed=2)
# Reduced-precision storage: BF16 / FP16 f with one FP32 scale per u_z line on
# 96^3 x 32^3 cells, the 16^3-parity setup (delta rms 0.01, external phi, CFL 0.7, a = 1).
LOWPREC = dict(name="lowprec_96x32", n=96, nu=32, V=5.0, delta_rms=0.01, seed=1, cfl=0.7)
# CPU baseline / reference arm: the oracle on a bounded sample of the same workload:
# the same 32^3 velocity cube on an 8^3 spatial grid (1.68e7 cells per step).
SAMPLE = dict(n=8, nu=32)
# Reverse mode: 32^3 x 16^3 FP32 cells, 16 external-potential steps, checkpoint every 4.
ADJOINT = dict(name="adjoint_32x16", n=32, nu=16, V=5.0, delta_rms=0.01, seed=1, cfl=0.7, steps=16, K=4)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-lowprec", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-large", action="store_true")
    p.add_argument("--fused-kick", type=int, default=None,
                   help="2: each kick in one pass over the velocity cubes, 1: D_ux then D_uy D_uz in one pass, "
                        "0: three sweeps (default: the library's, 2)")
    p.add_argument("--fused-moment", type=int, default=None,
                   help="1 / 0: let the x sweep sum the moment or run the moment kernel (default: the library's)")
    p.add_argument("--profile-case", action="store_true",
                   help="run the small profiling case instead of the benchmark: sweeps on a "
                        "(64, 8, 8) x 32^3 FP32 grid (537 MB, larger than L2), twice per axis")
    p.add_argument("--axes", default="0,1,2,3,4,5", help="sweep axes of --profile-case")
    p.add_argument("--profile-shape", default="64,8,8",
                   help="spatial cells nx,ny,nz of --profile-case")
    p.add_argument("--profile-nu", type=int, default=32, help="velocity cells per axis of --profile-case")
    p.add_argument("--streamed", action="store_true", help="--profile-case runs the streamed position sweeps")
    p.add_argument("--profile-dtype", default="f32", choices=["f32", "bf16", "f16"],
                   help="storage of --profile-case's sweeps (16-bit: codes with a scale per u_z line)")
    p.add_argument("--adjoint", action="store_true", help="--profile-case runs the adjoint sweeps")
    p.add_argument("--step", action="store_true", help="--profile-case runs one Eq. (5) step (fused kick tail)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, dist, device):
    """The largest of the ranks' times (every rank gets it); ms itself on one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, cells, steps, ms, sweeps=9):
    """Cell updates per second per sweep of the whole job: every rank advances its own
    replica of `cells` cells by `steps` steps of `sweeps` sweeps in the slowest rank's time."""
    return world * sweeps * cells * steps / (ms * 1e-3)


def schedule(k, nsteps, w=WORKLOAD):
    """a at the start / middle / end of step k of a run of nsteps steps that takes a
    linearly from a0 to a1 once, and step k's seeded Courant number."""
    rng = np.random.default_rng(1000 + k)
    cfl = rng.uniform(*w["cfl"])
    da = (w["a1"] - w["a0"]) / nsteps
    a_start = w["a0"] + da * k
    a_end = a_start + da
    return a_start, 0.5 * (a_start + a_end), a_end, cfl


def drift_dt(cfl, a_half, n, nu, V, L):
    """dt whose largest position-sweep Courant number u_max dt / (a^2 dx) is cfl."""
    du = 2.0 * V / nu
    umax = V - 0.5 * du
    return cfl * a_half * a_half * (L / n) / umax


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources each timed kernel kind is built from (its DRAM traffic record is void once
# one of them changes)
_COMMON_SOURCES = ("vk_common.cuh", "vk_kernels.h")
KERNEL_SOURCES = {
    # FP32 position sweeps of 16-64 cells: whole lines staged per tile
    "sweep_x": ("sweep_tile.cu",), "sweep_y": ("sweep_tile.cu",), "sweep_z": ("sweep_tile.cu",),
    "sweep_ux": ("sweep_lines.cu", "vk_lines.cuh"), "sweep_uy": ("sweep_lines.cu", "vk_lines.cuh"),
    "sweep_uz": ("sweep_lines.cu", "vk_lines.cuh"), "sweep_uyuz": ("sweep_lines.cu", "vk_lines.cuh"),
    "kick": ("kick_cube.cu", "vk_lines.cuh"),
}


def _code_only(text):
    """C++ source without comments and blank lines: edits to comments keep the hash."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash(kind):
    """Hash of the code of the sources `kind`'s kernel is built from (None for an unknown kind)."""
    if kind not in KERNEL_SOURCES:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_15867_gb300", "csrc")
    for fn in sorted(KERNEL_SOURCES[kind] + _COMMON_SOURCES):
        with open(os.path.join(csrc, fn), encoding="utf-8") as fh:
            h.update(fn.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def step_bandwidth(kind_n, sweep_kinds, cells, steps, ms_per_step, hbm_peak):
    """The step on the bandwidth basis: every launch of a sweep kind (the one-pass kick
    included) reads and writes f once, BYTES_PER_UPDATE per cell, whatever the updates it
    makes; those bytes per step over the step time, against the measured and nominal peaks."""
    passes = sum(kind_n.get(k, 0) for k in sweep_kinds) / steps
    b = passes * BYTES_PER_UPDATE * cells
    gbs = b / (ms_per_step * 1e-3) / 1e9
    return {"passes_per_step": passes, "bytes_per_step": b, "GBs": gbs, "frac_of_measured": gbs / hbm_peak,
            "frac_of_nominal_7900": gbs / NOMINAL_HBM_GBS,
            "what": "bytes the f-wide passes of a step read and write (8 B per cell and pass) over the step time"}


def committed_alu(kind):
    """ALU-pipe activity (% of peak, ncu sm__inst_executed_pipe_alu / sm__pipe_alu_cycles_active)
    of `kind` from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    ent = d.get("kernels", {}).get(kind)
    if not ent or ent.get("source_hash") != kernel_source_hash(kind):
        return None
    return ent.get("alu_pipe_pct")


def committed_traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    ent = d.get("kernels", {}).get(kind)
    if not ent or ent.get("source_hash") is None or ent.get("source_hash") != kernel_source_hash(kind):
        return None
    return ent.get("bytes_per_full_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        # samples under load: the upper half of the clock readings
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_setup():
    import oracle as O
    from paper_2110_15867_gb300 import inputs as I
    w = WORKLOAD
    n, nu = SAMPLE["n"], SAMPLE["nu"]
    g = O.grid(n, nu, L=w["L"], V=w["V"])
    Fu = I.fermi_dirac(nu, w["V"])
    f = I.initial_f(I.gaussian_field(n, w["delta_rms"], seed=w["seed"]), Fu, np.float32)
    f = f.astype(np.float64)
    rho0, _ = O.moment(g, f)
    rbar = rho0.mean()
    bg = rbar * (1.0 / w["f_nu"] - 1.0) * (1.0 + I.gaussian_field(n, w["cdm_rms"], seed=w["seed"] + 1))
    phi = O.poisson(g, rho0 + bg, w["a0"], w["four_pi_G"])
    return O, g, f, bg, phi


def oracle_steps(O, g, f, bg, phi, k0, nsteps, total):
    """Steps k0 .. k0 + nsteps - 1 of a run of `total` steps (a from a0 to a1)."""
    w = WORKLOAD
    n, nu = SAMPLE["n"], SAMPLE["nu"]
    for k in range(k0, k0 + nsteps):
        a_s, a_h, a_e, cfl = schedule(k, total)
        dt = drift_dt(cfl, a_h, n, nu, w["V"], w["L"])
        phi, _ = O.step(g, f, dt, a_h, a_e, phi, rho_bg=bg, four_pi_G=w["four_pi_G"],
                        self_consistent=True)
    return phi


def cpu_baseline(min_seconds=10.0):
    O, g, f, bg, phi = oracle_sample_setup()
    t0 = time.perf_counter()
    k = 0
    while True:
        phi = oracle_steps(O, g, f, bg, phi, k % 10, 1, 10)  # config 2's 10-step schedule, repeated
        k += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    t = time.perf_counter() - t0
    return {"value": 9.0 * f.size * k / t, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d steps of the FP64 oracle's Eq. (5) step on an %d^3 x %d^3 sample of the "
                      "workload (same velocity cube, dt scaled to the sample's dx), %.1f s"
                      % (k, SAMPLE["n"], SAMPLE["nu"], t)}


# Per-axis CPU rates: the oracle's single sweeps on the 16^3 x 16^3 parity grid, the
# 24^3 x 16^3 low-precision sub-run grid and a 32^3 x 32^3 grid (1.07e9 cells, 8.6 GB FP64)
CPU_AXIS_GRIDS = ((16, 16), (24, 16), (32, 32))


def cpu_per_axis():
    """Cell updates per second of one oracle sweep along each axis (CFL 0.7, external phi)."""
    import oracle as O
    from paper_2110_15867_gb300 import inputs as I
    out = {}
    names = ("x", "y", "z", "ux", "uy", "uz")
    for n, nu in CPU_AXIS_GRIDS:
        V = 5.0
        g = O.grid(n, nu, V=V)
        f = I.initial_f(I.gaussian_field(n, 0.01, seed=1), I.fermi_dirac(nu, V), np.float64)
        phi = I.fourier_potential(n, seed=11)
        c = courant_per_dt(phi, n, nu, V)
        rates = {}
        for ax in range(6):
            dt = 0.7 / c[ax]
            t0 = time.perf_counter()
            O.sweep(g, f, ax, dt, 1.0, phi)
            rates[names[ax]] = f.size / (time.perf_counter() - t0)
        out["%d^3 x %d^3" % (n, nu)] = rates
        del f
    return {"unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "what": "one FP64 oracle sweep per axis at Courant number 0.7 (external phi for the velocity "
                    "axes), cell updates per second", "grids": out}


def workload_config(world):
    """The `config` object of both arms' JSON line: the 64^3 x 32^3 workload."""
    w = WORKLOAD
    n, nu = w["n"], w["nu"]
    cells = n ** 3 * nu ** 3
    return {"workload": "%s: %d^3 x %d^3 cells FP32, self-consistent Eq. (5) steps "
                        "(9 SL-MPP5 sweeps + moment + Poisson)" % (w["name"], n, nu),
            "cells": cells, "bytes_f": int(cells * 4),
            "l2": "inputs larger than L2 (34.4 GB f vs 129 MB L2)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    O, g, f, bg, phi = oracle_sample_setup()
    phi = oracle_steps(O, g, f, bg, phi, 0, args.warmup, max(1, args.warmup))
    t0 = time.perf_counter()
    phi = oracle_steps(O, g, f, bg, phi, 0, args.steps, args.steps)
    t = time.perf_counter() - t0
    value = 9.0 * f.size * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "each step: the FP64 oracle's Eq. (5) step on an %d^3 x %d^3 sample of the "
                                       "workload (same velocity cube, dt scaled to the sample's dx)"
                                       % (SAMPLE["n"], SAMPLE["nu"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def build_inputs(torch, dev):
    """f0 on the device (formed in FP64 per x-slab, rounded once), rho_bg, phi0."""
    from paper_2110_15867_gb300 import inputs as I
    w = WORKLOAD
    n, nu, V = w["n"], w["nu"], w["V"]
    delta = torch.from_numpy(I.gaussian_field(n, w["delta_rms"], seed=w["seed"])).to(dev)
    Fu = torch.from_numpy(I.fermi_dirac(nu, V)).to(dev)
    f = torch.empty((n, n, n, nu, nu, nu), dtype=torch.float32, device=dev)
    for ix in range(n):
        f[ix] = ((1.0 + delta[ix])[:, :, None, None, None] * Fu[None, None]).to(torch.float32)
    du3 = (2.0 * V / nu) ** 3
    rho_bar = float(Fu.sum().item()) * du3  # mean of (1 + delta) is 1
    dc = torch.from_numpy(I.gaussian_field(n, w["cdm_rms"], seed=w["seed"] + 1)).to(dev)
    rho_bg = (rho_bar * (1.0 / w["f_nu"] - 1.0) * (1.0 + dc)).contiguous()
    return f, rho_bg


def courant_per_dt(phi, n, nu, V, L=1.0, a=1.0):
    """Largest |Courant number| per unit dt of each sweep axis x, y, z, u_x, u_y, u_z:
    |u| / (a^2 dx) for the position sweeps and |g_i| / du for the velocity sweeps, g the
    periodic 4th-order gradient of phi.  Host-side arithmetic that picks dt."""
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    du = 2.0 * V / nu
    out = [(V - 0.5 * du) * n[d] / (L * a * a) for d in range(3)]
    p = phi.astype(np.float64)
    for d in range(3):
        g = (8.0 * (np.roll(p, -1, d) - np.roll(p, 1, d)) - (np.roll(p, -2, d) - np.roll(p, 2, d))) / (12.0 * L / n[d])
        out.append(float(np.abs(g).max()) / du)
    return out


def run_lowprec(torch, B, dev, steps, warmup):
    """Per-sweep rate of Eq. (5) steps with BF16 and FP16 storage (FP32 arithmetic)."""
    from paper_2110_15867_gb300 import inputs as I
    w = LOWPREC
    n, nu, V = w["n"], w["nu"], w["V"]
    phi_np = I.fourier_potential(n, seed=w["seed"] + 10).astype(np.float32)
    # the largest Courant number of the 6 axes is cfl (a kick advances dt / 2)
    c = courant_per_dt(phi_np, n, nu, V)
    dt = w["cfl"] / max(max(c[:3]), 0.5 * max(c[3:]))
    delta = torch.from_numpy(I.gaussian_field(n, w["delta_rms"], seed=w["seed"])).to(dev)
    Fu = torch.from_numpy(I.fermi_dirac(nu, V)).to(dev)
    phi = torch.from_numpy(phi_np).to(dev)
    out = {"workload": "%s: %d^3 x %d^3 cells, external phi, 9 sweeps + moment per step" % (w["name"], n, nu),
           "cells": n ** 3 * nu ** 3}
    for name, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        codes = torch.empty((n, n, n, nu, nu, nu), dtype=tdt, device=dev)
        scale = torch.empty((n, n, n, nu, nu), dtype=torch.float32, device=dev)
        for ix in range(n):
            B.encode_lines((1.0 + delta[ix])[:, :, None, None, None] * Fu[None, None], tdt,
                           codes=codes[ix], scale=scale[ix])
        v = B.Vlasov(codes, V=V, scale=scale)
        rho = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        for _ in range(warmup):
            v.step(dt, 1.0, 1.0, phi, rho_nu=rho)
        v.status()
        v.read_timers()
        v.enable_timers(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            v.step(dt, 1.0, 1.0, phi, rho_nu=rho)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kind_ms, kind_n = v.read_timers()
        v.status()
        v.close()
        cells = codes.numel()
        alg = 2.0 * cells * 2 + 4.0 * 2 * scale.numel()  # 16-bit read + write, scales read + write
        out[name] = {"value": 9.0 * cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "kernels": {k: {"ms_per_launch": kind_ms[k] / kind_n[k], "launches": kind_n[k],
                                     "GBs_actual_bytes": alg / (kind_ms[k] / kind_n[k] * 1e-3) / 1e9,
                                     "cell_updates_per_s": UPDATES_PER_PASS.get(k, 1) * cells /
                                     (kind_ms[k] / kind_n[k] * 1e-3)}
                                 for k in kind_ms if kind_n[k] and (k.startswith("sweep_") or k == "kick")}}
        del codes, scale
        torch.cuda.empty_cache()
    return out


def run_large(torch, B, dev, steps, warmup):
    """The large self-consistent run (48^3 x 48^3 cells, |u| <= 8 u_T, delta rms 0.1, CDM
    contrast rms 3.0, a from 0.2 over a 50-step schedule to 1.0, moment and Poisson every
    step) in FP32 and in BF16 storage side by side: the first warmup + steps steps of the
    schedule, the last `steps` timed; per-sweep rate, per-kernel times, and the density of
    the last step in BF16 against FP32."""
    from paper_2110_15867_gb300 import inputs as I
    cfg = I.CONFIGS["large_48x48"]
    n, nu, V, L, f_nu = cfg["n"], cfg["nu"], cfg["V"], 1.0, 0.03
    delta = torch.from_numpy(I.gaussian_field(n, cfg["delta_rms"], seed=cfg["seed"])).to(dev)
    Fu = torch.from_numpy(I.fermi_dirac(nu, V)).to(dev)
    du = 2.0 * V / nu
    rho_bar = float(Fu.sum().item()) * du ** 3
    dc = torch.from_numpy(I.gaussian_field(n, cfg["cdm_rms"], seed=cfg["seed"] + 1)).to(dev)
    rho_bg = (rho_bar * (1.0 / f_nu - 1.0) * (1.0 + dc)).contiguous()
    da = (cfg["a1"] - cfg["a0"]) / cfg["steps"]
    umax = V - 0.5 * du
    cells = n ** 3 * nu ** 3
    out = {"workload": "large_48x48: %d^3 x %d^3 cells, |u| <= 8 u_T, self-consistent Eq. (5) steps "
                       "(moment + Poisson every step), steps %d..%d of the 50-step a = 0.2 -> 1.0 schedule"
                       % (n, nu, warmup, warmup + steps - 1), "cells": cells}
    dts = None
    rhos = {}
    for name in ("f32", "bf16"):
        if name == "f32":
            f = torch.empty((n, n, n, nu, nu, nu), dtype=torch.float32, device=dev)
            for ix in range(n):
                f[ix] = ((1.0 + delta[ix])[:, :, None, None, None] * Fu[None, None]).to(torch.float32)
            scale = None
        else:
            f = torch.empty((n, n, n, nu, nu, nu), dtype=torch.bfloat16, device=dev)
            scale = torch.empty((n, n, n, nu, nu), dtype=torch.float32, device=dev)
            for ix in range(n):
                B.encode_lines((1.0 + delta[ix])[:, :, None, None, None] * Fu[None, None], torch.bfloat16,
                               codes=f[ix], scale=scale[ix])
        v = B.Vlasov(f, L=L, V=V, scale=scale)
        rho = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        v.moment(rho)
        phi = v.poisson(rho, cfg["a0"], 1.0, rho_bg=rho_bg)
        phi2 = torch.empty_like(phi)
        if dts is None:
            # dt per step: the largest position Courant number at a_half is 0.9, capped so that a
            # kick's velocity Courant number under the initial potential stays <= 0.3 (room for
            # phi to grow); the same dt sequence for both storage types
            g0 = max(courant_per_dt(phi.cpu().numpy(), n, nu, V)[3:]) * du  # largest |grad phi|
            dt_vel = 0.3 * 2.0 * du / max(g0, 1e-30)
            dts = []
            for k in range(warmup + steps):
                a_h = cfg["a0"] + da * (k + 0.5)
                dts.append(min(cfg["cfl"] * a_h * a_h * (L / n) / umax, dt_vel))

        def one(k):
            nonlocal phi, phi2
            a_s = cfg["a0"] + da * k
            v.step(dts[k], a_s + 0.5 * da, a_s + da, phi, rho_bg=rho_bg, four_pi_G=1.0, phi_next=phi2, rho_nu=rho)
            phi, phi2 = phi2, phi

        for k in range(warmup):
            one(k)
        v.status()
        v.read_timers()
        v.enable_timers(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(warmup, warmup + steps):
            one(k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kind_ms, kind_n = v.read_timers()
        v.enable_timers(False)
        v.status()
        rhos[name] = rho.clone()
        out[name] = {"value": 9.0 * cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "kernels": {k: {"ms_per_launch": kind_ms[k] / kind_n[k], "launches": kind_n[k],
                                     "cell_updates_per_s": UPDATES_PER_PASS.get(k, 1) * cells /
                                     (kind_ms[k] / kind_n[k] * 1e-3)}
                                 for k in kind_ms if kind_n[k] and (k.startswith("sweep_") or k == "kick")}}
        v.close()
        del f, scale, v
        torch.cuda.empty_cache()
    out["bf16_vs_f32"] = out["bf16"]["value"] / out["f32"]["value"]
    d = (rhos["bf16"] - rhos["f32"]).abs()
    out["density_bf16_vs_f32"] = {"rel_l1": float(d.sum() / rhos["f32"].abs().sum()),
                                  "max_cell_rel": float((d / rhos["f32"].abs()).max())}
    return out


def run_adjoint(torch, dev, reps=3):
    """Reverse mode of a 16-step run (checkpoints every 4 steps) on 32^3 x 16^3 FP32
    cells: forward (16 steps + moment) and backward (segments re-recorded, 144 adjoint
    sweeps, moment adjoint) timed with CUDA events, median of reps."""
    from paper_2110_15867_gb300 import inputs as I
    from paper_2110_15867_gb300.autograd import Run, run_rho
    w = ADJOINT
    n, nu, V = w["n"], w["nu"], w["V"]
    f0 = I.initial_f(I.gaussian_field(n, w["delta_rms"], seed=w["seed"]), I.fermi_dirac(nu, V), np.float32)
    phi_np = I.fourier_potential(n, seed=w["seed"] + 10).astype(np.float32)
    c = courant_per_dt(phi_np, n, nu, V)
    dt = w["cfl"] / max(max(c[:3]), 0.5 * max(c[3:]))
    run = Run(f0.shape, torch.float32, V=V)
    ft = torch.from_numpy(f0).to(dev).requires_grad_()
    pt = torch.from_numpy(phi_np).to(dev).requires_grad_()
    kx = torch.fft.fftfreq(n, d=1.0 / n, device=dev)
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kx[None, None, :] ** 2
    mask = ((k2 > 0) & (k2 < 64)).to(torch.float64)  # modes 0 < |n| < 8

    def once():
        ft.grad = None
        pt.grad = None
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        rho = run_rho(ft, pt, run, dt, 1.0, w["steps"], w["K"])
        e[1].record()
        loss = (torch.fft.fftn(rho).abs() ** 2 * mask).sum()
        loss.backward()
        e[2].record()
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])

    nseg = (w["steps"] + w["K"] - 1) // w["K"]
    taped = run.taped_segments(nseg, w["K"])  # the default: as many segments as half the free memory holds
    once()
    ts = [once() for _ in range(reps)]
    fw = float(np.median([t[0] for t in ts]))
    bw = float(np.median([t[1] for t in ts]))
    # the same run with one taped segment (the backward runs the other segments again)
    run.tape_segments = 1
    run.release_tape()
    once()
    ts1 = [once() for _ in range(reps)]
    fw1 = float(np.median([t[0] for t in ts1]))
    bw1 = float(np.median([t[1] for t in ts1]))
    run.tape_segments = "auto"
    seg_gb = (8 * w["K"] + w["K"] - 1) * f0.size * 4 / 1e9
    run.v.read_timers()
    run.v.enable_timers(True)
    once()
    kind_ms, kind_n = run.v.read_timers()
    run.v.enable_timers(False)
    run.v.status()
    ok = bool(torch.isfinite(ft.grad).all()) and bool(torch.isfinite(pt.grad).all())
    cells = f0.size
    per = {}
    for k in kind_ms:
        if k.startswith("adj_") and kind_n[k]:
            # per sweep: a velocity sweep's adjoint may add a per-cell summing launch
            ms = kind_ms[k] / (w["steps"] * (2 if k in ("adj_ux", "adj_uy", "adj_uz") else 1))
            fk = "sweep_" + k[4:]
            fms = kind_ms[fk] / max(1, kind_n[fk]) if kind_ms.get(fk) else None
            per[k] = {"ms_per_sweep": ms, "launches": kind_n[k], "cell_updates_per_s": cells / (ms * 1e-3),
                      "GBs": 12.0 * cells / (ms * 1e-3) / 1e9,
                      "vs_forward_sweep": (ms / fms) if fms else None}
    # self-consistent run: phi^{n+1} from the post-drift moment plus a background
    from paper_2110_15867_gb300.autograd import run_rho_sc
    bg = torch.from_numpy(3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=w["seed"] + 1))).to(dev).requires_grad_()

    def once_sc():
        ft.grad = None
        pt.grad = None
        bg.grad = None
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        rho = run_rho_sc(ft, pt, bg, run, dt, 1.0, 1.0, w["steps"], w["K"])
        e[1].record()
        loss = (torch.fft.fftn(rho).abs() ** 2 * mask).sum()
        loss.backward()
        e[2].record()
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])

    once_sc()
    ts = [once_sc() for _ in range(reps)]
    sfw = float(np.median([t[0] for t in ts]))
    sbw = float(np.median([t[1] for t in ts]))
    run.v.status()
    ok_sc = bool(torch.isfinite(ft.grad).all()) and bool(torch.isfinite(pt.grad).all()) and \
        bool(torch.isfinite(bg.grad).all())
    run.close()
    del ft, pt, bg
    torch.cuda.empty_cache()
    return {"workload": "%s: %d^3 x %d^3 cells FP32, %d steps, checkpoint every %d, external phi, "
                        "loss sum over 0<|n|<8 of |rho_hat|^2" % (w["name"], n, nu, w["steps"], w["K"]),
            "forward_ms": fw, "backward_ms": bw, "backward_over_forward": bw / fw,
            "taped_segments": taped, "segments": nseg, "tape_GB": taped * seg_gb,
            "one_taped_segment": {"forward_ms": fw1, "backward_ms": bw1, "backward_over_forward": bw1 / fw1,
                                  "tape_GB": seg_gb,
                                  "what": "the backward runs the other segments again from their checkpoints"},
            "adjoint_sweeps": per, "gradients_finite": ok,
            "self_consistent": {"what": "the same run with phi^{n+1} from the post-drift moment plus a "
                                        "background (Poisson every step); gradients for f0, phi0, rho_bg",
                                "forward_ms": sfw, "backward_ms": sbw, "backward_over_forward": sbw / sfw,
                                "gradients_finite": ok_sc}}


def run_ours(args):
    import torch
    from paper_2110_15867_gb300 import binding as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.load()
    w = WORKLOAD
    n, nu, V, L = w["n"], w["nu"], w["V"], w["L"]
    f, rho_bg = build_inputs(torch, dev)
    cells = f.numel()
    v = B.Vlasov(f, L=L, V=V)
    if args.fused_kick is not None:
        v.set_fused_kick(args.fused_kick)
    if args.fused_moment is not None:
        v.set_fused_moment(bool(args.fused_moment))
    rho = torch.empty((n, n, n), dtype=torch.float64, device=dev)
    phi = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    phi2 = torch.empty_like(phi)
    v.moment(rho)
    v.poisson(rho, w["a0"], w["four_pi_G"], rho_bg=rho_bg, phi=phi)

    def one_step(k, total):
        nonlocal phi, phi2
        a_s, a_h, a_e, cfl = schedule(k, total)
        dt = drift_dt(cfl, a_h, n, nu, V, L)
        v.step(dt, a_h, a_e, phi, rho_bg=rho_bg, four_pi_G=w["four_pi_G"], phi_next=phi2, rho_nu=rho)
        phi, phi2 = phi2, phi

    for k in range(args.warmup):
        one_step(k, args.warmup)
    v.status()
    v.read_timers()  # reset the launch counters
    v.enable_timers(True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):  # a runs from a0 to a1 once over the timed steps
        one_step(k, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    kind_ms, kind_n = v.read_timers()
    v.enable_timers(False)
    v.status()
    ms_total = max_over_ranks(ms_total, dist, dev)
    value = whole_job_rate(world, cells, args.steps, ms_total)

    # dominant kernel and its roofline: algorithmic bytes = 8 B per cell update x the
    # updates one launch makes, over its mean event time, against the measured copy peak
    sweep_kinds = [k for k in kind_ms if k.startswith("sweep_") or k == "kick"]
    dom = max(sweep_kinds, key=lambda k: kind_ms[k])
    dom_ms = kind_ms[dom] / max(1, kind_n[dom])
    hbm_peak, peak_src = measured_peaks()
    upd = UPDATES_PER_PASS.get(dom, 1)
    alg_bytes = BYTES_PER_UPDATE * upd * cells
    moved_bytes = BYTES_PER_UPDATE * cells  # what one pass reads and writes
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                "peak_source": "%s copy peak (MEASURED_PEAKS.json hbm_gbs)" % peak_src if peak_src == "measured"
                else "fallback 6.8 TB/s", "unit": "GB/s", "frac": achieved / hbm_peak,
                "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
                "traffic": committed_traffic(dom), "algorithmic_bytes_per_launch": alg_bytes,
                "cell_updates_per_launch": upd * cells,
                "hbm_frac_actual_bytes": moved_bytes / (dom_ms * 1e-3) / 1e9 / hbm_peak,
                "ms_per_launch": dom_ms}
    alu = committed_alu(dom)
    if alu is not None:
        roofline["alu_pipe_active_pct_ncu"] = alu
    per_kind = {k: {"ms_per_launch": (kind_ms[k] / kind_n[k]) if kind_n[k] else 0.0,
                    "launches": kind_n[k]} for k in kind_ms if kind_n[k]}
    for k in sweep_kinds:
        if kind_n[k]:
            t = per_kind[k]["ms_per_launch"] * 1e-3
            u = UPDATES_PER_PASS.get(k, 1)
            per_kind[k]["cell_updates_per_s"] = u * cells / t
            per_kind[k]["GBs"] = BYTES_PER_UPDATE * u * cells / t / 1e9
            per_kind[k]["frac"] = per_kind[k]["GBs"] / hbm_peak
            if u > 1:
                per_kind[k]["GBs_actual_bytes"] = BYTES_PER_UPDATE * cells / t / 1e9
    gpu_launches = int(sum(kind_n.values()))
    step_hbm = step_bandwidth(kind_n, sweep_kinds, cells, args.steps, ms_total / args.steps, hbm_peak)

    # velocity moments of the final state (density, mean velocity, dispersion tensor), timed alone
    um = torch.empty((3, n, n, n), dtype=torch.float64, device=dev)
    s2 = torch.empty((6, n, n, n), dtype=torch.float64, device=dev)
    B.vlasov_moments(v.ctx, rho.data_ptr(), um.data_ptr(), s2.data_ptr())
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(3):
        B.vlasov_moments(v.ctx, rho.data_ptr(), um.data_ptr(), s2.data_ptr())
    m1.record(stream)
    torch.cuda.synchronize()
    v.status()
    m_ms = m0.elapsed_time(m1) / 3
    moments = {"ms_per_launch": m_ms, "GBs": 4.0 * cells / (m_ms * 1e-3) / 1e9,
               "what": "rho, mean velocity, dispersion tensor of the 64^3 x 32^3 state (4 B read per cell)"}
    del um, s2

    # end to end through the C ABI with host buffers: vlasov_step_host reads f from pinned
    # host memory, steps and writes it back (x-slabs copied in and out on streams of their
    # own behind the cell-local sweeps; a step's uploads run beside the previous step's
    # downloads); rho comes back too
    e2e = None
    if not args.no_e2e:
        fh = torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
        fh.copy_(f)
        # each step's rho is read back on a side stream into one of two buffers, so that the
        # read (queued behind the slab downloads on the copy engine) does not hold up the
        # next step; the step after next writes the same rho buffer once that read is done
        rho_d = [rho, torch.empty_like(rho)]
        rho_h = [torch.empty(rho.shape, dtype=rho.dtype, pin_memory=True) for _ in range(2)]
        side = torch.cuda.Stream(device=dev)
        stepped = [torch.cuda.Event() for _ in range(2)]
        read = [torch.cuda.Event() for _ in range(2)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

        def host_step(k, total):
            nonlocal phi, phi2
            a_s, a_h, a_e, cfl = schedule(k, total)
            dt = drift_dt(cfl, a_h, n, nu, V, L)
            b = k % 2
            if k >= 2:
                stream.wait_event(read[b])
            v.step_host(fh, dt, a_h, a_e, phi, rho_bg=rho_bg, four_pi_G=w["four_pi_G"], phi_next=phi2,
                        rho_nu=rho_d[b])
            stepped[b].record(stream)
            side.wait_event(stepped[b])
            with torch.cuda.stream(side):
                rho_h[b].copy_(rho_d[b], non_blocking=True)
            read[b].record(side)
            phi, phi2 = phi2, phi

        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        host_step(0, 1)  # warm-up: the copy streams and their events
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.e2e_steps):
            host_step(k, args.e2e_steps)
        v.host_wait()  # the last step's downloads inside the timed region
        for b in range(2):
            stream.wait_event(read[b])  # and the last reads of rho
        t1.record(stream)
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1)
        e_ms = max_over_ranks(e_ms, dist, dev)
        v.status()
        # the copies alone, for scale
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(stream)
        v.upload(fh)
        c1.record(stream)
        v.download(fh)
        c2.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": whole_job_rate(world, cells, args.e2e_steps, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(f.numel() * f.element_size()),
               "d2h_bytes_per_step": int(f.numel() * f.element_size() + rho.numel() * rho.element_size()),
               "steps": args.e2e_steps, "ms_per_step": e_ms / args.e2e_steps,
               "call": "vlasov_step_host on pinned host memory",
               "copy_alone_ms": {"h2d": c0.elapsed_time(c1), "d2h": c1.elapsed_time(c2)}}
        del fh

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
        cpu["per_axis"] = cpu_per_axis()
    v.close()
    del f, v
    torch.cuda.empty_cache()
    lowprec = None
    if not args.no_lowprec:
        lowprec = run_lowprec(torch, B, dev, max(2, min(args.steps, 3)), 2)
        for k in ("bf16", "f16"):
            lowprec[k]["vs_fp32"] = lowprec[k]["value"] / (9.0 * cells * args.steps / (ms_total * 1e-3))
    large = None
    if not args.no_large:
        large = run_large(torch, B, dev, 5, 2)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(torch, dev)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world),
            "roofline": roofline,
            "step_hbm": step_hbm,
            "kernels": per_kind,
            "cpu_baseline": cpu,
            "lowprec": lowprec,
            "large": large,
            "adjoint": adjoint,
            "moments": moments,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Each requested sweep (or, with --adjoint, its adjoint) twice plus the moment on a
    small FP32 grid (default (64, 8, 8) x 32^3: 1.34e8 cells, 537 MB)."""
    import torch
    from paper_2110_15867_gb300 import binding as B
    from paper_2110_15867_gb300 import inputs as I
    n, nu, V = tuple(int(x) for x in args.profile_shape.split(",")), args.profile_nu, 5.0
    axes = [int(a) for a in args.axes.split(",")]
    dev = torch.device("cuda", 0)
    delta = torch.from_numpy(I.gaussian_field(n, 0.05, seed=2)).to(dev)
    Fu = torch.from_numpy(I.fermi_dirac(nu, V)).to(dev)
    f = ((1 + delta)[:, :, :, None, None, None] * Fu[None, None, None]).float().contiguous()
    scale = None
    if args.profile_dtype != "f32":
        f, scale = B.encode_lines(f, {"bf16": torch.bfloat16, "f16": torch.float16}[args.profile_dtype])
    phi_np = I.fourier_potential(n, seed=3)
    phi = torch.from_numpy(phi_np.astype(np.float32)).to(dev)
    cmax = courant_per_dt(phi_np, n, nu, V)
    rho = torch.empty(n, dtype=torch.float64, device=dev)
    if args.step:
        # one Eq. (5) step: the one-pass kicks and the three drift sweeps
        v = B.Vlasov(f, V=V, scale=scale)
        dt = 0.7 / max(max(cmax[:3]), 0.5 * max(cmax[3:]))
        for _ in range(2):
            v.step(dt, 1.0, 1.0, phi, rho_nu=rho)  # the x sweep sums the moment
    elif args.adjoint:
        lam = torch.from_numpy(np.random.default_rng(4).standard_normal(f.shape).astype(np.float32)).to(dev)
        dLdg = torch.zeros(n, dtype=torch.float64, device=dev)
        v = B.Vlasov(torch.empty_like(f), V=V)
        for _ in range(2):
            for ax in axes:
                v.sweep_adjoint(f, lam, ax, 0.7 / cmax[ax], 1.0, phi, dLdg if ax >= 3 else None)
    else:
        v = B.Vlasov(f, V=V, scale=scale)
        if args.streamed:
            v.set_position_tiles(False)
        for _ in range(2):
            for ax in axes:
                v.sweep(ax, 0.7 / cmax[ax], 1.0, phi)
            v.moment(rho)
    v.status()
    v.close()
    return 0


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
