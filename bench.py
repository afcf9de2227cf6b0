#!/usr/bin/env python3
"""Benchmark of the GM checkpoint-restart hot path on GB300.

One step = compress (adaptive penalised EM + final unpenalised step + target
charge deposit) and reconstruct (sampling, Gauss'-law weight correction,
Lemons projection) of one batch of cells.  Metric: particles/s =
N_in / (t_compress + t_reconstruct), with N' = N_in per cell.

Default workload: the full-scale 1D-3V pipeline -- 262144 cells with
log-normal particle counts N_j = round(512 exp(0.47 Z)) clipped to
[16, 8192] (about 1.5e8 particles), one bi-Maxwellian per cell (v_th,par =
0.1 along x, T_perp/T_par ~ U[4, 25], drift U[-0.1, 0.1]^3), FP32
velocities, FP64 weights and positions, Kmax = 10, quadratic B-spline shape
functions; learned initialisation against plain EM, both timed, with the
M-step in FP64 (statistic sums, covariance updates, Cholesky factors and
inverses).  ``--workload mixture_1d1v`` and ``bimaxwellian_1d3v`` select the
4096-cell 1D-1V and the 2048 x 4000 1D-3V batches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmcr|reference]

Under torchrun every rank fits its own independent batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "GM CR particles/s (compress+reconstruct) on GB300, learned-init vs plain EM"
UNIT = "particles/s"
WORKLOAD_DESCS = {
    "lognormal_1d3v": ("lognormal_1d3v: full-scale 1D-3V pipeline, 262144 cells x round(512 exp(0.47 Z)) "
                       "particles (clip 16-8192, ~1.5e8), one bi-Maxwellian per cell (T_perp/T_par "
                       "U[4,25], drift U[-0.1,0.1]^3), FP32 v, FP64 x/alpha, Kmax=10, S2 shape, "
                       "tol=1e-6, max_sweeps=1000, N'=N per cell"),
    "mixture_1d1v": ("mixture_1d1v: 4096 cells x Poisson(2000) particles (clip 200-8000), "
                     "1-4 drifting Maxwellians per cell, FP32 v, FP64 x/alpha, Kmax=8, S2 shape, "
                     "tol=1e-6, max_sweeps=1000, N'=N per cell"),
    "bimaxwellian_1d3v": ("bimaxwellian_1d3v: 2048 cells x 4000 particles, one bi-Maxwellian per cell "
                          "(T_perp/T_par U[4,25], drift U[-0.1,0.1]^3), FP32 v, FP64 x/alpha, Kmax=10, "
                          "S2 shape, tol=1e-6, max_sweeps=1000, N'=N per cell"),
}
WORKLOAD_DESC = WORKLOAD_DESCS["lognormal_1d3v"]


def workload_desc(name: str) -> str:
    return WORKLOAD_DESCS.get(name, name)
L2_BYTES = 126 * 1024 * 1024


def rank_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Each rank fits an independent batch: its own generator seed."""
    return workloads.GEN_SEED_BASE + 1 + 1000 * rank


def make_workload(name: str, rank: int):
    if name == "mixture_1d1v":
        return workloads.mixture_1d1v(seed=rank_seed(rank))
    if name == "two_stream_1d1v":
        return workloads.two_stream_1d1v(seed=rank_seed(rank))
    if name == "bimaxwellian_1d3v":
        return workloads.bimaxwellian_1d3v(seed=rank_seed(rank))
    if name == "lognormal_1d3v":
        return workloads.lognormal_1d3v(seed=rank_seed(rank))
    raise SystemExit(f"unknown workload {name}")


def reduce_max(value: float, dist, device=None) -> float:
    """Max over ranks (the slowest rank sets the job time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"gmcr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic work of the EM kernel
# ---------------------------------------------------------------------------
FLOPS_PER_PK = {1: 30, 3: 90}  # FP32 flops per particle per component step


# DRAM bytes (read + write) of one em_kernel launch per particle, from an
# ncu capture of 1216 cells of the 1D-1V batch (FP32 v): 30.30 MB for
# 2434617 particles, i.e. the inputs read once (4 B v + 8 B alpha).  The
# traffic grows with the particles, so a full launch is this times n.
EM_DRAM_BYTES_PER_PARTICLE = 30.302464e6 / 2434617


def em_flops(counts: np.ndarray, kwork: np.ndarray, D: int) -> float:
    return float(np.sum(counts.astype(np.float64) * kwork.astype(np.float64))) * FLOPS_PER_PK[D]


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# Second rooflines of the EM kernel: the special-function unit and the FP64
# pipe.  MUFU work per particle and component step: two base-2 exponentials
# (the replaced term of the previous component and the density of the
# current one) and one reciprocal (gamma = alpha G / s); per particle and
# sweep one base-2 logarithm (eq. lnL-GM).  Its peak: 16 results per SM per
# clock (the documented throughput of exp2 / log2 / reciprocal on compute
# capability 10.x) x 152 SMs x the clock.  FP64 work per particle: the
# prologue's moments, 2 (1 + D + D(D+1)/2) flops, and per component of the
# final step the FP64 responsibility (3), the centred velocity (2 D) and its
# statistics (1 + 2 D + D(D+1)); its peak is GB300's nominal FP64 rate.
MUFU_PER_PK = 3
MUFU_PER_PSWEEP = 1
MUFU_PER_SM_CLK = 16
FP64_PEAK_TFLOPS = 1.25


def fp64_flops_per_particle(D: int, K: np.ndarray) -> np.ndarray:
    NM = D * (D + 1) // 2
    return 2 * (1 + D + NM) + K.astype(np.float64) * (3 + 2 * D + 1 + 2 * D + 2 * NM)


def em_secondary_rooflines(counts: np.ndarray, K: np.ndarray, kwork: np.ndarray,
                           sweeps: np.ndarray, D: int, seconds: float, sm_mhz: float,
                           sms: int = 152) -> list:
    n = counts.astype(np.float64)
    mufu = float(np.sum(n * (MUFU_PER_PK * kwork.astype(np.float64) +
                             MUFU_PER_PSWEEP * sweeps.astype(np.float64))))
    mufu_rate = mufu / seconds / 1e12
    mufu_peak = sms * MUFU_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    f64 = float(np.sum(n * fp64_flops_per_particle(D, K)))
    f64_rate = f64 / seconds / 1e12
    return [{"unit": "MUFU Top/s", "achieved": mufu_rate, "peak": mufu_peak,
             "frac": mufu_rate / mufu_peak,
             "note": f"sum_j N_j ({MUFU_PER_PK} kwork_j + {MUFU_PER_PSWEEP} sweeps_j); peak = "
                     f"{sms} SMs x {MUFU_PER_SM_CLK} / clock x {sm_mhz:.0f} MHz"},
            {"unit": "FP64 TFLOP/s", "achieved": f64_rate, "peak": FP64_PEAK_TFLOPS,
             "frac": f64_rate / FP64_PEAK_TFLOPS,
             "note": "prologue moments + final FP64 step per particle; peak = nominal GB300 FP64"}]


def fp64_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """152 SMs x 2 FP64 FMA lanes per clock x 2 flops x the clock (at
    2070 MHz 1.26 TFLOP/s, GB300's nominal 1.25)"""
    return sms * 2 * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic work of the kernels of one step, per particle of the cells a
# kernel handles, D = 1 or 3, NM = D (D + 1) / 2, and the bound each is
# reported against:
#  em_k1_kernel      HBM: x and alpha read once for every cell (the charge
#                    deposit is fused in), v (FP32) once for the cells whose
#                    start has one component: 16 + 4 D bytes for those, 16
#                    for the others.  (The method's FP64 moments, 1 + 3 D +
#                    2 NM flops, run as exact integer sums: a secondary line.)
#  recon_stats_kernel ALU: the sampler's 32-bit integer / FP32 operations,
#                    counted from the definitions: two Philox4x32-10 blocks
#                    (10 rounds of two 32x32->64 multiplies and two
#                    three-input XORs, 40 ops each), two operations per
#                    52-bit uniform and one per 32-bit uniform (1V: four
#                    52-bit; 3V: two 52-bit, four 32-bit), Box-Muller (ln 10
#                    + sqrt 1 + scale 1 per radius, 8 per sine or cosine, 1
#                    per product; 1V one radius and one cosine, 3V two
#                    radii, three trig values), f = L xi (1 or 6), and the
#                    exact sums (position 8, each velocity dimension 14):
#                    132 (1V), 195 (3V) ops; peak = 152 SMs x 128 lanes x the
#                    clock.  Secondary: the staged draws written, 20 bytes
#                    (12 for 1V).
#  recon_emit_kernel HBM: the staged draw read (20 / 12 bytes) and x, v,
#                    alpha written (16 + 8 D); secondary FP64: x = (j + u0)
#                    dx (2 flops) and v = c + a f (2 D).
#  deposit           HBM: x and alpha read, 16 bytes; secondary FP64: the
#                    cell fraction x / dx - j (2 flops)
#  features_kernel   HBM: v (FP32) and alpha read once, 4 D + 8
#  mlp_forward       BF16 tensor flops 2 (F H + 2 H^2 + H O) per cell
#  em_kernel         FP32 flops FLOPS_PER_PK per particle and component step
K1_FP64_PER_P = {1: 1 + 3 + 2, 3: 1 + 9 + 12}
STATS_OPS_PER_P = {1: 2 * 40 + 2 * 4 + (12 + 8 + 1) + 1 + (8 + 14),
                   3: 2 * 40 + (2 * 2 + 4) + (2 * 12 + 3 * 8 + 3) + 6 + (8 + 3 * 14)}
STAGED_BYTES_PER_P = {1: 12, 3: 20}
EMIT_FP64_PER_P = {1: 2 + 2, 3: 2 + 6}
DEPOSIT_FP64_PER_P = 2


# DRAM traffic (read + write) per particle of the learned step's largest
# kernels, from one ncu capture (--set full, one launch each) of the
# first 16384 cells of the 262144-cell lognormal_1d3v batch (9324406
# particles), the learned step run with a saved network under
# ncu --set full --clock-control none -k regex:<kernel> -c 1.  The traffic
# grows with the particles, so a full launch is this times n.
# An entry must be removed when its kernel changes.
DRAM_BYTES_PER_PARTICLE = {
    ("lognormal_1d3v", "recon_stats_kernel"): (3.977728e6 + 165.554688e6) / 9324406,
    ("lognormal_1d3v", "recon_emit_kernel"): (230.330880e6 + 315.433472e6) / 9324406,
    ("lognormal_1d3v", "features_kernel"): (214.720768e6 + 20.601088e6) / 9324406,
}


def alu_peak_tops(sm_mhz: float, sms: int = 152) -> float:
    """152 SMs x 128 32-bit lanes (FP32 / INT32) x the clock, in T ops/s"""
    return sms * 128 * sm_mhz * 1e6 / 1e12


def kernel_roofline(kernels: dict, ctx: dict) -> dict:
    """Roofline of the step's dominant kernel (largest traced device time):
    algorithmic work per launch / the kernel's traced time per step against
    the bounding unit's peak (FP64, FP32 and the 32-bit lanes from unit
    counts and the clock, HBM and BF16 measured)."""
    if not kernels:
        return None
    name, kt = max(kernels.items(), key=lambda kv: kv[1]["ms"])
    sec = kt["ms"] * 1e-3
    n = ctx["counts"].astype(np.float64)
    D = ctx["D"]
    hbm = ctx["hbm_gbs"]
    f64_peak = fp64_peak_tflops(ctx["sm_mhz"])
    f32_peak = fp32_peak_tflops(ctx["sm_mhz"])
    f64_note = f"peak = 152 SMs x 2 FP64 FMA/clock x 2 x {ctx['sm_mhz']:.0f} MHz"

    bpp = DRAM_BYTES_PER_PARTICLE.get((ctx.get("workload"), name))
    traffic = None if bpp is None else bpp * float(n.sum()) / max(1, kt["launches_per_step"])

    def line(bound, achieved, peak, unit, note, secondary=None):
        return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "ms_per_launch": kt["ms"] / max(1, kt["launches_per_step"]),
                "note": note, "secondary": secondary or []}

    def sec_line(unit, achieved, peak, note):
        return {"unit": unit, "achieved": achieved, "peak": peak, "frac": achieved / peak, "note": note}

    if name == "em_k1_kernel":
        sel = ctx["K0"] == 1 if ctx["K0"] is not None else np.ones_like(n, dtype=bool)
        np_ = float(n[sel].sum())
        b = (float(n.sum()) * 16 + np_ * 4 * D) / sec / 1e9
        f = np_ * K1_FP64_PER_P[D] / sec / 1e12
        return line("hbm", b, hbm, "GB/s",
                    f"x and alpha (16 B) read per particle, and v ({4 * D} B) per particle of the one-component "
                    f"cells ({int(sel.sum())} cells, {np_:.0f} particles); peak measured (copy)",
                    [sec_line("TFLOP/s", f, f64_peak, f"the method's FP64 moment flops ({K1_FP64_PER_P[D]} per "
                              f"particle), run as exact integer sums; {f64_note}")])
    if name == "recon_stats_kernel":
        o = float(n.sum()) * STATS_OPS_PER_P[D] / sec / 1e12
        b = float(n.sum()) * STAGED_BYTES_PER_P[D] / sec / 1e9
        return line("alu", o, alu_peak_tops(ctx["sm_mhz"]), "Tops/s",
                    f"the sampler's 32-bit operations, {STATS_OPS_PER_P[D]} per resampled particle (Philox, "
                    f"Box-Muller, f = L xi, exact sums); peak = 152 SMs x 128 lanes x {ctx['sm_mhz']:.0f} MHz",
                    [sec_line("GB/s", b, hbm, f"{STAGED_BYTES_PER_P[D]} B of staged draws written per particle; "
                              "peak measured (copy)")])
    if name == "recon_emit_kernel":
        by = STAGED_BYTES_PER_P[D] + 16 + 8 * D
        b = float(n.sum()) * by / sec / 1e9
        f = float(n.sum()) * EMIT_FP64_PER_P[D] / sec / 1e12
        return line("hbm", b, hbm, "GB/s",
                    f"{by} B per particle: the staged draw read, x, v, alpha written; peak measured (copy)",
                    [sec_line("TFLOP/s", f, f64_peak, f"FP64 flops = {EMIT_FP64_PER_P[D]} per particle; {f64_note}")])
    if name.startswith("deposit"):
        b = float(n.sum()) * 16 / sec / 1e9
        f = float(n.sum()) * DEPOSIT_FP64_PER_P / sec / 1e12
        return line("hbm", b, hbm, "GB/s", "16 B (x, alpha) read per particle; peak measured (copy)",
                    [sec_line("TFLOP/s", f, f64_peak, f"FP64 flops = {DEPOSIT_FP64_PER_P} per particle; {f64_note}")])
    if name == "features_kernel":
        b = float(n.sum()) * (4 * D + 8) / sec / 1e9
        return line("hbm", b, hbm, "GB/s", f"{4 * D + 8} B read per particle; peak measured (copy)")
    if name.startswith("mlp_forward"):
        H = 256
        f = 2.0 * len(n) * (ctx["F"] * H + 2 * H * H + H * ctx["O"]) / sec / 1e12
        return line("tensor", f, ctx["bf16_tflops"], "TFLOP/s", "BF16 dense flops of the 4 layers; peak measured (cuBLAS burst)")
    if name == "em_kernel":
        f = em_flops(ctx["counts"], ctx["kwork"], D) / sec / 1e12
        return line("alu", f, f32_peak, "TFLOP/s",
                    f"FP32 flops = sum_j N_j * kwork_j * {FLOPS_PER_PK[D]}; peak = 152 SMs x 128 FP32 lanes x 2 "
                    f"x {ctx['sm_mhz']:.0f} MHz",
                    em_secondary_rooflines(ctx["counts"], ctx["K"], ctx["kwork"], ctx["sweeps"], D, sec,
                                           ctx["sm_mhz"]))
    b = float(len(n)) * 64 / sec / 1e9
    return line("hbm", b, hbm, "GB/s", "per-cell records, ~64 B per cell")


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample of cells
# ---------------------------------------------------------------------------
def sub_workload(wl, ncells: int):
    ncells = min(ncells, wl.C)
    n = int(wl.cell_off[ncells])
    p = dict(wl.params)
    p["L"] = wl.params["L"] * ncells / wl.C  # same dx
    return workloads.Workload(wl.name + "_sample", wl.cell_off[: ncells + 1].copy(), wl.x[:n].copy(),
                              np.ascontiguousarray(wl.v[:, :n]), wl.alpha[:n].copy(), p)


def strided_sample(wl, ncells: int):
    """Every (C / ncells)-th cell of the workload (at most ncells cells), as
    a workload of its own: a sample that follows the batch's size
    distribution.  Positions are moved into the sample's own periodic mesh
    (same dx) so that the reconstruction's mesh is consistent."""
    stride = max(1, wl.C // max(1, ncells))
    cells = np.arange(0, wl.C, stride)[:ncells]
    counts = wl.counts()[cells]
    off = np.zeros(len(cells) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    idx = np.concatenate([np.arange(wl.cell_off[j], wl.cell_off[j + 1]) for j in cells]) \
        if len(cells) else np.zeros(0, dtype=np.int64)
    dx = wl.params["L"] / wl.C
    shift = np.repeat((np.arange(len(cells)) - cells) * dx, counts)
    p = dict(wl.params)
    p["L"] = dx * len(cells)
    sw = workloads.Workload(wl.name + "_sample", off, wl.x[idx] + shift, np.ascontiguousarray(wl.v[:, idx]),
                            wl.alpha[idx].copy(), p)
    return sw, cells


def oracle_step(wl, nthreads: int, cell_ids=None) -> float:
    import oracle
    t0 = time.perf_counter()
    out = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=nthreads, cell_ids=cell_ids)
    oracle.reconstruct(wl.params, out["K"], out["params"], out["W"], out["rho_target"], wl.cell_off,
                       nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the ISA)."""
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
    import platform
    return platform.machine()


ORACLE_MAX_SAMPLE_CELLS = 8192


def sized_oracle_sample(wl, cores: int, budget_s: float):
    """A strided sample of the workload's cells whose oracle step
    (compress + reconstruct, OpenMP over cells on `cores` threads) takes
    about budget_s, grown from 2 cells per core up to 8192 cells; returns
    (sample, cells, seconds of the last timed step)."""
    ncells = min(wl.C, max(2 * cores, 8))
    while True:
        sw, cells = strided_sample(wl, ncells)
        t = oracle_step(sw, cores, cell_ids=cells)
        if t >= budget_s / 3 or ncells >= min(wl.C, ORACLE_MAX_SAMPLE_CELLS):
            return sw, cells, t
        ncells = min(wl.C, ORACLE_MAX_SAMPLE_CELLS,
                     max(2 * ncells, int(ncells * budget_s / max(t, 1e-3) / 1.5)))


def cpu_baseline(wl, budget_s: float = 15.0) -> dict:
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    sw, cells, t = sized_oracle_sample(wl, cores, budget_s)
    # one thread on a few cells of the same strided sample
    s1, c1 = strided_sample(wl, 4)
    t1 = oracle_step(s1, 1, cell_ids=c1)
    full_s = t * wl.ntot / max(1, sw.ntot)
    return {"value": sw.ntot / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {wl.C // len(cells)}-th cell: {sw.C} cells ({sw.ntot} particles) of the "
                      f"workload, compress+reconstruct, OpenMP over cells, {t:.1f} s",
            "extrapolated_full_workload_s": full_s,
            "extrapolation": "linear in particles: sample seconds x total / sample particles",
            "cpu_model": cpu_model(),
            "single_thread": {"value": s1.ntot / t1, "unit": UNIT, "cores": 1,
                              "sample": f"{s1.C} strided cells ({s1.ntot} particles), {t1:.1f} s"}}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    wl = make_workload(args.workload, 0)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # each step is a bounded strided sample of the workload, sized so that
    # warmup + steps together take about ref_budget seconds
    per_step = max(2.0, args.ref_budget / max(1, args.steps + args.warmup))
    sw, cells, _ = sized_oracle_sample(wl, cores, per_step)
    for _ in range(args.warmup):
        oracle_step(sw, cores, cell_ids=cells)
    times = [oracle_step(sw, cores, cell_ids=cells) for _ in range(args.steps)]
    tot = sum(times)
    value = sw.ntot * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload),
                       "sample_cells": sw.C, "sample_particles": sw.ntot,
                       "init": "paper (random particles)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"every {wl.C // len(cells)}-th cell: {sw.C} cells "
                                       f"({sw.ntot} particles) per step",
                             "extrapolated_full_workload_s": (tot / args.steps) * wl.ntot / max(1, sw.ntot),
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def make_train_workload(name: str, rank: int, chunk: int, C: int):
    """Training cells: the same generator family as the benchmark workload,
    with seeds disjoint from every rank's benchmark batch."""
    seed = rank_seed(rank) + 7919 * (chunk + 1)
    if name == "mixture_1d1v":
        return workloads.mixture_1d1v(C=C, seed=seed)
    if name == "two_stream_1d1v":
        return workloads.two_stream_1d1v(seed=seed)
    if name == "bimaxwellian_1d3v":
        return workloads.bimaxwellian_1d3v(C=C, seed=seed)
    return workloads.lognormal_1d3v(C=C, seed=seed)


def run_gmcr(args):
    import torch
    rank, world, local = rank_info()
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    from paper_2007_12273_gb300 import build as gbuild
    from paper_2007_12273_gb300 import gm, learned
    gbuild.build()
    gm.load()

    wl = make_workload(args.workload, rank)
    if args.cells:
        wl = sub_workload(wl, args.cells)
    D = wl.D
    over = dict(precision=0 if args.mstep == "fp64" else 1, threads_per_cell=args.threads_per_cell,
                smem_particles=args.smem_particles)
    cfg = gm.config(wl.params, **over)
    rcfg = gm.config(wl.params, seed_key="recon_seed", **over)
    counts = wl.counts()
    n = wl.ntot
    C = wl.C
    use_learned = args.init in ("learned", "both")
    use_plain = args.init in ("plain", "both")

    # inputs resident in HBM
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    cell_off, x, v, alpha = t(wl.cell_off), t(wl.x), t(wl.v), t(wl.alpha)
    out_off = cell_off

    def comp_out():
        return dict(K=torch.empty(C, dtype=torch.int32, device=device),
                    params=torch.empty((C, cfg.Kmax, gm.P_of(D)), dtype=torch.float64, device=device),
                    W=torch.empty(C, dtype=torch.float64, device=device),
                    rho_target=torch.empty(C, dtype=torch.float64, device=device),
                    lnL=torch.empty(C, dtype=torch.float64, device=device),
                    sweeps=torch.empty(C, dtype=torch.int32, device=device),
                    kwork=torch.empty(C, dtype=torch.int32, device=device),
                    status=torch.empty(C, dtype=torch.int32, device=device))
    rout = dict(x=torch.empty(n, dtype=torch.float64, device=device),
                v=torch.empty((D, n), dtype=torch.float64, device=device),
                alpha=torch.empty(n, dtype=torch.float64, device=device),
                status=torch.empty(C, dtype=torch.int32, device=device))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    # a side stream: CUDA graphs cannot capture the legacy default stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    # ---- launch shape of the EM kernel: the library's autotuner (untimed)
    tune = None
    if not args.threads_per_cell and not args.smem_particles:
        trial_ms = gm.gm_autotune(cfg, cell_off, x, v, alpha, stream=stream)
        tune = {"threads_per_cell": cfg.threads_per_cell, "smem_particles": cfg.smem_particles,
                "trial_ms": [round(z, 4) for z in trial_ms]}

    # ---- learned initialisation: the network is trained (untimed) on cells
    # of the same generator family fitted by the paper's method
    net, train_info = None, None
    if use_learned and args.load_net:
        # a network trained and saved by an earlier run (--save-net): lets a
        # profiler run skip the training launches
        saved = np.load(args.load_net)
        net = gm.Net(D, cfg.Kmax)
        net.load([saved[f"W{i}"] for i in range(4)], [saved[f"b{i}"] for i in range(4)])
        train_info = {"cells": int(saved["cells"]), "loaded_from": args.load_net}
        if args.presence_logit is None:
            args.presence_logit = float(saved["presence_logit"])
    elif use_learned:
        t0 = time.perf_counter()
        feats, Ts, Mks = [], [], []
        train_cells = args.train_cells or (65536 if D == 1 else 32768)
        nchunk = max(1, train_cells // 4096)
        for ch in range(nchunk):
            tw = make_train_workload(args.workload, rank, ch, 4096)
            f_, T_, M_, fit_ = learned.fit_targets(cfg, t(tw.cell_off), t(tw.x), t(tw.v), t(tw.alpha))
            feats.append(f_)
            Ts.append(T_)
            Mks.append(M_)
        calib = (tw, fit_["lnL"].clone())  # the last training chunk and its plain-EM objective
        feat = torch.cat(feats)
        T = torch.cat(Ts)
        Mk = torch.cat(Mks)
        torch.cuda.synchronize()
        t_fit = time.perf_counter() - t0
        net = gm.Net(D, cfg.Kmax)
        net.init_weights(seed=1)
        hist = learned.train(net, feat, T, Mk, epochs=args.epochs, batch=1024, lr=1e-3)
        train_info = {"cells": int(feat.shape[0]), "fit_seconds": t_fit,
                      "train_seconds": hist["seconds"], "epochs": args.epochs,
                      "adam_steps": hist["steps"], "loss_first": hist["loss"][0],
                      "loss_last": hist["loss"][-1]}
        del feat, T, Mk, feats, Ts, Mks
        # the decode's presence threshold, chosen on that training chunk
        # (untimed): the fastest threshold whose start reaches plain EM's
        # objective (eq. lnL-GM within 1e-4) as often as the best one, less
        # half a percent
        if args.presence_logit is None:
            args.presence_logit, train_info["presence_calibration"] = learned.calibrate_presence(
                net, cfg, *(t(a) for a in (calib[0].cell_off, calib[0].x, calib[0].v, calib[0].alpha)),
                calib[1])
        if args.save_net and rank == 0:
            np.savez(args.save_net, cells=train_info["cells"], presence_logit=args.presence_logit,
                     **{f"W{i}": w.cpu().numpy() for i, w in enumerate(net.W)},
                     **{f"b{i}": b.cpu().numpy() for i, b in enumerate(net.b)})

    feat_wstat = {}

    def init_learned(out_tensors):
        f_, w_ = gm.gm_features(cfg, cell_off, v, alpha, stream=stream)
        o_ = net.forward(f_, stream=stream)
        return gm.gm_mlp_decode(cfg, o_, w_, cell_off, stream=stream, presence_logit=args.presence_logit)

    # the learned path's EM launch shape, tuned from the learned start
    # (untimed): most of its cells start with one component, a cost balance
    # unlike the random start's
    cfg_l, tune_l = cfg, None
    if use_learned and tune is not None:
        cfg_l = gm.config(wl.params, **over)
        K0_, prm0_ = init_learned(None)
        trial_l = gm.gm_autotune(cfg_l, cell_off, x, v, alpha, stream=stream, init_K=K0_, init_params=prm0_)
        tune_l = {"threads_per_cell": cfg_l.threads_per_cell, "smem_particles": cfg_l.smem_particles,
                  "trial_ms": [round(z, 4) for z in trial_l]}
        # the tuners time samples; where they disagree, one fit of the whole
        # batch from the learned start per shape decides (untimed)
        if (cfg_l.threads_per_cell, cfg_l.smem_particles) != (cfg.threads_per_cell, cfg.smem_particles):
            fit_ms = {}
            for name, cf in (("plain-tuned", cfg), ("learned-tuned", cfg_l)):
                gm.gm_compress(cf, cell_off, x, v, alpha, stream=stream, init_K=K0_, init_params=prm0_)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                gm.gm_compress(cf, cell_off, x, v, alpha, stream=stream, init_K=K0_, init_params=prm0_)
                ev1.record(stream)
                torch.cuda.synchronize()
                fit_ms[name] = ev0.elapsed_time(ev1)
            tune_l["whole_batch_fit_ms"] = {k: round(z, 3) for k, z in fit_ms.items()}
            if fit_ms["plain-tuned"] < fit_ms["learned-tuned"]:
                cfg_l = cfg
        del K0_, prm0_

    def timed(path: str, steps: int, warmup: int):
        """per-step CUDA events (init, compress, reconstruct), L2 flushed
        between steps; the phases are replayed from CUDA graphs captured
        after the warm-up (unless --no-graph); returns per-phase mean ms and
        the compress outputs"""
        cout = comp_out()
        ecfg = cfg_l if path == "learned" else cfg

        def one(ev=None):
            if ev:
                ev[0].record(stream)
            kw = {}
            if path == "learned":
                K0, prm = init_learned(cout)
                kw = dict(init_K=K0, init_params=prm)
            if ev:
                ev[1].record(stream)
            gm.gm_compress(ecfg, cell_off, x, v, alpha, stream=stream, out=cout, **kw)
            if ev:
                ev[2].record(stream)
            gm.gm_reconstruct(rcfg, cout["K"], cout["params"], cout["W"], cout["rho_target"],
                              out_off, n_out=n, stream=stream, out=rout)
            if ev:
                ev[3].record(stream)

        for _ in range(warmup):
            one()
        torch.cuda.synchronize()
        one_direct = one
        graphs = None
        if not args.no_graph:
            graphs = []
            if path == "learned":
                f_, w_ = gm.gm_features(cfg, cell_off, v, alpha, stream=stream)
                o_ = net.forward(f_, stream=stream)
                K0, prm = gm.gm_mlp_decode(cfg, o_, w_, cell_off, stream=stream, presence_logit=args.presence_logit)
                gi = gm.Graph(stream)
                with gi:
                    gm.gm_features(cfg, cell_off, v, alpha, stream=stream, out=(f_, w_))
                    net.forward(f_, out=o_, stream=stream)
                    gm.gm_mlp_decode(cfg, o_, w_, cell_off, stream=stream, dest=(K0, prm),
                                     presence_logit=args.presence_logit)
                gi.keep(f_, w_, o_, K0, prm)
                graphs.append(gi)
                kw = dict(init_K=K0, init_params=prm)
            else:
                graphs.append(None)
                kw = {}
            gc = gm.Graph(stream)
            with gc:
                gm.gm_compress(ecfg, cell_off, x, v, alpha, stream=stream, out=cout, **kw)
            graphs.append(gc)
            gr = gm.Graph(stream)
            with gr:
                gm.gm_reconstruct(rcfg, cout["K"], cout["params"], cout["W"], cout["rho_target"],
                                  out_off, n_out=n, stream=stream, out=rout)
            graphs.append(gr)

            def one(ev=None):  # noqa: F811  (graph replay of the same step)
                for a, g_ in enumerate(graphs):
                    if ev:
                        ev[a].record(stream)
                    if g_ is not None:
                        g_.launch(stream)
                if ev:
                    ev[3].record(stream)

            for _ in range(warmup):
                one()
            torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(float(i))
            torch.cuda.nvtx.range_push("gmcr_step")  # lets a profiler select the timed steps
            one(evs[i])
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = [sum(e[a].elapsed_time(e[a + 1]) for e in evs) / steps for a in range(3)]
        if graphs:
            for g_ in graphs:
                if g_ is not None:
                    g_.close()
        # per-kernel device times: the same steps as direct calls, with the
        # library's event trace (CUDA events on the launching stream after
        # each kernel), the L2 flushed between steps as above
        tsteps = min(steps, 3)
        with gm.Trace() as tr:
            for i in range(tsteps):
                flush.fill_(float(i))
                one_direct()
            torch.cuda.synchronize()
        kern = {k: {"ms": v[0] / tsteps, "launches_per_step": v[1] / tsteps} for k, v in tr.times.items()}
        return {"ms_init": ms[0], "ms_compress": ms[1], "ms_reconstruct": ms[2], "kernels": kern}, cout

    clocks = ClockSampler(local)
    clocks.start()
    res = {}
    outs = {}
    for path in (["plain"] if use_plain else []) + (["learned"] if use_learned else []):
        r, co = timed(path, args.steps, args.warmup)
        r["ms_per_step"] = reduce_max(r["ms_init"] + r["ms_compress"] + r["ms_reconstruct"], dist, device)
        res[path] = r
        outs[path] = {k: vv.cpu().numpy() for k, vv in co.items() if k in ("K", "kwork", "sweeps", "status", "lnL")}
    clk = clocks.stop()
    head = "learned" if use_learned else "plain"
    step_ms = res[head]["ms_per_step"]
    total_particles = reduce_sum(float(n), dist, device)
    value = total_particles / (step_ms * 1e-3)
    rst = rout["status"].cpu().numpy()

    # ---- end to end through the API with host buffers ----------------------
    # Every step copies its inputs from pinned host memory and all its outputs
    # (particles, mixtures) back.  The copies run on streams of their own with
    # two device buffer sets, so step i's inputs arrive while step i - 1
    # computes and its outputs leave while step i + 1 computes -- a restart
    # code streaming its batches through the library would do the same.
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(wl.cell_off), pin(wl.x), pin(wl.v), pin(wl.alpha)]
    NB = 2
    d_in = [[torch.empty_like(h, device=device) for h in h_in] for _ in range(NB)]
    couts = [comp_out() for _ in range(NB)]
    routs = [rout] + [{k: torch.empty_like(vv) for k, vv in rout.items()} for _ in range(NB - 1)]
    out_keys = list(rout.keys()) + ["params", "K", "W", "rho_target"]
    src_of = lambda b, k: routs[b][k] if k in routs[b] else couts[b][k]
    h_out = [{k: torch.empty(tuple(src_of(b, k).shape), dtype=src_of(b, k).dtype).pin_memory()
              for k in out_keys} for b in range(NB)]
    h2d = sum(h.numel() * h.element_size() for h in h_in)
    d2h = sum(h.numel() * h.element_size() for h in h_out[0].values())
    e2e_steps = max(4, min(args.steps, 6))
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    ev_in, ev_done, ev_out = [ev() for _ in range(NB)], [ev() for _ in range(NB)], [ev() for _ in range(NB)]

    def e2e_step(i):
        b = i % NB
        s_in.wait_event(ev_done[b])  # step i - 2 has finished with this input set
        with torch.cuda.stream(s_in):
            for h, d in zip(h_in, d_in[b]):
                d.copy_(h, non_blocking=True)
        ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])  # step i - 2's outputs have left this set
        di, co, ro = d_in[b], couts[b], routs[b]
        kw = {}
        if head == "learned":
            f_, w_ = gm.gm_features(cfg, di[0], di[2], di[3], stream=stream)
            o_ = net.forward(f_, stream=stream)
            K0, prm = gm.gm_mlp_decode(cfg, o_, w_, di[0], stream=stream,
                                         presence_logit=args.presence_logit)
            kw = dict(init_K=K0, init_params=prm)
        gm.gm_compress(cfg_l if head == "learned" else cfg, di[0], di[1], di[2], di[3],
                       stream=stream, out=co, **kw)
        gm.gm_reconstruct(rcfg, co["K"], co["params"], co["W"], co["rho_target"],
                          di[0], n_out=n, stream=stream, out=ro)
        ev_done[b].record(stream)
        s_out.wait_event(ev_done[b])
        with torch.cuda.stream(s_out):
            for k, h in h_out[b].items():
                h.copy_(src_of(b, k), non_blocking=True)
        ev_out[b].record(s_out)

    for i in range(NB):
        e2e_step(i)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for i in range(e2e_steps):
        e2e_step(i)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / e2e_steps, dist, device)
    e2e_value = total_particles / (e2e_ms * 1e-3)

    # ---- statistics of the fit and the roofline of the EM kernel -----------
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_mhz)
    P = gm.P_of(D)
    numbers_per_particle = 1 + D + 1  # x, v, alpha

    def summary(path):
        o = outs[path]
        flops = em_flops(counts, o["kwork"], D)
        achieved = flops / (res[path]["ms_compress"] * 1e-3) / 1e12
        return {"value": total_particles / (res[path]["ms_per_step"] * 1e-3),
                "ms_init": res[path]["ms_init"], "ms_compress": res[path]["ms_compress"],
                "ms_reconstruct": res[path]["ms_reconstruct"],
                "Kbar": float(o["K"].mean()), "sweeps_mean": float(o["sweeps"].mean()),
                "maxsweeps_frac": float(np.mean((o["status"] & 1) != 0)),
                "compression_ratio": float(counts.sum() * numbers_per_particle /
                                           max(1.0, float(np.sum(o["K"])) * P)),
                "em_tflops": achieved, "em_frac_fp32_peak": achieved / peak,
                "em_secondary": em_secondary_rooflines(counts, o["K"], o["kwork"], o["sweeps"], D,
                                                       res[path]["ms_compress"] * 1e-3, sm_mhz)}

    paths = {p_: summary(p_) for p_ in res}
    if "plain" in outs and "learned" in outs:
        Lp, Ll = outs["plain"]["lnL"], outs["learned"]["lnL"]
        paths["learned"]["reaches_plain_L_1e-4"] = float(np.mean(Ll >= Lp - 1e-4 * np.abs(Lp)))
        paths["learned"]["mean_lnL_minus_plain"] = float(np.mean(Ll - Lp))
        paths["learned"]["training"] = train_info
        # calibration of that rate: plain EM from other random initial picks
        # (another seed, untimed) against the same plain run
        cfg2 = gm.config(dict(wl.params, seed=int(wl.params.get("seed", 1)) + 1000), **over)
        cfg2.threads_per_cell, cfg2.smem_particles = cfg.threads_per_cell, cfg.smem_particles
        L2 = gm.gm_compress(cfg2, cell_off, x, v, alpha, stream=stream)["lnL"].cpu().numpy()
        paths["plain"]["other_seed_reaches_plain_L_1e-4"] = float(np.mean(L2 >= Lp - 1e-4 * np.abs(Lp)))
        paths["plain"]["other_seed_mean_lnL_minus_plain"] = float(np.mean(L2 - Lp))
    hs = paths[head]
    K0_head = None
    if head == "learned":
        K0_head = init_learned(None)[0].cpu().numpy()

    def head_ctx(path):
        o = outs[path]
        return dict(counts=counts, D=D, K=o["K"], kwork=o["kwork"], sweeps=o["sweeps"], K0=K0_head,
                    sm_mhz=sm_mhz, hbm_gbs=float(peaks.get("hbm_gbs", 6800.0)),
                    bf16_tflops=float(peaks.get("bf16_tflops", 1900.0)), F=gm.feat_width(D),
                    O=gm.out_width(D, cfg.Kmax), ms_compress=res[path]["ms_compress"],
                    workload=args.workload if not args.cells else None)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "cells": C, "particles": n, "D": D, "Kmax": cfg.Kmax,
                   "init": ("learned (network trained untimed on %d cells of the same generator, "
                            "init time included in every step; decode presence threshold %g)"
                            % (train_info["cells"], args.presence_logit)
                            if head == "learned" else "paper (random particles)"),
                   "precision": ("fp64 m-step (statistic sums, covariance, factor, inverse), fp64 "
                                 "convergence log-likelihood, fp64 final step; fp32 e-step"
                                 if args.mstep == "fp64" else
                                 "fp32 m-step, fp64 means and final step; fp32 e-step"),
                   "l2": "inputs > L2 and a 252 MB flush between timed steps",
                   "launch": ("CUDA-graph replay of init / compress / reconstruct" if not args.no_graph
                              else "direct calls"),
                   "em_shape": ({"threads_per_cell": cfg.threads_per_cell,
                                 "smem_particles": cfg.smem_particles, "autotune": tune}),
                   "em_shape_learned": ({"threads_per_cell": cfg_l.threads_per_cell,
                                         "smem_particles": cfg_l.smem_particles,
                                         "autotune_from_learned_start": tune_l}),
                   "parallelism": f"replicas x{world} (independent batches)"},
        "ms_init": hs["ms_init"], "ms_compress": hs["ms_compress"],
        "ms_reconstruct": hs["ms_reconstruct"],
        "cells_per_s": C * world / (step_ms * 1e-3),
        "paths": paths,
        "fit": {"Kbar": hs["Kbar"], "sweeps_mean": hs["sweeps_mean"],
                "maxsweeps_frac": hs["maxsweeps_frac"], "compression_ratio": hs["compression_ratio"],
                "proj_skipped_frac": float(np.mean((rst & 0x100) != 0))},
        "roofline": kernel_roofline(res[head]["kernels"], head_ctx(head)),
        "kernels": {k: dict(v, share=v["ms"] / max(1e-9, sum(z["ms"] for z in res[head]["kernels"].values())))
                    for k, v in sorted(res[head]["kernels"].items(), key=lambda kv: -kv[1]["ms"])},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
                "copies": "inputs in and outputs out on their own streams, overlapping the "
                          "neighbouring steps' compute (two device buffer sets)"},
        "gpu_launches": int(round(sum(v["launches_per_step"] for v in res[head]["kernels"].values())
                                  + (4 if head == "learned" else 0) + 2)) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the acceleration study of Sec. 4: standard EM, K-means, Anderson
# ---------------------------------------------------------------------------
# FP32 flops per particle, per component and per iteration of std_kernel,
# counted once for what the iteration needs: the exponent of one component
# (D = 1: difference, square, scale, offset; D = 3: difference, triangular
# whitening, sum of squares), the normaliser and the responsibility, and the
# moment sums (1 + D + D(D+1)/2 fused multiply-adds).
STD_FLOPS_PER_PKI = {1: 14, 3: 46}
# DRAM bytes of one std_kernel launch (K-means + AA5) per particle: None,
# because the kernel's output step changed after its last ncu capture (1216
# cells of the 1D-1V batch: 29.38 MB for 2434617 particles, the inputs read
# once); a new capture sets it again (a full launch is it times n)
STD_DRAM_BYTES_PER_PARTICLE = None
STD_MODES = (("random", 0, 0, False), ("kmeans", 1, 0, False), ("random+aa5", 0, 5, False),
             ("kmeans+aa5", 1, 5, False), ("penalised", 0, 0, True))


def mml_objective(K, params, lnL, counts, D):
    """eq. (lnL-GM) of each cell's output mixture: lnL - (d/2) ln N -
    (T/2) sum_k ln omega_k, d = K (T + 1) - 1 (cells with K > 0)"""
    T = D * (D + 3) / 2
    ok = K > 0
    w = np.where(np.arange(params.shape[1])[None, :] < K[:, None], params[:, :, 0], 1.0)
    pen = np.sum(np.log(np.maximum(w, 1e-300)), axis=1)
    d = K * (T + 1) - 1
    return np.where(ok, lnL - 0.5 * d * np.log(np.maximum(counts, 1)) - 0.5 * T * pen, 0.0)


def run_standard(args):
    """One step = gm_compress_standard (standard EM to tol, final FP64 EM
    step, charge deposit) of the whole batch, for each initialisation and
    acceleration of Sec. 4, and the simultaneous penalised EM beside the
    component-wise gm_compress; the headline is K-means + Anderson
    (memory 5)."""
    import torch
    import oracle
    rank, world, local = rank_info()
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_2007_12273_gb300 import build as gbuild
    from paper_2007_12273_gb300 import gm
    gbuild.build()
    gm.load()
    wl = make_workload(args.workload, 0)
    if args.cells:
        wl = sub_workload(wl, args.cells)
    D, C, n = wl.D, wl.C, wl.ntot
    cfg = gm.config(wl.params)
    counts = wl.counts().astype(np.float64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    cell_off, x, v, alpha = t(wl.cell_off), t(wl.x), t(wl.v), t(wl.alpha)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_mhz)

    clocks = ClockSampler(local)
    clocks.start()
    modes = {}
    outs = {}
    def time_calls(call):
        out = call(None)
        for _ in range(args.warmup):
            call(out)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            call(out)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return out, sum(a.elapsed_time(b) for a, b in evs) / args.steps

    for name, init, aa, pen in STD_MODES:
        out, ms = time_calls(lambda o_: gm.gm_compress_standard(
            cfg, cell_off, x, v, alpha, init=init, aa_memory=aa, penalised=pen, stream=stream, out=o_))
        o = {k: out[k].cpu().numpy() for k in ("K", "iters", "status", "lnL", "aa_steps", "km_passes",
                                                "params")}
        outs[name] = o
        flops = float(np.sum(counts * o["K"] * o["iters"])) * STD_FLOPS_PER_PKI[D]
        tf = flops / (ms * 1e-3) / 1e12
        modes[name] = {"ms": ms, "value": n / (ms * 1e-3), "iters_mean": float(o["iters"].mean()),
                       "iters_p90": float(np.percentile(o["iters"], 90)),
                       "converged_frac": float(np.mean((o["status"] & 1) == 0)),
                       "Kbar": float(o["K"].mean()), "lnL_mean": float(o["lnL"].mean()),
                       "mml_objective_mean": float(np.mean(mml_objective(o["K"], o["params"], o["lnL"],
                                                                         counts, D))),
                       "aa_steps_mean": float(o["aa_steps"].mean()),
                       "kmeans_passes_mean": float(o["km_passes"].mean()),
                       "tflops": tf, "frac_fp32_peak": tf / peak}
    # the component-wise adaptive EM (gm_compress, default launch shape) on
    # the same batch, beside its simultaneous variant
    out, ms = time_calls(lambda o_: gm.gm_compress(cfg, cell_off, x, v, alpha, stream=stream, out=o_))
    o = {k: out[k].cpu().numpy() for k in ("K", "sweeps", "status", "lnL", "params")}
    modes["component-wise (gm_compress)"] = {
        "ms": ms, "value": n / (ms * 1e-3), "sweeps_mean": float(o["sweeps"].mean()),
        "converged_frac": float(np.mean((o["status"] & 1) == 0)), "Kbar": float(o["K"].mean()),
        "lnL_mean": float(o["lnL"].mean()),
        # gm_compress reports eq. (lnL-GM) itself, the penalised objective
        "mml_objective_mean": float(o["lnL"].mean())}
    clk = clocks.stop()
    head = "kmeans+aa5"
    hm = modes[head]
    Lp = outs["random"]["lnL"]
    for name in outs:
        Ln = outs[name]["lnL"]
        modes[name]["reaches_random_plain_L_1e-4"] = float(np.mean(Ln >= Lp - 1e-4 * np.abs(Lp)))

    # ---- end to end through the API with host buffers (headline mode) -------
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(wl.cell_off), pin(wl.x), pin(wl.v), pin(wl.alpha)]
    d_in = [h.to(device) for h in h_in]
    out = gm.gm_compress_standard(cfg, *d_in, init=1, aa_memory=5, stream=stream)
    h_out = {k: torch.empty(tuple(out[k].shape), dtype=out[k].dtype).pin_memory()
             for k in ("K", "params", "W", "rho_target")}
    h2d = sum(h.numel() * h.element_size() for h in h_in)
    d2h = sum(h.numel() * h.element_size() for h in h_out.values())

    def e2e_step():
        for h, d in zip(h_in, d_in):
            d.copy_(h, non_blocking=True)
        gm.gm_compress_standard(cfg, *d_in, init=1, aa_memory=5, stream=stream, out=out)
        for k, h in h_out.items():
            h.copy_(out[k], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, min(args.steps, 5))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    result = {
        "metric": "standard EM (K-means + Anderson) particles/s on GB300", "value": hm["value"],
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": hm["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "cells": C, "particles": n, "D": D, "Kmax": cfg.Kmax,
                   "mode": "K = Kmax components, K-means init, Anderson memory 5, tol 1e-6",
                   "l2": "inputs > L2 and a 252 MB flush between timed steps",
                   "launch": "direct calls"},
        "modes": modes,
        "roofline": {"kernel": "std_kernel (gm_compress_standard)", "bound": "alu",
                     "achieved": hm["tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": hm["frac_fp32_peak"],
                     "traffic": (STD_DRAM_BYTES_PER_PARTICLE * n
                                 if STD_DRAM_BYTES_PER_PARTICLE is not None and D == 1
                                 and wl.v.dtype == np.float32 else None),
                     "note": f"FP32 flops = sum_j N_j * K_j * iters_j * {STD_FLOPS_PER_PKI[D]}; peak = "
                             f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"},
        "e2e": {"value": n / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        oracle.build()
        cores = os.cpu_count() or 1
        ncells = max(cores, 4)
        while True:
            sw = sub_workload(wl, ncells)
            t0 = time.perf_counter()
            oracle.standard(sw.params, sw.cell_off, sw.x, sw.v, sw.alpha, init=1, aa_memory=5,
                            nthreads=cores)
            dt = time.perf_counter() - t0
            if dt >= args.cpu_budget / 3 or ncells >= C:
                break
            ncells = min(C, ncells * max(2, int(args.cpu_budget / max(dt, 1e-3) / 1.5)))
        result["cpu_baseline"] = {"value": sw.ntot / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"first {sw.C} cells ({sw.ntot} particles), K-means + AA5, "
                                            f"OpenMP over cells, {dt:.1f} s"}
    print(json.dumps(result), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the 2D mesh: the paper's Weibel geometry tiled to fill a GPU
# ---------------------------------------------------------------------------
MESH2D_MAX_ITER = 64  # the library's cap on the 2D solve's iterations
MESH2D_DESC = ("weibel_2d3v: 128 x 128 cells x 512 particles (8.4 M), doubly periodic 80 x 80 "
               "(dx = 0.625, the paper's 10/16), v_th,x = 0.1, v_th,y,z = 0.3 x U[0.8, 1], FP32 v, "
               "Kmax = 8, S2 x S2 shape, tol 1e-6, N' = N per cell")


def run_mesh2d(args):
    """One step = gm_compress (plain EM, no 1D deposit) + gm_deposit_2d (the
    target rho') + gm_reconstruct_2d of the whole mesh, replayed from CUDA
    graphs; particles/s = N / step time."""
    import torch
    import oracle
    rank, world, local = rank_info()
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_2007_12273_gb300 import build as gbuild
    from paper_2007_12273_gb300 import gm
    gbuild.build()
    gm.load()
    side = 128 if not args.cells else int(round(math.sqrt(args.cells)))
    wl = workloads.weibel_2d3v(Cx=side, Cy=side, ppc=512, Lx=side * 0.625, Ly=side * 0.625,
                               seed=rank_seed(rank))
    p = dict(wl.params)
    cfg = gm.config(p)
    rcfg = gm.config(p, seed_key="recon_seed")
    mesh = gm.mesh2d(p)
    C, n, D = wl.C, wl.ntot, wl.D
    counts = wl.counts()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    off, x, y, v, a = t(wl.cell_off), t(wl.x), t(wl.y), t(wl.v), t(wl.alpha)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    trial_ms = gm.gm_autotune(cfg, off, x, v, a, stream=stream)
    rcfg.threads_per_cell, rcfg.smem_particles = cfg.threads_per_cell, cfg.smem_particles
    fit = gm.gm_compress(cfg, off, None, v, a, stream=stream)
    rho_t = gm.gm_deposit_2d(cfg, mesh, off, x, y, a, stream=stream)
    rec = gm.gm_reconstruct_2d(rcfg, mesh, fit["K"], fit["params"], fit["W"], rho_t, off, n_out=n,
                               stream=stream)
    torch.cuda.synchronize()
    graphs = []
    for fn in (lambda: gm.gm_compress(cfg, off, None, v, a, stream=stream, out=fit),
               lambda: gm.gm_deposit_2d(cfg, mesh, off, x, y, a, stream=stream, out=rho_t),
               lambda: gm.gm_reconstruct_2d(rcfg, mesh, fit["K"], fit["params"], fit["W"], rho_t, off,
                                            n_out=n, stream=stream, out=rec)):
        g_ = gm.Graph(stream)
        with g_:
            fn()
        graphs.append(g_)

    def step(ev=None):
        for k, g_ in enumerate(graphs):
            if ev:
                ev[k].record(stream)
            g_.launch(stream)
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        step(evs[i])
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = [sum(e[k].elapsed_time(e[k + 1]) for e in evs) / args.steps for k in range(3)]
    step_ms = sum(ms)
    for g_ in graphs:
        g_.close()
    st = rec["status"].cpu().numpy()
    kwork = fit["kwork"].cpu().numpy()
    K = fit["K"].cpu().numpy()
    sweeps = fit["sweeps"].cpu().numpy()
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_mhz)
    em_tf = em_flops(counts, kwork, D) / (ms[0] * 1e-3) / 1e12

    # end to end through the API with host buffers
    pin = lambda z: torch.from_numpy(np.ascontiguousarray(z)).pin_memory()
    h_in = [pin(wl.cell_off), pin(wl.x), pin(wl.y), pin(wl.v), pin(wl.alpha)]
    d_in = [h.to(device) for h in h_in]
    h_out = {k: torch.empty(tuple(rec[k].shape), dtype=rec[k].dtype).pin_memory()
             for k in ("x", "y", "v", "alpha", "status")}
    h2d = sum(h.numel() * h.element_size() for h in h_in)
    d2h = sum(h.numel() * h.element_size() for h in h_out.values())

    def e2e_step():
        for h, d in zip(h_in, d_in):
            d.copy_(h, non_blocking=True)
        gm.gm_compress(cfg, d_in[0], None, d_in[3], d_in[4], stream=stream, out=fit)
        gm.gm_deposit_2d(cfg, mesh, d_in[0], d_in[1], d_in[2], d_in[4], stream=stream, out=rho_t)
        gm.gm_reconstruct_2d(rcfg, mesh, fit["K"], fit["params"], fit["W"], rho_t, d_in[0], n_out=n,
                             stream=stream, out=rec)
        for k, h in h_out.items():
            h.copy_(rec[k], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, min(args.steps, 5))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    result = {
        "metric": "GM CR particles/s on a 2D mesh (compress + target deposit + reconstruct) on GB300",
        "value": n / (step_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": MESH2D_DESC if not args.cells else f"weibel_2d3v {side} x {side} x 512",
                   "cells": C, "particles": n, "init": "paper (random particles)",
                   "l2": "inputs > L2 and a 252 MB flush between timed steps",
                   "launch": "CUDA-graph replay of compress / deposit / reconstruct",
                   "em_shape": {"threads_per_cell": cfg.threads_per_cell,
                                "smem_particles": cfg.smem_particles,
                                "trial_ms": [round(z, 4) for z in trial_ms]}},
        "ms_compress": ms[0], "ms_deposit_2d": ms[1], "ms_reconstruct_2d": ms[2],
        "fit": {"Kbar": float(K.mean()), "sweeps_mean": float(sweeps.mean()),
                "mm_not_converged_cells": int(np.sum((st & 0x1000) != 0)),
                "proj_skipped_frac": float(np.mean((st & 0x100) != 0))},
        "roofline": {"kernel": "em_kernel (gm_compress)", "bound": "alu", "achieved": em_tf,
                     "peak": peak, "unit": "TFLOP/s", "frac": em_tf / peak, "traffic": None,
                     "note": f"FP32 flops = sum_j N_j * kwork_j * {FLOPS_PER_PK[D]}; peak = 152 SMs "
                             f"x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                     "secondary": em_secondary_rooflines(counts, K, kwork, sweeps, D, ms[0] * 1e-3,
                                                         sm_mhz)},
        "e2e": {"value": n / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        # em_kernel; 2 deposit kernels; reconstruct: stats, factors, assemble,
        # 3 per solve iteration (no-ops once converged), the last residual,
        # finish, emit
        "gpu_launches": (1 + 2 + 3 + 3 * MESH2D_MAX_ITER + 3) * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        sw = workloads.weibel_2d3v(Cx=16, Cy=16, ppc=512, seed=rank_seed(rank))
        sp = dict(sw.params)
        cores = os.cpu_count() or 1
        oracle.build()
        t0 = time.perf_counter()
        o = oracle.compress(sp, sw.cell_off, sw.x, sw.v, sw.alpha, nthreads=cores)
        rt = oracle.deposit2d(sp, sw.cell_off, sw.x, sw.y, sw.alpha)
        oracle.reconstruct2d(sp, o["K"], o["params"], o["W"], rt, sw.cell_off, nthreads=cores)
        dt = time.perf_counter() - t0
        result["cpu_baseline"] = {"value": sw.ntot / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"the paper's 16 x 16 mesh x 512 particles ({sw.ntot}), "
                                            f"compress + deposit + reconstruct (dense solve), {dt:.1f} s"}
    print(json.dumps(result), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the learned initialisation's own evaluation: train on cells of the 1D-1V
# batch's generator lifted to 3V and of the 1D-3V generator, evaluate on
# held-out 1D-3V cells against plain EM
# ---------------------------------------------------------------------------
C4_DESC = ("learned init, 1D-3V: network trained on cells fitted by plain EM, half from the 1D-1V "
           "mixture generator lifted to 3V (isotropic y, z), half from the 2048 x 4000 bi-Maxwellian "
           "generator; inference + EM on held-out bi-Maxwellian cells (4000 particles each, seed + 1000) "
           "against plain EM on the eq. (lnL-GM) objective and the sweep count")


def run_c4(args):
    """The learned initialisation evaluated as its own configuration:
    training cells from two generator families, evaluation cells held out;
    reports per-cell objective and sweeps of the learned start against
    plain EM, and both paths' compress throughput."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_2007_12273_gb300 import build as gbuild
    from paper_2007_12273_gb300 import gm, learned
    gbuild.build()
    gm.load()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    train_cells = args.train_cells or 200704
    eval_cells = args.cells or 65536
    # ---- training set (untimed) -------------------------------------------
    t0 = time.perf_counter()
    feats, Ts, Mks = [], [], []
    nchunk = max(2, train_cells // 4096)
    calib = None
    cfg = None
    for ch in range(nchunk):
        seed = workloads.GEN_SEED_BASE + 50000 + ch
        if ch % 2 == 0:
            tw = workloads.mixture_lifted_3v(C=4096, seed=seed)
        else:
            tw = workloads.bimaxwellian_1d3v(C=4096, ppc=4000, seed=seed)
        if cfg is None:
            cfg = gm.config(tw.params)
        dev_tw = (t(tw.cell_off), t(tw.x), t(tw.v), t(tw.alpha))
        f_, T_, M_, fit_ = learned.fit_targets(cfg, *dev_tw)
        feats.append(f_)
        Ts.append(T_)
        Mks.append(M_)
        if ch % 2 == 1:
            calib = (dev_tw, fit_["lnL"].clone())
        del dev_tw
    feat, T, Mk = torch.cat(feats), torch.cat(Ts), torch.cat(Mks)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    net = gm.Net(3, cfg.Kmax)
    net.init_weights(seed=1)
    hist = learned.train(net, feat, T, Mk, epochs=args.epochs, batch=1024, lr=1e-3)
    thr, calib_info = learned.calibrate_presence(net, cfg, *calib[0], calib[1])
    if args.presence_logit is not None:
        thr = args.presence_logit
    del feat, T, Mk, feats, Ts, Mks, calib
    # ---- held-out evaluation cells -------------------------------------------
    ew = workloads.bimaxwellian_1d3v(C=eval_cells, ppc=4000, seed=workloads.GEN_SEED_BASE + 2 + 1000)
    off, x, v, a = t(ew.cell_off), t(ew.x), t(ew.v), t(ew.alpha)
    ecfg = gm.config(ew.params)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)

    def timed(fn, steps):
        out = fn(None)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            fn(out)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return out, sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps

    clocks = ClockSampler(0)
    clocks.start()
    plain, ms_plain = timed(lambda o: gm.gm_compress(ecfg, off, x, v, a, stream=stream, out=o), args.steps)
    bufs = {}

    def learned_step(o):
        f_, w_ = gm.gm_features(ecfg, off, v, a, stream=stream, out=bufs.get("f"))
        bufs["f"] = (f_, w_)
        y_ = net.forward(f_, out=bufs.get("y"), stream=stream)
        bufs["y"] = y_
        K0, prm = gm.gm_mlp_decode(ecfg, y_, w_, off, stream=stream, presence_logit=thr, dest=bufs.get("d"))
        bufs["d"] = (K0, prm)
        return gm.gm_compress(ecfg, off, x, v, a, stream=stream, out=o, init_K=K0, init_params=prm)

    lrn, ms_learned = timed(learned_step, args.steps)
    clk = clocks.stop()
    n = ew.ntot
    Lp, Ll = plain["lnL"].cpu().numpy(), lrn["lnL"].cpu().numpy()
    Kp, Kl = plain["K"].cpu().numpy(), lrn["K"].cpu().numpy()
    K0 = bufs["d"][0].cpu().numpy()
    sp, sl = plain["sweeps"].cpu().numpy(), lrn["sweeps"].cpu().numpy()
    reach = Ll >= Lp - 1e-4 * np.abs(Lp)
    cfg2 = gm.config(dict(ew.params, seed=int(ew.params.get("seed", 1)) + 1000))
    L2 = gm.gm_compress(cfg2, off, x, v, a, stream=stream)["lnL"].cpu().numpy()
    short = ~reach
    result = {
        "metric": "c4: learned-init vs plain EM, compress particles/s on held-out 1D-3V cells",
        "value": n / (ms_learned * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": 1, "ms_per_step": ms_learned, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": C4_DESC, "train_cells": int(nchunk * 4096), "eval_cells": eval_cells,
                   "eval_particles": n, "presence_threshold": thr,
                   "l2": "inputs > L2 and a 252 MB flush between timed steps", "launch": "direct calls"},
        "training": {"fit_seconds": t_fit, "train_seconds": hist["seconds"], "epochs": args.epochs,
                     "adam_steps": hist["steps"], "loss_first": hist["loss"][0], "loss_last": hist["loss"][-1],
                     "presence_calibration": calib_info},
        "plain": {"value": n / (ms_plain * 1e-3), "ms": ms_plain, "sweeps_mean": float(sp.mean()),
                  "Kbar": float(Kp.mean()), "maxsweeps_frac": float(np.mean((plain["status"].cpu().numpy() & 1) != 0))},
        "learned": {"value": n / (ms_learned * 1e-3), "ms": ms_learned, "sweeps_mean": float(sl.mean()),
                    "Kbar": float(Kl.mean()), "K0bar": float(K0.mean()),
                    "maxsweeps_frac": float(np.mean((lrn["status"].cpu().numpy() & 1) != 0))},
        "objective": {"reaches_plain_L_1e-4": float(reach.mean()),
                      "mean_lnL_minus_plain": float(np.mean(Ll - Lp)),
                      "median_rel_shortfall": float(np.median(((Lp - Ll) / np.abs(Lp))[short])) if short.any() else 0.0,
                      "short_cells_with_K_below_plain": float(np.mean(Kl[short] < Kp[short])) if short.any() else 0.0,
                      "short_cells_with_K0_below_plain": float(np.mean(K0[short] < Kp[short])) if short.any() else 0.0,
                      "other_seed_reaches_plain_L_1e-4": float(np.mean(L2 >= Lp - 1e-4 * np.abs(Lp)))},
        "gpu_launches": 8 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(result), flush=True)
    return 0


def run_gemm(args):
    """The tcgen05 BF16 GEMM on its own: C = relu(A B^T + bias) with A
    [M, K], B [N, K], BF16 output, at the network's first-layer shape
    (K = 576, N = 256) and M = 65536 rows, and the four layers of the
    forward pass on M = 262144 rows.  CUDA events per launch, L2 flushed
    between launches."""
    import torch
    from paper_2007_12273_gb300 import gm
    torch.manual_seed(0)
    dev_ = torch.device("cuda")
    peaks = measured_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    flush = torch.empty(252 << 20 >> 2, dtype=torch.float32, device=dev_)
    stream = torch.cuda.current_stream()

    def time_gemm(M, N, K):
        A = torch.randn(M, K, device=dev_).to(torch.bfloat16)
        B = torch.randn(N, K, device=dev_).to(torch.bfloat16)
        bias = torch.randn(N, device=dev_)
        out = torch.empty(M, N, dtype=torch.bfloat16, device=dev_)
        for _ in range(max(3, args.warmup)):
            gm.gm_gemm_bf16(A, B, bias=bias, relu=True, out_bf16=out)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            gm.gm_gemm_bf16(A, B, bias=bias, relu=True, out_bf16=out)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / args.steps
        return ms, 2.0 * M * N * K / (ms * 1e-3) / 1e12

    clocks = ClockSampler(0)
    clocks.start()
    ms, tf = time_gemm(65536, 256, 576)
    layers = [time_gemm(262144, n, k) for n, k in ((256, 576), (256, 256), (256, 256), (112, 256))]
    clk = clocks.stop()
    fwd_ms = sum(l[0] for l in layers)
    fwd_flops = 2.0 * 262144 * (576 * 256 + 2 * 256 * 256 + 256 * 112)
    result = {
        "metric": "tcgen05 BF16 GEMM TFLOP/s (M = 65536, N = 256, K = 576, bias + ReLU, BF16 out)",
        "value": tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "one GEMM launch of the network's first-layer shape; the four layers of the "
                               "forward pass on 262144 rows",
                   "l2": "a 252 MB flush between timed launches", "launch": "direct calls"},
        "roofline": {"kernel": "tc_gemm_kernel", "bound": "tensor", "achieved": tf, "peak": bf16,
                     "unit": "TFLOP/s", "frac": tf / bf16, "traffic": None,
                     "note": "dense BF16 flops 2 M N K; peak = measured cuBLAS BF16 burst"},
        "forward_262144_rows": {"ms": fwd_ms, "tflops": fwd_flops / (fwd_ms * 1e-3) / 1e12,
                                "layers_ms": [l[0] for l in layers]},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    print(json.dumps(result), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmcr", choices=["gmcr", "reference"])
    ap.add_argument("--workload", default="lognormal_1d3v")
    ap.add_argument("--mstep", default="fp64", choices=["fp64", "fp32"],
                    help="fp64: FP64 M-step (statistic sums, covariance, factor, inverse) and the "
                         "corrected convergence test (the library default); fp32: FP32 M-step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=60.0,
                    help="--impl reference: seconds of oracle work over warmup + steps")
    ap.add_argument("--cells", type=int, default=0, help="use only the first N cells (profiling)")
    ap.add_argument("--threads-per-cell", type=int, default=0)
    ap.add_argument("--init", default="both", choices=["plain", "learned", "both"])
    ap.add_argument("--train-cells", type=int, default=0,
                    help="training cells of the learned initialisation (default 65536 for 1V, "
                         "32768 for 3V)")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--save-net", default="", help="save the trained network (.npz)")
    ap.add_argument("--load-net", default="", help="use a saved network instead of training")
    ap.add_argument("--smem-particles", type=int, default=0)
    ap.add_argument("--no-graph", action="store_true", help="time direct calls instead of graph replay")
    ap.add_argument("--presence-logit", type=float, default=None,
                    help="learned init: decode slots whose presence logit exceeds this "
                         "(default: calibrated on a training chunk)")
    ap.add_argument("--mesh2d", action="store_true",
                    help="the 2D-mesh pipeline (compress, target deposit, 2D reconstruct; one GPU)")
    ap.add_argument("--standard", action="store_true",
                    help="the acceleration study: standard EM with random or K-means start, "
                         "with or without Anderson acceleration (one GPU)")
    ap.add_argument("--c4", action="store_true",
                    help="the learned initialisation's evaluation: train on 200704 cells of two "
                         "generator families, evaluate on 65536 held-out 1D-3V cells (one GPU)")
    ap.add_argument("--gemm", action="store_true",
                    help="the tcgen05 BF16 GEMM on its own (M = 65536, N = 256, K = 576) and the "
                         "network's four layers on 262144 rows")
    args = ap.parse_args(argv)
    if args.gemm and args.impl != "reference":
        return run_gemm(args)
    if args.c4 and args.impl != "reference":
        if args.epochs == 60 and not any(a.startswith("--epochs") for a in (argv or sys.argv[1:])):
            args.epochs = 20
        return run_c4(args)
    if args.standard and args.impl != "reference":
        return run_standard(args)
    if args.mesh2d and args.impl != "reference":
        return run_mesh2d(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gmcr(args)


if __name__ == "__main__":
    sys.exit(main())
