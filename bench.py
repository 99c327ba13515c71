"""Benchmark: Poisson solves/s of the variable-density pressure solve on one GB300.

One step = one complete solve (all phases: rhs mean removal, inner iterations with FP64
refinement, gauge) of the 512^3 periodic hot-spot workload: rho = T0/T with 200k Gaussian hot
spots (density ratio capped at 10), rhs = divergence of a random low-k velocity field, in mixed
precision (FP32 inner arithmetic inside FP64 iterative refinement) to relative residual 1e-8, by
the paper's own iteration (Sec. 3.4, Eq. (Pois)): the residual is multiplied by rho and inverted
with the constant-coefficient FFT Laplacian, p += that update.  Inputs are resident in HBM when
timing starts; the working set (~15 GB) is far larger than L2.  Beside it, on the same input and
to the same tolerance, the plain FP64 solve (``fp64_1e-8``; their ratio is ``mixed_over_fp64``).
The JSON line also carries the end-to-end number through the C ABI with host buffers, per-kernel
timings and the roofline of the dominant kernel, the 256^3 FP64 workload (to 1e-10, and every
method at 1e-8 in FP64, mixed and BF16-coefficient precision), the 64-grid batch, the serving
stream and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  torchrun --nproc-per-node N bench.py --gpus N ...   (N independent replicas, weak scaling)
  python bench.py --workload c1 | --workload grid --grid 192 --precision fp64   (profiling cases)
"""
from __future__ import annotations

import argparse
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

METRIC = "Poisson solves/s and % HBM roofline to 1e-8 rel. residual, mixed vs FP64"
WORKLOAD_C2 = ("512^3 periodic box L=2pi, rho=T0/T (200k hot spots, density ratio capped at 10), rhs=div of "
               "random |k|<=4 velocity; mixed (FP32 inner, FP64 refinement), relative residual 1e-8")
WORKLOAD_C1 = ("256^3 periodic box L=2pi, rho=T0/T (20k hot spots, density ratio 4), rhs=div of random "
               "|k|<=4 velocity; FP64, relative residual 1e-10")
METHOD_FP = ("the paper's fixed-point iteration (Sec. 3.4, Eq. (Pois)): update = constant-coefficient FFT "
             "inverse of rho * residual; the residual recurs in the inner precision between FP64 residuals")
PRECONDS = {"spectral": 2, "cheb": 1, "jacobi": 0, "mg": 3}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 vector peak from the unit counts: GB300 issues 2 FP64 FMA per clock per SM, so
# 152 SMs x 2 x 2 flop x 2.07 GHz = 1.259 TFLOP/s.  The line divides by the figure the library's
# FP64 FMA probe (vdp_probe_fp64) measures on the same GPU, and reports both.
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_BYTES = 129e6

# Algorithmic bytes and flops per cell of one launch of each sweep kind (inner type T bytes,
# coefficient type B bytes; the BF16 ablation also reads a per-cell diagonal correction):
#   stencil: read rt (or z), d_old, 3 coefficients; write d, q           -> 4T + 3B (+B)
#            d = z + beta d_old (1 FMA), q = d - sum_6 b d_nb (6 FMA), <d,q> (1 FMA) -> 16 flop
#            FP64 form (q = At z + beta q_old): also reads q_old -> 5T + 3B; 9 FMA -> 18 flop
#   fixed-point sweep (the paper's iteration; stencil and update in one pass): read z (FP32),
#            3 coefficients, rt, x; write rt, x                          -> 4 + 4T + 3B (+B)
#            rt -= At z: 6 FMA, x += z: 1 add, rt - q: 1 add; FP64 <rt,rt> is summed in FP32
#                                                                        -> 14 flop, 8 FP64 pipe ops
#   update : read x, d, q, rt; write x, rt                                -> 6T;  3 FMA -> 6 flop
#   res64  : read p, f - <f> (stored), sinv, D, 3 FP64 coefficients; write rt -> 56 + T
#            r = (f - <f>) + D p - sum of 6 b p_nb: 7 FMA (+ the FP64 inner's scaling multiply)
#                                                                          -> 14 flop (15), 7 FP64 ops (8)
#            the first residual of a solve from p = 0 is f - <f>: read f, sinv; write f - <f>, rt
#            -> 24 + T; FP64 inner: subtraction, scaling, |r|^2, |rt|^2 in FP64 -> 6 flop, 4 FP64
#            ops; FP32 inner: subtraction and |r|^2 in FP64, scaling and |rt|^2 in FP32 -> 3 flop
#   cheb   : sweep 1 reads rt and 3 coefficients, writes z, dz           -> 3T + 3B (+B)
#            later sweeps also read z and dz                              -> 5T + 3B (+B); 18 flop
#   other  : rhs mean removal, refinement correction, gauge: not in the roofline
#   spectral passes, S = bytes of the half spectrum per cell (8 (nx/2 + pad) / nx):
#   spec_x : X+ reads rt, W, writes S; X- reads S, W, rt, writes z   -> (3T + 8 + 2S) / 2 per launch
#   spec_y : read and write S                                        -> 2S
#   spec_z : read and write S (forward FFT, division, inverse FFT)   -> 2S
#   When the half spectrum fits in L2 (256^3: 71 MB) the S bytes never reach HBM: the HBM bytes
#   of a spectral pass are then only its rt / W / z traffic, and Y and Z have none (their roof
#   is the L2 bandwidth, reported as plain GB/s without an HBM fraction).
SIZES = {"fp64": (8, 8, False), "mixed": (4, 4, False), "mixed_bf16": (4, 2, True)}
KERNEL_NAMES = {"res64": "k_res64_direct", "stencil": "k_stencil_direct", "cheb": "k_stencil_direct",
                "update": "k_flat", "other": "k_flat", "spec_x": "k_spec_x_fwd(_persistent) / k_spec_x_inv_persistent",
                "spec_y": "k_spec_y", "spec_z": "k_spec_z",
                "mg": "k_mg_down / k_mg_restrict / k_mg_coarse / k_mg_prolong / k_mg_up"}
FP64_PIPE_OPS = {"stencil_fixed": 8.0, "res64": 8.0, "res64_first": 4.0}  # FP64 inner type


def fixed_inner_tol(workload: str, prec: str) -> float:
    """Least relative reduction per inner solve of the mixed fixed-point solve (vdp_opts.inner_tol).

    The paper's iteration reduces the residual by about 0.18 per iteration on the 512^3 input
    whatever the precision, so it needs 12 iterations to 1e-8; the inner target only decides how
    many FP64 residuals (and corrections) the mixed solve spends on the way.  Measured at 512^3
    (FP32 inner): 1e-4 -> 12 iterations and 4 FP64 residuals (31.7 ms); 5e-5 and 3e-5 -> 12 and 3
    (29.3 ms, final residual 9.2e-9); 2e-5 -> 13 and 3; 1e-5 -> 14 and 3 (the first inner solve,
    from the largest residual, stalls near FP32 rounding).  With BF16 coefficients 1e-4 is best
    (19 iterations against 21 at 5e-5).  Elsewhere the library default 1e-4."""
    if workload == "c2" and prec == "mixed":
        return 4e-5
    return 1e-4


def spectrum_bytes(nx: int) -> float:
    """Bytes of the half spectrum per cell (row pitch padded to 8 complex values)."""
    nxp = ((nx // 2 + 1 + 7) // 8) * 8
    return 8.0 * nxp / nx


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# kernel at this precision and grid (192^3 captures, fixed-point method, FP64), keyed (precision,
# sweep, grid, fixed-point); 256^3 entries scale by the cell count 256^3 / 192^3.  A changed
# kernel drops its entries until it is re-captured, and the residual is left out (the capture
# holds the residual from p = 0 only, the table averages both kinds).
_SCALE_256 = (256 / 192) ** 3
_TRAFFIC_192 = {("fp64", "stencil", True): 317.8e6 + 85.3e6}
TRAFFIC = {(p, k, 192, f): v for (p, k, f), v in _TRAFFIC_192.items()}
TRAFFIC.update({(p, k, 256, f): v * _SCALE_256 for (p, k, f), v in _TRAFFIC_192.items()})
# the fused FP32 sweep of the mixed fixed-point solve: captured at 256^3 (a launch with x read and
# written), scaled to 512^3 by the cell count
TRAFFIC[("mixed", "stencil", 256, True)] = 343.2e6 + 107.0e6
TRAFFIC[("mixed", "stencil", 512, True)] = (343.2e6 + 107.0e6) * 8


def spec_bytes(prec: str, kind: str, nx: int, ncell: int, slabbed: bool, fixed: bool):
    """(operand bytes, HBM bytes) per cell of the spectral passes of kind spec_x (X+ and X-),
    spec_y (Y+ and Y-) or spec_z over one application.  X+ reads rt (T) and its weight (4) and
    writes the half spectrum (S per cell); Y+ / Y- read and write it; Z reads and writes it; X-
    reads it and its weight (4) and writes z (4 for the fixed-point iteration, else T).  When the
    whole spectrum fits in L2 (256^3: 71 MB) no S byte reaches HBM; when the passes run slab by
    slab (512^3) X+ hands its slab to Y+ and Y- to X- through L2, so only Y+'s write and Y-'s
    read of S reach HBM."""
    T = SIZES[prec][0]
    zT = 4 if fixed else T
    S = spectrum_bytes(nx)
    whole_l2 = S * ncell <= 0.6 * L2_BYTES
    if kind == "spec_x":
        alg = T + 4 + S + S + 4 + zT
        hbm = T + 4 + 4 + zT + (0 if (whole_l2 or slabbed) else 2 * S)
    elif kind == "spec_y":
        alg = 4 * S
        hbm = 0 if whole_l2 else (2 * S if slabbed else 4 * S)
    else:
        alg = 2 * S
        hbm = 0 if whole_l2 else 2 * S
    return alg, hbm


def sweep_cost(prec: str, kind: str, cheb_k: int = 1, nx: int = 256, fixed: bool = False, ncell: int = 0):
    """(bytes, flops, hbm_bytes) per cell of one launch of sweep `kind`, or None (the spectral
    passes: see spec_bytes, per application)."""
    T, B, diag = SIZES[prec]
    Bd = B if diag else 0
    if fixed and kind == "stencil":
        b = 4 + 4 * T + 3 * B + Bd
        return b, 14.0 + (2.0 if diag else 0.0), b
    if kind == "mg":  # one V-cycle: level 0 down 24 B, restriction 4.5, prolongation 12, up 24
        # (FP32 rt, bt, W, t, z), the coarser levels 68.5 B per cell x 1/7 of the fine cells; an
        # FP64 solve adds the rounding of rt (12 B) and its FP64 z (4 B)
        b = 64.5 + 68.5 / 7.0 + (16.0 if prec == "fp64" else 0.0)
        return b, 0.0, b
    if kind == "stencil":
        if prec == "fp64":
            return 5 * T + 3 * B, 18.0, 5 * T + 3 * B
        b = 4 * T + 3 * B + Bd
        return b, 16.0 + (2.0 if diag else 0.0), b
    if kind == "update":
        return 6 * T, 6.0, 6 * T
    if kind == "res64":
        f64 = prec == "fp64"
        return 56 + T, 15.0 if f64 else 14.0, 56 + T
    if kind == "res64_first":
        f64 = prec == "fp64"
        return 24 + T, 6.0 if f64 else 3.0, 24 + T
    if kind == "cheb":
        k = max(cheb_k - 1, 1)
        b = ((3 * T + 3 * B + Bd) + (k - 1) * (5 * T + 3 * B + Bd)) / k
        return b, 18.0, b
    return None


def algorithmic(prec: str, ncell: int, iters: int, outer: int, spectral: bool = False, nx: int = 256,
                fixed: bool = False, slabbed: bool = False):
    """Algorithmic HBM bytes of a whole solve (the roofline of the step as a whole)."""
    T = SIZES[prec][0]
    spec = sum(spec_bytes(prec, k, nx, ncell, slabbed, fixed)[1] for k in ("spec_x", "spec_y", "spec_z"))
    if fixed:  # per update: one application and the fused sweep
        per_iter = spec + sweep_cost(prec, "stencil", fixed=True)[2]
    else:
        per_iter = sweep_cost(prec, "stencil")[2] + sweep_cost(prec, "update")[2] + (spec if spectral else 0)
    res = sweep_cost(prec, "res64")[2] * max(outer - 1, 0) + sweep_cost(prec, "res64_first")[2]
    return (iters * per_iter + res + max(outer - 1, 0) * (24 + T) + 32) * ncell


def kernel_table(prec: str, ncell: int, kinds: dict, peaks: dict, grid: int, cheb_k: int = 1, nx: int = 256,
                 fixed: bool = False, slabbed: bool = False):
    """Per sweep kind: launches, mean/min duration (CUDA events around each launch), share of the
    summed kernel time, algorithmic GB/s (all operand bytes), the HBM fraction of the bytes that
    reach HBM, and for FP64 sweeps the FP64 TFLOP/s and its fraction of the measured FP64 peak.
    Spectral kinds are counted per application (their launches may be slabs)."""
    total = sum(k["ms"] for k in kinds.values()) or 1.0
    apps = max(kinds.get("spec_z", {}).get("launches", 0), 1)
    out = {}
    for name, k in kinds.items():
        if not k["launches"]:
            continue
        row = {"kernel": KERNEL_NAMES[name], "launches": k["launches"], "mean_us": 1e3 * k["ms_mean"],
               "min_us": 1e3 * k["ms_min"], "share": k["ms"] / total}
        t_all = k["ms"] / 1e3
        if name.startswith("spec_"):
            alg, hbm = spec_bytes(prec, name, nx, ncell, slabbed, fixed)
            row["us_per_application"] = 1e6 * t_all / apps
            row["alg_bytes_per_launch"] = alg * ncell * apps / k["launches"]
            row["gbs"] = alg * ncell * apps / t_all / 1e9
            if hbm > 0:
                row["hbm_alg_bytes_per_launch"] = hbm * ncell * apps / k["launches"]
                row["hbm_frac"] = hbm * ncell * apps / t_all / 1e9 / peaks["hbm_gbs"]
            else:
                row["bytes_in"] = "L2 (half spectrum resident): gbs is L2 traffic, no HBM fraction"
            row["tflops"] = 0.0
            row["traffic"] = None
            out[name] = row
            continue
        cost = sweep_cost(prec, name, cheb_k, nx, fixed, ncell)
        ops = FP64_PIPE_OPS.get("stencil_fixed" if (fixed and name == "stencil") else name)
        if name == "res64" and k["launches"] > 0:
            # every benchmarked solve starts from p = 0: one of its residual launches is the
            # short first one; the row averages over the launches (bytes, flops, FP64 ops)
            n, first = k["launches"], sweep_cost(prec, "res64_first")
            cost = tuple(((n - 1) * c + f) / n for c, f in zip(cost, first))
            ops = ((n - 1) * ops + FP64_PIPE_OPS["res64_first"]) / n
        if cost is not None:
            t = k["ms_mean"] / 1e3
            row["alg_bytes_per_launch"] = cost[0] * ncell
            row["gbs"] = cost[0] * ncell / t / 1e9
            row["hbm_alg_bytes_per_launch"] = cost[2] * ncell
            row["hbm_frac"] = cost[2] * ncell / t / 1e9 / peaks["hbm_gbs"]
            row["tflops"] = cost[1] * ncell / t / 1e12
            if prec == "fp64" and cost[1] > 0:
                row["fp64_flop_frac"] = row["tflops"] / peaks["fp64_tflops"]
                if ops:
                    row["fp64_issue_frac"] = ops * ncell / t / (peaks["fp64_tflops"] * 1e12 / 2.0)
            row["traffic"] = TRAFFIC.get((prec, name, grid, fixed))
        out[name] = row
    return out


def roofline(prec: str, table: dict, peaks: dict):
    """The roofline object of the dominant sweep kind (largest share of kernel time)."""
    name = max((n for n in table if "gbs" in table[n]), key=lambda n: table[n]["share"])
    row = table[name]
    hbm = row.get("hbm_alg_bytes_per_launch", 0.0)
    t_hbm = hbm / (peaks["hbm_gbs"] * 1e9)
    t_alu = row["tflops"] * row["mean_us"] * 1e-6 / peaks["fp64_tflops"] if prec == "fp64" else 0.0
    if t_alu > t_hbm:  # FP64 arithmetic needs more time than the bytes: the FP64 pipe bounds it
        roof = {"bound": "alu", "achieved": row["tflops"], "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                "frac": row["tflops"] / peaks["fp64_tflops"], "frac_basis": "FP64 flops (FMA = 2)",
                "issue_frac": row.get("fp64_issue_frac"), "peak_source": peaks["fp64_source"]}
    else:
        roof = {"bound": "hbm", "achieved": hbm / (row["mean_us"] * 1e-6) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": row["hbm_frac"], "frac_basis": "algorithmic HBM bytes per launch",
                "peak_source": peaks["source"]}
    roof.update({"traffic": row["traffic"], "kernel": row["kernel"], "sweep": name, "precision": prec,
                 "launches": row["launches"], "mean_us": row["mean_us"], "share": row["share"],
                 "alg_bytes_per_launch": hbm,
                 "timing": "CUDA events around each launch of an instrumented solve of the same workload "
                           "on the same stream and solver, after the timed region"})
    return roof


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        out = {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except Exception:
        out = dict(PEAKS_FALLBACK, source="fallback")
    out["fp64_tflops"] = FP64_PEAK_DERIVED_TFLOPS
    out["fp64_source"] = "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"
    return out


def measure_fp64_peak(vdp, peaks, stream):
    """Replace the derived FP64 peak by the library probe's measurement on this GPU."""
    try:
        t = vdp.vdp_probe_fp64(stream)
    except Exception as e:  # keep the derived figure, say why
        peaks["fp64_source"] += f" (probe failed: {e})"
        return
    peaks["fp64_tflops_derived"] = FP64_PEAK_DERIVED_TFLOPS
    peaks["fp64_tflops"] = t
    peaks["fp64_source"] = "measured: vdp_probe_fp64 (independent FP64 FMA chains, CUDA events)"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def wait_first(self, timeout: float = 10.0):
        """Block until the sampler has printed its first line (nvidia-smi's start-up, which
        initialises the driver in another process, then lies before the timed region)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time sets the whole job's); x itself when
    there is one rank.  device: where the reduction tensor lives (the GPU for NCCL)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, steps: int, elapsed: float) -> float:
    """Whole-job throughput of N replicas: every rank solves `steps` times (weak scaling)."""
    return world * steps / elapsed


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _golden_iterations(key: str) -> int:
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    with open(path) as fh:
        return int(json.load(fh)[key]["oracle_iterations"])


def cpu_baseline(prob, key: str, iters_per_sample: int = 12):
    """The CPU oracle (FP64 Jacobi-PCG, all host cores) on a bounded sample of the workload:
    `iters_per_sample` iterations of the solve, scaled to solves/s with the oracle's own iteration
    count to the workload's tolerance on this input (tests/golden/oracle_iterations.json)."""
    import oracle
    n_it = _golden_iterations(key)
    t0 = time.perf_counter()
    _, info = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=0.0, maxit=iters_per_sample)
    dt = time.perf_counter() - t0
    t_iter = dt / max(info["iters"], 1)
    nz, ny, nx = prob.shape
    return {"value": 1.0 / (t_iter * n_it), "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{info['iters']} FP64 Jacobi-PCG iterations of the {nx}^3 workload in {dt:.1f} s "
                      f"(incl. set-up), scaled by the oracle's {n_it} iterations to {prob.tol:g}",
            "sample_s": dt}


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle as the reference arm (rank 0 only).  Each step is a bounded
    sample (--ref-iters Jacobi-PCG iterations of the headline workload); ms_per_step is that
    sample's own wall time, value the solves/s it implies at the oracle's iteration count."""
    if rank != 0:
        return 0
    import vdp_inputs as V
    prob, key, workload = (V.config2(), "c2", WORKLOAD_C2) if args.workload == "c2" else (V.config1(), "c1",
                                                                                            WORKLOAD_C1)
    for _ in range(args.warmup):
        cpu_baseline(prob, key, iters_per_sample=1)
    vals, secs = [], []
    cb = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(prob, key, iters_per_sample=args.ref_iters)
        secs.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    v = statistics.median(vals)
    nz, ny, nx = prob.shape
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "grid": [nx, ny, nz], "tol": prob.tol,
                       "density_ratio": round(prob.info["ratio"], 4), "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"] + f"; each step one such sample (ms_per_step = its wall "
                                                      f"time), value = median of {args.steps}"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config3_all(count: int = 64):
    """The 64 batch instances, generated in a spawn pool (no fork after CUDA initialisation)."""
    import multiprocessing as mp
    import vdp_inputs as V
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(V.config3_instance, range(count))


def run_batch(torch, vdp, dev, probs, persistent=False, precond="fixed_point"):
    """The 64-grid batch: all instances in one batch, mixed precision to 1e-8, autotuned layouts."""
    from paper_1601_05448_gb300 import tune
    sizes = {}
    for pr in probs:
        sizes.setdefault(pr.shape, pr)
    for shape, pr in sizes.items():  # tune each distinct grid once (cached)
        nz, ny, nx = shape
        tune.tune(nx, ny, nz, pr.L, torch.from_numpy(pr.rho).to(dev), torch.from_numpy(pr.f).to(dev), "mixed",
                  iters=30, batchable=True)
    solvers, fs, ps = [], [], []
    for pr in probs:
        nz, ny, nx = pr.shape
        opts = dict(tune.cached_options(nx, ny, nz, "mixed", batchable=True) or {})
        if precond == "fixed_point":
            opts.update(method=vdp.VDP_METHOD_FIXED_POINT)
        else:
            opts["precond"] = PRECONDS[precond]
        s = vdp.Solver(nx, ny, nz, pr.L, precision="mixed", **opts)
        s.set_density(torch.from_numpy(pr.rho).to(dev))
        solvers.append(s)
        fs.append(torch.from_numpy(pr.f).to(dev))
        ps.append(torch.empty_like(fs[-1]))
    out = {}
    with vdp.Batch("mixed", persistent=persistent) as b:
        for rep in range(2):  # the first pass warms up (graph capture, caches)
            for s, f, p, pr in zip(solvers, fs, ps, probs):
                b.add(s, f, p, pr.tol)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            runs = 0
            while b.run(64) > 0:
                runs += 1
            torch.cuda.synchronize(dev)
            el = time.perf_counter() - t0
            stats = [s.stats() for s in solvers]
            for s in solvers:
                b.remove(s)
        ncell = sum(int(np.prod(pr.shape)) for pr in probs)
        dofit = sum(int(np.prod(pr.shape)) * st.iters for pr, st in zip(probs, stats))
        out = {"instances": len(probs), "total_cells": ncell, "seconds": el, "solves_per_s": len(probs) / el,
               "gdof_iter_per_s": dofit / el / 1e9, "persistent_launch": bool(persistent), "precond": precond,
               "iterations_total": sum(st.iters for st in stats), "runs": runs + 1,
               "all_ok": all(st.ok for st in stats), "max_rel_res": max(st.rel_res for st in stats),
               "sizes": sorted({pr.shape[0] for pr in probs}), "tuned_layouts": {str(k[0]): tune.cached_options(
                   k[2], k[1], k[0], "mixed", batchable=True) for k in sizes}}
    for s in solvers:
        s.close()
    return out


# one projection substep (App. A) around the solve: FP64 operations and bytes per cell of its two
# kernels (right side: 4 mul + 5 fma + 1 add, reads m x3, b x3, RHS^div, writes f; correction:
# 3 sub + 3 fma, reads p, m x3, writes m x3)
PROJ_COST = {"rhs": {"bytes": 64.0, "fp64_ops": 10.0}, "correct": {"bytes": 56.0, "fp64_ops": 6.0}}


def run_projection(torch, vdp, dev, solver, prob, stream, peaks, steps=5):
    """The steps either side of the solve (App. A): Poisson right side from seeded face momenta and
    a divergence target on the benchmark density, the benchmark solve, and the momentum correction
    of Eq. (mom).  The momenta are restored before every step (outside the events)."""
    import vdp_inputs as V
    rng = np.random.default_rng(7)
    m0 = [torch.from_numpy(x).to(dev) for x in V.face_momenta(prob.shape, prob.L, rng)]
    rd = torch.from_numpy(V.divergence_target(prob.shape, rng)).to(dev)
    m = [x.clone() for x in m0]
    pp = torch.zeros_like(rd)
    c = 0.5 * 1e-3  # C_pre[0] dt with dt = 1e-3
    ncell = rd.numel()

    def reset():
        for a, b in zip(m, m0):
            a.copy_(b)

    reset()
    solver.project(m, rd, c, prob.tol, pp)
    ms_steps, st = [], None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        reset()
        e0.record(stream)
        st = solver.project(m, rd, c, prob.tol, pp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_steps.append(e0.elapsed_time(e1))
    reset()
    st_t, kt = solver.project_timed(m, rd, c, prob.tol, pp)
    out = {"ms_per_step": statistics.median(ms_steps), "steps_per_s": 1e3 / statistics.median(ms_steps),
           "solve_ms": st.ms, "iters": st.iters, "rel_res": st.rel_res, "status": vdp.vdp_strerror(st.status),
           "chi": -c * st.rhs_mean, "c": c,
           "timing": "CUDA events around vdp_project per step (median of %d); kernels from vdp_project_timed"
                     % steps}
    for name, key in (("rhs", "rhs_ms"), ("correct", "correct_ms")):
        t = kt[key] / 1e3
        cost = PROJ_COST[name]
        out[name] = {"us": kt[key] * 1e3, "alg_bytes": cost["bytes"] * ncell,
                     "gbs": cost["bytes"] * ncell / t / 1e9,
                     "hbm_frac": cost["bytes"] * ncell / t / 1e9 / peaks["hbm_gbs"],
                     "fp64_pipe_frac": cost["fp64_ops"] * ncell / t / (peaks["fp64_tflops"] * 1e12 / 2.0)}
    return out


def run_mg_non_fft(torch, vdp, dev, stream, n=160):
    """A grid the FFT passes cannot take (160 = 2^5 x 5): the hot-spot recipe (hot spots scaled by
    volume, density ratio 4), mixed to 1e-8, by CG with the multigrid V-cycle and with Jacobi."""
    import vdp_inputs as V
    prob = V.hotspot_problem(n, seed=2, nspots=int(round(20000 * n ** 3 / 256 ** 3)), tol=1e-8,
                             target_ratio=4.0)
    rho = torch.from_numpy(prob.rho).to(dev)
    f = torch.from_numpy(prob.f).to(dev)
    out = {"grid": [n, n, n], "tol": 1e-8, "precision": "mixed",
           "fft_supported": vdp.spectral_supported(n, n, n)}
    for name, pc in (("mg", vdp.VDP_PRECOND_MG), ("jacobi", vdp.VDP_PRECOND_JACOBI)):
        with vdp.Solver(n, n, n, prob.L, precision="mixed", stream=stream, precond=pc) as s:
            s.set_density(rho)
            p = torch.empty_like(f)
            s.solve(f, p, 1e-8)
            ts = [s.solve(f, p, 1e-8) for _ in range(3)]
        b = min(ts, key=lambda x: x.ms)
        out[name] = {"solves_per_s": 1e3 / b.ms, "ms": b.ms, "iters": b.iters, "status": vdp.vdp_strerror(b.status)}
    return out


def run_duct(torch, vdp, dev, stream, shape=(128, 128, 256), lengths=(4.0 * math.pi, 2.0 * math.pi, 2.0 * math.pi)):
    """The inflow-outflow duct (periodic y, z; no pressure flux through the x ends), 256 x 128 x
    128 cells of equal size: the paper's fixed-point iteration (FP64 to 1e-10, mixed to 1e-8) and
    CG with the multigrid V-cycle (mixed to 1e-8)."""
    import vdp_inputs as V
    prob = V.duct_problem(shape, lengths, seed=21)
    rho = torch.from_numpy(prob.rho).to(dev)
    f = torch.from_numpy(prob.f).to(dev)
    nz, ny, nx = shape
    out = {"grid": [nx, ny, nz], "lengths": list(lengths), "density_ratio": round(prob.info["ratio"], 3)}
    for name, prec, tol, opts in (("fp64_fixed_point_1e-10", "fp64", 1e-10, {"method": vdp.VDP_METHOD_FIXED_POINT}),
                                  ("mixed_fixed_point_1e-8", "mixed", 1e-8, {"method": vdp.VDP_METHOD_FIXED_POINT}),
                                  ("mixed_cg_mg_1e-8", "mixed", 1e-8, {"precond": vdp.VDP_PRECOND_MG})):
        with vdp.Solver(nx, ny, nz, lengths[1], precision=prec, stream=stream, lengths=lengths,
                        bc_x=vdp.VDP_BC_DUCT, **opts) as s:
            s.set_density(rho)
            p = torch.empty_like(f)
            s.solve(f, p, tol)
            ts = [s.solve(f, p, tol) for _ in range(3)]
        b = min(ts, key=lambda x: x.ms)
        out[name] = {"solves_per_s": 1e3 / b.ms, "ms": b.ms, "iters": b.iters, "status": vdp.vdp_strerror(b.status)}
    return out


# Serving: worker slots (each a CUDA stream and a host thread); the process asks the driver for
# as many hardware work queues as there are slots (CUDA_DEVICE_MAX_CONNECTIONS, read when CUDA
# starts) so that the slots' streams do not share queues.
SERVE_SLOTS = 16


def _serve_bank_jobs():
    import vdp_inputs as V
    return [(n, k) for n in V.SERVE_SIZES for k in range(V.SERVE_BANK)]


def gpu_hotspot_scales(torch, base, H, goals, chunk: int = 32):
    """vdp_inputs.hotspot_scale for many ratios at once on the GPU: the same bracket (first power
    of two reaching the ratio) and the same 60 bisection steps, evaluated over the cells that can
    hold the extremes (the same values elementwise; max and min are exact), so each scale is the
    one the host function returns."""
    def ratio_full(s):
        T = base + s * H
        return float(T.max() / T.min())
    hi = 1.0
    while ratio_full(hi) < max(goals) and hi < 1e6:
        hi *= 2.0
    top = base + hi * H
    keep = (top >= base.max()) | (base <= top.min())
    bc, hc = base[keep], H[keep]
    out = []
    for i in range(0, len(goals), chunk):
        g = torch.tensor(goals[i:i + chunk], dtype=torch.float64, device=base.device)

        def ratio(sv):
            T = bc[None, :] + sv[:, None] * hc[None, :]
            return T.max(dim=1).values / T.min(dim=1).values
        lo = torch.zeros_like(g)
        hi_v = torch.ones_like(g)
        for _ in range(24):
            hi_v = torch.where(ratio(hi_v) < g, 2.0 * hi_v, hi_v)
        for _ in range(60):
            mid = 0.5 * (lo + hi_v)
            below = ratio(mid) < g
            lo = torch.where(below, mid, lo)
            hi_v = torch.where(below, hi_v, mid)
        out.extend((0.5 * (lo + hi_v)).tolist())
    return out


def run_serving(torch, vdp, dev, banks, count=5000):
    """Config 4: the Poisson stream (lambda = 200/s, request j from seed 100000 + j).  Each
    request's inputs are made at its arrival by the client on the GPU from its seeded field set
    of its grid size: rho = 1 / (base + s H) with s giving its density ratio exactly, and f, each
    periodically shifted by its seeded draw (vdp_inputs.request_fields, evaluated with torch on
    device-resident field sets)."""
    import vdp_inputs as V
    from paper_1601_05448_gb300 import serve
    meta = V.config4_requests(count)
    gb = {key: tuple(torch.from_numpy(a).to(dev) for a in bank) for key, bank in banks.items()}
    draws = [V.request_draw(r) for r in meta]
    scales = [0.0] * len(meta)
    for key in gb:
        idx = [i for i, (r, d) in enumerate(zip(meta, draws)) if (r.n, d[0]) == key]
        if idx:
            for i, sv in zip(idx, gpu_hotspot_scales(torch, gb[key][0], gb[key][1], [meta[i].ratio for i in idx])):
                scales[i] = sv
    client = torch.cuda.Stream(device=dev)
    reqs = [serve.ServeRequest(r.j, r.arrival_s, (r.n, r.n, r.n), V.TWO_PI, None, None, r.tol) for r in meta]

    def source(req):  # the client makes the request's inputs on the GPU when it arrives (its
        # own stream; the event tells the serving slot when they are written)
        r, d = meta[req.rid], draws[req.rid]
        base, H, f = gb[(r.n, d[0])]
        with torch.cuda.stream(client):
            req.rho = torch.roll(1.0 / (base + scales[req.rid] * H), d[1], dims=(0, 1, 2))
            req.f = torch.roll(f, d[2], dims=(0, 1, 2))
            req.ready = torch.cuda.Event()
            req.ready.record(client)

    def done(req):  # the client takes the result and lets go of the inputs and the result
        req.rho = req.f = req.p = req.ready = None

    # the client makes two requests' fields of every size once before the stream (its kernels
    # loaded and its allocations cached on its stream, as in a client that is already running)
    for n in V.SERVE_SIZES:
        for r_ in [r for r in reqs if r.shape[0] == n][:2]:
            source(r_)
            done(r_)
    torch.cuda.synchronize(dev)

    torch.cuda.synchronize(dev)
    with serve.Server("mixed", hbm_budget=96 << 30, max_active=SERVE_SLOTS, precond="fixed_point",
                      mode="streams") as srv:
        warmed = srv.warm([(n, n, n) for n in V.SERVE_SIZES], V.TWO_PI)
        stats = srv.run(reqs, source=source, on_done=done)
    ok = all(r.status == vdp.VDP_OK for r in reqs)
    s = stats.summary()
    by = {}
    for n in V.SERVE_SIZES:  # latency (arrival to result) and service time (admission to result)
        rs = [r for r in reqs if r.shape[0] == n and r.status == vdp.VDP_OK]
        if rs:
            lat = np.array([r.latency_s for r in rs])
            svc = np.array([r.t_done - r.t_admit for r in rs])
            by[n] = {"requests": len(rs), "p50_latency_s": float(np.percentile(lat, 50)),
                     "p99_latency_s": float(np.percentile(lat, 99)), "p50_service_s": float(np.percentile(svc, 50)),
                     "p99_service_s": float(np.percentile(svc, 99)), "mean_iters": float(np.mean([r.iters for r in rs]))}
    s["by_grid"] = by
    arr = np.array([r.arrival_s for r in reqs])
    late = [r for r in reqs if r.latency_s > 0.1]
    s["late_over_100ms"] = {"count": len(late), "first_arrival_s": float(min((r.arrival_s for r in late), default=0)),
                           "last_arrival_s": float(max((r.arrival_s for r in late), default=0)),
                           "stream_s": float(arr.max())}
    s.update({"requests": count, "offered_rate_per_s": 200.0, "engine": f"streams ({SERVE_SLOTS} worker slots)",
              "contexts_warmed": warmed,
              "method": "the paper's fixed-point iteration, mixed precision, per-request tolerance",
              "statuses_ok": ok,
              "inputs": f"per request: its seeded field set ({V.SERVE_BANK} per grid size), density ratio U[2,10] "
                        "exact, seeded periodic shifts of rho and f; made on the GPU at arrival"})
    return s


def timed(torch, solver, f, p, tol, steps, warmup, stream, barrier):
    """K solves bracketed by CUDA events on the solver's stream after >= 3 warm-up solves."""
    for _ in range(max(warmup, 3)):
        solver.solve(f, p, tol)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(steps):
        stats.append(solver.solve(f, p, tol))
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1) / 1e3, stats


def best_of(solver, f, p, tol, n=3):
    solver.solve(f, p, tol, check=False)
    ts = [solver.solve(f, p, tol, check=False) for _ in range(n)]
    return min(ts, key=lambda x: x.ms)


def solve_summary(vdp, st, extra=None):
    out = {"solves_per_s": 1e3 / st.ms, "ms": st.ms, "iters": st.iters, "outer": st.outer_iters,
           "rel_res": st.rel_res, "status": vdp.vdp_strerror(st.status)}
    out.update(extra or {})
    return out


def _guard(line, key, fn):
    """Run one extra of the line; a failure is recorded instead of ending the benchmark."""
    try:
        line[key] = fn()
    except Exception as e:  # pragma: no cover - reported in the line
        line[key] = {"error": f"{type(e).__name__}: {e}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-iters", type=int, default=3, help="oracle iterations per reference-arm sample")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, the FP64 comparison, 256^3, batch, serving, "
                                                              "CPU baseline")
    ap.add_argument("--serve-requests", type=int, default=5000, help="requests of the serving stream")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "grid"],
                    help="c2: 512^3 mixed to 1e-8 (the benchmark); c1: 256^3 FP64 to 1e-10; grid: the hot-spot "
                         "recipe at --grid (density ratio 4), for profiling small cases")
    ap.add_argument("--grid", type=int, default=192, help="grid size of --workload grid")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "mixed_bf16"],
                    help="precision of the main solve (default: mixed for c2, fp64 otherwise)")
    ap.add_argument("--precond", default="spectral", choices=list(PRECONDS),
                    help="preconditioner of the main solve when --method cg")
    ap.add_argument("--steps-per-sync", type=int, default=0,
                    help="0: each solve is one graph launch with a device-side loop (the benchmark); N > 0: "
                         "graphs of N rounds polled by the host (kernels visible to ncu, which cannot profile "
                         "kernels inside conditional graph nodes)")
    ap.add_argument("--method", default="fixed_point", choices=["cg", "fixed_point"],
                    help="fixed_point: the paper's iteration (the benchmark); cg: preconditioned conjugate "
                         "gradients (--precond)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(2 * SERVE_SLOTS))

    import multiprocessing as mp
    import vdp_inputs as V

    extras = not args.no_extras and rank == 0
    pool = jobs = None
    if extras:  # inputs of the extras, made in a spawn pool (before CUDA starts) while the main
        # process makes the benchmark's own input
        pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
        jobs = {"batch": pool.map_async(V.config3_instance, range(64)),
                "serve": pool.starmap_async(V.serve_bank, _serve_bank_jobs())}
        if args.workload == "c2":
            jobs["c1"] = pool.apply_async(V.config1)
    if args.workload == "c2":
        prob, key, workload, prec = V.config2(), "c2", WORKLOAD_C2, args.precision or "mixed"
    elif args.workload == "c1":
        prob, key, workload, prec = V.config1(), "c1", WORKLOAD_C1, args.precision or "fp64"
    else:
        n = args.grid
        prec = args.precision or "fp64"
        prob = V.hotspot_problem(n, seed=2, nspots=int(round(20000 * n ** 3 / 256 ** 3)), tol=1e-10,
                                 target_ratio=4.0)
        key = None
        workload = (f"{n}^3 periodic box L=2pi, rho=T0/T (hot spots scaled by volume, density ratio 4), rhs=div "
                    f"of random |k|<=4 velocity; {prec} (profiling case)")
    prob.tol = 1e-10 if (args.workload != "c2" and prec == "fp64") else 1e-8

    import torch
    import paper_1601_05448_gb300 as vdp

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    fixed = args.method == "fixed_point"
    method = METHOD_FP if fixed else {
        "spectral": "CG preconditioned by the constant-coefficient FFT inverse (Sec. 3.4)",
        "cheb": "CG preconditioned by a degree-3 Chebyshev polynomial", "jacobi": "Jacobi-preconditioned CG",
        "mg": "CG preconditioned by a geometric multigrid V-cycle"}[args.precond]
    nz, ny, nx = prob.shape
    ncell = nx * ny * nz
    rho = torch.from_numpy(prob.rho).to(dev)
    f = torch.from_numpy(prob.f).to(dev)
    p = torch.empty_like(f)
    stream = torch.cuda.current_stream(dev)
    if fixed:
        popts = {"method": vdp.VDP_METHOD_FIXED_POINT, "inner_tol": fixed_inner_tol(args.workload, prec)}
    else:
        popts = {"precond": PRECONDS[args.precond]}
        if args.precond == "cheb":
            popts["cheb_degree"] = 3
    solver = vdp.Solver(nx, ny, nz, prob.L, precision=prec, stream=stream, steps_per_sync=args.steps_per_sync,
                        **popts)
    solver.set_density(rho)
    peaks = load_peaks()
    measure_fp64_peak(vdp, peaks, stream)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    with ClockSampler(local) as clk:
        # the sampler runs from before the warm-up to the end of the timed region; its start-up
        # (a second process initialising the driver) is over before the timed solves begin
        clk.wait_first()
        elapsed, stats = timed(torch, solver, f, p, prob.tol, args.steps, args.warmup, stream, barrier)
    elapsed = max_over_ranks(elapsed, pg, dev)
    value = replica_rate(world, args.steps, elapsed)
    iters, outer = stats[-1].iters, stats[-1].outer_iters

    # per-kernel durations: one instrumented solve of the same workload on the same solver and
    # stream, every launch bracketed by CUDA events
    pt = torch.empty_like(f)
    st_t, kinds = solver.solve_timed(f, pt, prob.tol)
    assert st_t.iters == iters and torch.equal(pt, p), "instrumented solve differs from the timed solves"
    del pt
    slabbed = solver.spectral_slabs() > 1
    table = kernel_table(prec, ncell, kinds, peaks, nx, nx=nx, fixed=fixed, slabbed=slabbed)
    roof = roofline(prec, table, peaks)
    b_solve = algorithmic(prec, ncell, iters, outer, args.precond == "spectral", nx, fixed, slabbed)
    dtype = {"fp64": "f64", "mixed": "f32 inner, f64 outer",
             "mixed_bf16": "f32 inner (bf16 coefficients), f64 outer"}[prec]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": workload, "method": method, "grid": [nx, ny, nz], "tol": prob.tol,
                   "inner_tol": popts.get("inner_tol"),
                   "density_ratio": round(prob.info["ratio"], 4),
                   "l2": f"inputs larger than L2 (~{ncell * 115 / 1e9:.1f} GB working set)", "replicas": world},
        "gpu_launches": sum(s_.launches for s_ in stats),
        "roofline": roof,
        "clocks": clk.summary(),
        "iterations": iters, "outer_iterations": outer, "rel_res": stats[-1].rel_res,
        # each solve's own device time (library events around its graph launch): the gap to
        # ms_per_step is host time between solves
        "solve_ms_median": statistics.median(st_.ms for st_ in stats),
        "gdof_iter_per_s": ncell * iters * args.steps * world / elapsed / 1e9,
        "solve_hbm_frac": b_solve * args.steps * world / elapsed / 1e9 / peaks["hbm_gbs"],
        "fp64_peak": {k: peaks[k] for k in ("fp64_tflops", "fp64_tflops_derived", "fp64_source") if k in peaks},
        "spectral_slabs": solver.spectral_slabs(),
        "kernels": table,
    }

    summary = {}
    if not args.no_extras:
        # end to end through the C ABI with host buffers: H2D of rhs and D2H of p inside the timing
        def e2e():
            fh = torch.from_numpy(prob.f).pin_memory()
            ph = torch.empty(prob.shape, dtype=torch.float64).pin_memory()
            solver.solve(fh, ph, prob.tol)
            barrier()
            t0 = time.perf_counter()
            ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ee0.record(stream)
            for _ in range(args.steps):
                solver.solve(fh, ph, prob.tol)
            ee1.record(stream)
            barrier()
            e_el = max_over_ranks(max(ee0.elapsed_time(ee1) / 1e3, 1e-9), pg, dev)
            return {"value": replica_rate(world, args.steps, e_el), "unit": "solves/s",
                    "h2d_bytes_per_step": int(prob.f.nbytes), "d2h_bytes_per_step": int(prob.f.nbytes),
                    "wall_s": time.perf_counter() - t0}
        _guard(line, "e2e", e2e)

    if extras and args.workload == "c2" and fixed:
        # the plain FP64 solve on the same input to the same tolerance, timed the same way
        def fp64_same_input():
            with vdp.Solver(nx, ny, nz, prob.L, precision="fp64", stream=stream, **popts) as s64:
                s64.set_density(rho)
                p64 = torch.empty_like(f)
                el64, st64 = timed(torch, s64, f, p64, prob.tol, args.steps, args.warmup, stream, barrier)
                _, k64 = s64.solve_timed(f, p64, prob.tol)
                sl64 = s64.spectral_slabs() > 1
            tab = kernel_table("fp64", ncell, k64, peaks, nx, nx=nx, fixed=True, slabbed=sl64)
            return {"solves_per_s": args.steps / el64, "ms_per_step": 1e3 * el64 / args.steps,
                    "iters": st64[-1].iters, "outer": st64[-1].outer_iters, "rel_res": st64[-1].rel_res,
                    "roofline": roofline("fp64", tab, peaks),
                    "kernels": {n_: {x: r[x] for x in ("launches", "mean_us", "share", "gbs", "hbm_frac",
                                                       "fp64_flop_frac", "fp64_issue_frac") if x in r}
                                for n_, r in tab.items()}}
        _guard(line, "fp64_1e-8", fp64_same_input)
        if "solves_per_s" in line["fp64_1e-8"]:
            summary["fp64_1e-8_solves_per_s"] = line["fp64_1e-8"]["solves_per_s"]
            summary["mixed_over_fp64"] = value / line["fp64_1e-8"]["solves_per_s"]
            summary["fp64_1e-8_iters"] = line["fp64_1e-8"]["iters"]

        def c2_variants():
            out = {}
            bf16_opts = {"method": vdp.VDP_METHOD_FIXED_POINT,
                         "inner_tol": fixed_inner_tol(args.workload, "mixed_bf16")}
            for label, prec2, opts in (("mixed_bf16_fixed_point", "mixed_bf16", bf16_opts),
                                       ("mixed_cg_spectral", "mixed", {"precond": vdp.VDP_PRECOND_SPECTRAL}),
                                       ("fp64_cg_spectral", "fp64", {"precond": vdp.VDP_PRECOND_SPECTRAL})):
                with vdp.Solver(nx, ny, nz, prob.L, precision=prec2, stream=stream, **opts) as s2:
                    s2.set_density(rho)
                    out[label] = solve_summary(vdp, best_of(s2, f, torch.empty_like(f), prob.tol))
            return out
        _guard(line, "c2_variants_1e-8", c2_variants)

    if extras:
        c1 = prob if args.workload == "c1" else (jobs["c1"].get() if "c1" in jobs else None)
        if c1 is not None and args.workload == "c2":
            _guard(line, "c1_256", lambda: run_c1(torch, vdp, dev, c1, stream, peaks, args, barrier))
            if "solves_per_s" in line["c1_256"]:
                summary["c1_fp64_1e-10_solves_per_s"] = line["c1_256"]["solves_per_s"]
        if c1 is not None:
            _guard(line, "mixed_vs_fp64_at_1e-8_256", lambda: run_c1_variants(torch, vdp, dev, c1, stream, peaks))
            _guard(line, "mg_non_fft_grid", lambda: run_mg_non_fft(torch, vdp, dev, stream))
            _guard(line, "duct", lambda: run_duct(torch, vdp, dev, stream))
            _guard(line, "projection_step", lambda: run_c1_projection(torch, vdp, dev, c1, stream, peaks))
        batch_probs = jobs["batch"].get()
        _guard(line, "batch", lambda: run_batch(torch, vdp, dev, batch_probs))
        keep = ("seconds", "solves_per_s", "gdof_iter_per_s", "iterations_total", "all_ok")
        _guard(line, "batch_cg_spectral", lambda: {k: v for k, v in run_batch(
            torch, vdp, dev, batch_probs, precond="spectral").items() if k in keep})
        _guard(line, "batch_jacobi", lambda: {k: v for k, v in run_batch(
            torch, vdp, dev, batch_probs, precond="jacobi").items() if k in keep})
        _guard(line, "batch_jacobi_persistent", lambda: {k: v for k, v in run_batch(
            torch, vdp, dev, batch_probs, True, "jacobi").items() if k in keep})
        banks = dict(zip(_serve_bank_jobs(), jobs["serve"].get()))
        pool.close()
        _guard(line, "serving", lambda: run_serving(torch, vdp, dev, banks, args.serve_requests))
        del banks
        if key is not None:
            _guard(line, "cpu_baseline", lambda: cpu_baseline(prob, key, iters_per_sample=3))
        if "solves_per_s" in line.get("batch", {}):
            summary["batch_solves_per_s"] = line["batch"]["solves_per_s"]
        sv = line.get("serving", {})
        for k_ in ("solves_per_s", "p50_latency_s", "p99_latency_s", "completed"):
            if k_ in sv:
                summary["serving_" + k_] = sv[k_]
    solver.close()
    # compact comparison last, so the end of the line carries it
    line["summary"] = dict(summary, headline_solves_per_s=value, headline_iters=iters,
                           roofline_frac=roof["frac"], roofline_kernel=roof["kernel"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_c1(torch, vdp, dev, prob, stream, peaks, args, barrier):
    """The 256^3 FP64 workload to 1e-10 by the fixed-point iteration, timed like the headline,
    with its kernel table and roofline; CG with the spectral, multigrid and Jacobi
    preconditioners beside it."""
    nz, ny, nx = prob.shape
    ncell = nx * ny * nz
    rho = torch.from_numpy(prob.rho).to(dev)
    f = torch.from_numpy(prob.f).to(dev)
    p = torch.empty_like(f)
    fp = {"method": vdp.VDP_METHOD_FIXED_POINT, "inner_tol": 1e-4}
    with vdp.Solver(nx, ny, nz, prob.L, precision="fp64", stream=stream, **fp) as s:
        s.set_density(rho)
        el, st = timed(torch, s, f, p, 1e-10, args.steps, args.warmup, stream, barrier)
        _, kinds = s.solve_timed(f, p, 1e-10)
    tab = kernel_table("fp64", ncell, kinds, peaks, nx, nx=nx, fixed=True)
    out = {"workload": WORKLOAD_C1, "solves_per_s": args.steps / el, "ms_per_step": 1e3 * el / args.steps,
           "iters": st[-1].iters, "outer": st[-1].outer_iters, "rel_res": st[-1].rel_res,
           "roofline": roofline("fp64", tab, peaks), "kernels": tab}
    for label, opts in (("cg_spectral", {"precond": vdp.VDP_PRECOND_SPECTRAL}), ("cg_mg", {"precond": vdp.VDP_PRECOND_MG}),
                        ("cg_jacobi", {"precond": vdp.VDP_PRECOND_JACOBI})):
        with vdp.Solver(nx, ny, nz, prob.L, precision="fp64", stream=stream, **opts) as s:
            s.set_density(rho)
            out["fp64_" + label + "_1e-10"] = solve_summary(vdp, best_of(s, f, p, 1e-10, 2))
    try:
        out["cpu_baseline"] = cpu_baseline(prob, "c1")
    except Exception as e:  # the stored iteration count is missing
        out["cpu_baseline"] = {"value": None, "unit": "solves/s", "kind": "oracle", "error": str(e)}
    return out


def run_c1_variants(torch, vdp, dev, prob, stream, peaks):
    """Every method and precision on the 256^3 input to relative residual 1e-8 (equal final
    accuracy), each residual confirmed by the oracle's operator."""
    import oracle
    nz, ny, nx = prob.shape
    ncell = nx * ny * nz
    rho = torch.from_numpy(prob.rho).to(dev)
    f = torch.from_numpy(prob.f).to(dev)
    paths = {}
    variants = {"fp64_fixed_point": ("fp64", "fixed_point", 1), "mixed_fixed_point": ("mixed", "fixed_point", 1),
                "mixed_bf16_fixed_point": ("mixed_bf16", "fixed_point", 1),
                "fp64_spectral": ("fp64", "spectral", 1), "mixed_spectral": ("mixed", "spectral", 1),
                "mixed_bf16_spectral": ("mixed_bf16", "spectral", 1), "fp64_mg": ("fp64", "mg", 1),
                "mixed_mg": ("mixed", "mg", 1), "fp64_jacobi": ("fp64", "jacobi", 1),
                "mixed_jacobi": ("mixed", "jacobi", 1), "mixed_cheb3": ("mixed", "cheb", 3),
                "mixed_bf16_jacobi": ("mixed_bf16", "jacobi", 1)}
    for label, (prec, pc, k) in variants.items():
        opts = ({"method": vdp.VDP_METHOD_FIXED_POINT, "inner_tol": 1e-4} if pc == "fixed_point"
                else {"precond": PRECONDS[pc]})
        if pc == "cheb":
            opts["cheb_degree"] = k
        with vdp.Solver(nx, ny, nz, prob.L, precision=prec, stream=stream, **opts) as s2:
            s2.set_density(rho)
            pp = torch.empty_like(f)
            best = best_of(s2, f, pp, 1e-8)
            _, kk = s2.solve_timed(f, pp, 1e-8, check=False)
            tab = kernel_table(prec, ncell, kk, peaks, nx, cheb_k=k, nx=nx, fixed=pc == "fixed_point")
            paths[label] = solve_summary(vdp, best, {
                "oracle_rel_res": oracle.relative_residual(prob.rho, prob.L, prob.f, pp.cpu().numpy()),
                "kernels": {n: {x: r[x] for x in ("mean_us", "share", "gbs", "hbm_frac") if x in r}
                            for n, r in tab.items()}})
    return paths


def run_c1_projection(torch, vdp, dev, prob, stream, peaks):
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, prob.L, precision="fp64", stream=stream, method=vdp.VDP_METHOD_FIXED_POINT,
                    inner_tol=1e-4) as s:
        s.set_density(torch.from_numpy(prob.rho).to(dev))
        return run_projection(torch, vdp, dev, s, prob, stream, peaks)


if __name__ == "__main__":
    sys.exit(main())
