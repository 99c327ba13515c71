"""The benchmark's roofline bookkeeping (host logic, no GPU): the algorithmic bytes and FP64
operations per cell that bench.py charges each sweep, written out here from the sweeps' operand
lists, and the roofline object recomputed from the kernel table's own fields."""
import math

import pytest

import bench

N512 = 512 ** 3
N256 = 256 ** 3


def test_fused_sweep_and_residual_bytes():
    # fused fixed-point sweep: z (FP32), three coefficients, rt and x read, rt and x written
    assert bench.sweep_cost("mixed", "stencil", fixed=True)[0] == 4 + 3 * 4 + 2 * 4 + 2 * 4
    assert bench.sweep_cost("fp64", "stencil", fixed=True)[0] == 4 + 3 * 8 + 2 * 8 + 2 * 8
    assert bench.sweep_cost("mixed_bf16", "stencil", fixed=True)[0] == 4 + 3 * 2 + 2 * 4 + 2 * 4 + 2
    # full residual: p, f - <f>, sinv, D, three FP64 coefficients read, rt written
    b, fl, hbm = bench.sweep_cost("mixed", "res64")
    assert (b, hbm) == (7 * 8 + 4, 7 * 8 + 4) and fl == 14.0      # 7 FMA
    assert bench.sweep_cost("fp64", "res64")[1] == 15.0            # and the FP64 scaling multiply
    # first residual from p = 0: f and sinv read, f - <f> and rt written
    assert bench.sweep_cost("mixed", "res64_first")[0] == 8 + 8 + 8 + 4
    assert bench.FP64_PIPE_OPS["res64"] == 8.0 and bench.FP64_PIPE_OPS["stencil_fixed"] == 8.0


def test_spectral_bytes_follow_the_half_spectrum():
    S = 8.0 * 264 / 512                                    # 264 complex values per row of 512
    assert bench.spectrum_bytes(512) == S
    # 512^3: the half spectrum (553 MB) goes through HBM in every pass
    alg, hbm = bench.spec_bytes("mixed", "spec_x", 512, N512, False, True)
    assert alg == hbm == 4 + 4 + S + S + 4 + 4             # rt, W -> S; S, W -> z (FP32)
    assert bench.spec_bytes("mixed", "spec_y", 512, N512, False, True) == (4 * S, 4 * S)
    assert bench.spec_bytes("mixed", "spec_z", 512, N512, False, True) == (2 * S, 2 * S)
    # 256^3: the half spectrum stays in L2, only rt / W / z reach HBM
    S256 = bench.spectrum_bytes(256)
    assert S256 * N256 <= 0.6 * bench.L2_BYTES
    assert bench.spec_bytes("mixed", "spec_x", 256, N256, False, True)[1] == 4 + 4 + 4 + 4
    assert bench.spec_bytes("mixed", "spec_y", 256, N256, False, True)[1] == 0


def test_roofline_is_reproducible_from_the_table():
    peaks = {"hbm_gbs": 6789.0, "bf16_tflops": 1887.0, "fp64_tflops": 1.05, "source": "measured",
             "fp64_source": "measured"}
    kinds = {
        "res64": {"launches": 3, "ms": 3 * 1.38, "ms_min": 0.72, "ms_mean": 1.38},
        "stencil": {"launches": 12, "ms": 12 * 0.668, "ms_min": 0.60, "ms_mean": 0.668},
        "spec_x": {"launches": 24, "ms": 24 * 0.265, "ms_min": 0.25, "ms_mean": 0.265},
        "spec_y": {"launches": 24, "ms": 24 * 0.191, "ms_min": 0.18, "ms_mean": 0.191},
        "spec_z": {"launches": 12, "ms": 12 * 0.327, "ms_min": 0.32, "ms_mean": 0.327},
    }
    table = bench.kernel_table("mixed", N512, kinds, peaks, 512, nx=512, fixed=True)
    roof = bench.roofline("mixed", table, peaks)
    assert roof["sweep"] == "stencil" and roof["bound"] == "hbm"     # the largest share
    row = table["stencil"]
    achieved = row["hbm_alg_bytes_per_launch"] / (row["mean_us"] * 1e-6) / 1e9
    assert math.isclose(roof["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(roof["frac"], achieved / peaks["hbm_gbs"], rel_tol=1e-12)
    assert row["hbm_alg_bytes_per_launch"] == 32 * N512
    # the residual row averages the first (short) launch with the full ones
    full, first = bench.sweep_cost("mixed", "res64")[0], bench.sweep_cost("mixed", "res64_first")[0]
    assert table["res64"]["alg_bytes_per_launch"] == pytest.approx((2 * full + first) / 3 * N512)
    # spectral kinds per application: bytes over all launches of the kind, over its time
    alg = bench.spec_bytes("mixed", "spec_x", 512, N512, False, True)[0]
    assert table["spec_x"]["gbs"] == pytest.approx(alg * N512 * 12 / (24 * 0.265e-3) / 1e9)


def test_headline_inner_reduction():
    assert bench.fixed_inner_tol("c2", "mixed") == 4e-5
    assert bench.fixed_inner_tol("c2", "mixed_bf16") == 1e-4
    assert bench.fixed_inner_tol("c1", "mixed") == 1e-4
