"""The bench's algorithmic-bytes model against the figures of the hot-path scope table
(whole step: grids written and read once, spectra once per use)."""
import pytest

import bench
from paper_2302_08694_gb300 import workloads as wl


def test_step_bytes_match_the_stated_floors():
    # 3D NS mixed, N = 128, M = 40322 (n_f = 256, N~ = 192): about 2.98 GB per step
    assert bench.step_bytes(wl.config_ns3d_mixed(), "mixed", 256, 192) == pytest.approx(2.98e9, rel=0.01)
    # 3D NS FP64, N = 64, M = 10082 (n_f = 128, N~ = 96): about 0.75 GB per step
    assert bench.step_bytes(wl.config_ns3d_fp64(), "fp64", 128, 96) == pytest.approx(0.75e9, rel=0.01)
    # differentiable 3D Stokes, N = 96, M = 20002 (n_f = 192): about 0.85 GB per forward step
    assert bench.step_bytes(wl.config_stokes3d_adjoint(), "mixed", 192, 144) == pytest.approx(0.85e9, rel=0.01)


def test_step_roofline_fraction():
    prob = wl.config_ns3d_fp64()
    r = bench.step_roofline(prob, "fp64", 128, 96, 1.0, {"hbm_gbs": 1000.0})
    assert r["achieved_gbs"] == pytest.approx(r["bytes"] / 1e6)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 1000.0)


def test_df64_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3 T FP32 instructions/s; a double-float
    # multiply-add takes 12 of them and counts as 2 flops
    assert bench.DF64_PEAK_GFLOPS == pytest.approx(152 * 128 * 2.07 * 2 / 12)
    assert 6.0e3 < bench.DF64_PEAK_GFLOPS < 7.0e3


def test_roofline_picks_the_pipe_of_the_arithmetic():
    pk = {"hbm_gbs": 6000.0}
    # 1 GFLOP and 10 MB in 1 ms: ALU-bound on every pipe
    site = {"name": "spread", "total_ms": 2.0, "launches": 2, "bytes": 1e7, "flops": 1e9}
    r = bench.roofline_of(site, "df64", pk, "measured", 1200.0, 70000.0, "w")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(1000.0 / bench.DF64_PEAK_GFLOPS)
    r = bench.roofline_of(site, "f64", pk, "measured", 1200.0, 70000.0, "w")
    assert r["frac"] == pytest.approx(1000.0 / 1200.0)
    # 1 MFLOP and 1 GB in 1 ms: HBM-bound, 1000 GB/s of 6000
    site = {"name": "rows", "total_ms": 1.0, "launches": 1, "bytes": 1e9, "flops": 1e6}
    r = bench.roofline_of(site, "f32", pk, "measured", 1200.0, 70000.0, "w")
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(1000.0 / 6000.0)
