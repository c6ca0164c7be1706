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
    assert r["achieved_gbs"] == pytest.approx(r["algorithmic_bytes_per_step"] / 1e6)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 1000.0)
