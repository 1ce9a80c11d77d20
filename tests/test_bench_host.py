"""Host-side pieces of bench.py that need no GPU: the roofline record of a stage
launch (its numerator is the counted work per cell-stage, its denominator the
slower of the measured HBM and FMA bounds) and the rule that a DRAM traffic
figure is reported only for the kernel sources and launch configuration it was
measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

CELLS = 1024 * 1024
PEAKS = {"hbm_gbs": 6400.0}


def test_mixed_roofline_is_the_fp32_bound_at_the_counted_flops():
    alu = {"fp32": 75.0, "fp64": 1.0}
    r = bench.stage_roofline("mixed", CELLS, 0.25, PEAKS, alu, {"tile_x": 32, "tile_y": 8, "threads": 256})
    # 3813 flops x 2^20 cells in 0.25 ms against 75 TFLOP/s; 256 B x 2^20 at 6400 GB/s
    t_alu = bench.FLOPS_PER_CELL_STAGE * CELLS / 75e12
    t_hbm = bench.BYTES_PER_CELL_STAGE_MIXED * CELLS / 6400e9
    assert t_alu > t_hbm and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.FLOPS_PER_CELL_STAGE * CELLS / 0.25e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 75.0)
    assert r["alu_frac"] == pytest.approx(t_alu / 0.25e-3) and r["hbm_frac"] == pytest.approx(t_hbm / 0.25e-3)
    assert r["launch_config"] == "32x8x256"


def test_fp64_roofline_uses_the_fp64_peak_and_409_6_bytes():
    r = bench.stage_roofline("fp64", CELLS, 4.0, PEAKS, {"fp32": 75.0, "fp64": 1.0})
    assert bench.BYTES_PER_CELL_STAGE_FP64 == pytest.approx(3.2 * 16 * 8)
    assert r["bound"] == "alu" and r["peak"] == 1.0
    assert r["frac"] == pytest.approx(bench.FLOPS_PER_CELL_STAGE * CELLS / 4.0e-3 / 1e12)


def test_traffic_only_for_the_measured_sources_and_configuration():
    alu = {"fp32": 75.0, "fp64": 1.0}
    dig = bench.kernel_digest("mixed")
    measured = {k: v for k, v in bench.MEASURED_TRAFFIC.items() if k.startswith(dig + ":")}
    for key, bytes_ in measured.items():
        tx, ty, th = (int(v) for v in key.rsplit(":", 1)[1].split("x"))
        r = bench.stage_roofline("mixed", CELLS, 0.25, PEAKS, alu, {"tile_x": tx, "tile_y": ty, "threads": th})
        assert r["traffic"] == bytes_
    r = bench.stage_roofline("mixed", CELLS, 0.25, PEAKS, alu, {"tile_x": 16, "tile_y": 16, "threads": 256})
    assert ("mixed:%s:16x16x256" % dig) in bench.MEASURED_TRAFFIC or r["traffic"] is None
    r = bench.stage_roofline("mixed", CELLS, 0.25, PEAKS, alu, None)
    assert r["traffic"] is None


def test_fallback_hbm_peak_is_stated():
    r = bench.stage_roofline("mixed", CELLS, 0.001, {}, {"fp32": 75.0, "fp64": 1.0})
    assert r["hbm_peak_gbs"] == 6400.0
    r2 = bench.stage_roofline("mixed", CELLS, 0.001, {}, {})
    assert r2["peak_source"].startswith("of derived") or r2["bound"] == "hbm"
