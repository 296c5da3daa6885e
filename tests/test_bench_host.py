"""Host-side arithmetic of bench.py: the binding roofline and the whole-job rate."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_hbm_roof_binds_below_the_ridge():
    # 14.8 flop/B against a 578 TFLOP/s compute peak and 6.79 TB/s: ridge 85 flop/B
    bind, other, inten, ridge = bench.binding_roofline(3.68e14, 2.49e13, 9.77, ("tensor", 578.3, "c"), (6789.6, "h"))
    assert bind["bound"] == "hbm" and other["bound"] == "tensor"
    assert inten == pytest.approx(3.68e14 / 2.49e13) and ridge == pytest.approx(578.3e12 / 6789.6e9)
    assert bind["achieved"] == pytest.approx(2.49e13 / 9.77 / 1e9)
    assert bind["frac"] == pytest.approx(bind["achieved"] / 6789.6)
    assert other["achieved"] == pytest.approx(3.68e14 / 9.77 / 1e12)


def test_compute_roof_binds_above_the_ridge():
    bind, other, _, ridge = bench.binding_roofline(1e15, 1e12, 2.0, ("alu", 80.5, "c"), (6789.6, "h"))
    assert 1e15 / 1e12 > ridge
    assert bind["bound"] == "alu" and bind["unit"] == "TFLOP/s"
    assert bind["frac"] == pytest.approx(1e15 / 2.0 / 1e12 / 80.5)
    assert other["bound"] == "hbm"


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(4, 512, 2, 10.0) == pytest.approx(4 * 512 * 2 / 10.0)
