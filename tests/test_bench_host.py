"""Host-side logic of bench.py: sharding, kernel grouping, whole-job rate, defaults."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(4, 512, 2, 10.0) == pytest.approx(4 * 512 * 2 / 10.0)


def test_rank_share_slices_one_job():
    from paper_1908_09359_gb300 import inputs
    w = dict(inputs.WORKLOADS["peps_8x8"], seed=inputs.SEED_BASE + 1, n_chains=8)
    parts = [bench.rank_share(w, r, 4) for r in range(4)]
    whole = bench.rank_share(dict(w, n_chains=32), 0, 1)
    assert np.array_equal(np.concatenate([p["spins"] for p in parts]), whole["spins"])
    assert [p["chain_offset"] for p in parts] == [0, 8, 16, 24]
    assert len({p["key"] for p in parts}) == 1


def test_kernel_groups_totals():
    shapes = [{"shape": "fused4 32 32 32 32", "launches": 2, "flops": 4.0, "ms": 1.0},
              {"shape": "fused4 8 8 32 32", "launches": 1, "flops": 1.0, "ms": 0.5},
              {"shape": "gemm tc M256 N32 K256", "launches": 3, "flops": 3.0, "ms": 0.3},
              {"shape": "qr 256x32", "launches": 5, "flops": 0.0, "ms": 0.2},
              {"shape": "fusedP 32 32 32 32 x 8 8 8 8", "launches": 4, "flops": 8.0, "ms": 0.4},
              {"shape": "metropolis", "launches": 6, "flops": 0.0, "ms": 0.1},
              {"shape": "normalize_pow2", "launches": 2, "flops": 0.0, "ms": 0.05}]
    g = bench.kernel_groups(shapes)
    assert g["fused4"] == {"launches": 3, "flops": 5.0, "ms": 1.5}
    assert g["gemm_tc"]["launches"] == 3 and g["qr"]["ms"] == 0.2
    assert g["fusedP"]["launches"] == 4 and g["reductions"]["launches"] == 8
    assert abs(g["reductions"]["ms"] - 0.15) < 1e-12


def test_default_arguments():
    a = bench.parse([])
    assert (a.gpus, a.steps, a.warmup, a.impl, a.precision) == (1, 2, 3, "ours", "bf16x3")
    assert a.case is None and a.study is None


def test_traffic_records_name_their_sources_and_summaries():
    for t in bench.NCU_TRAFFIC.values():
        assert os.path.exists(os.path.join(bench.ROOT, t["source"]))
        assert os.path.exists(os.path.join(bench.ROOT, t["summary"]))
        assert len(bench.source_sha(t["source"])) == 16 and t["bytes_per_chain"] > 0


def test_binding_roof_follows_the_ridge_point():
    """A kernel whose algorithmic intensity lies below the ridge point (compute peak over
    HBM bandwidth) is reported against HBM, one above it against the compute peak."""
    import bench
    cpeak, hbm = (("tensor", 1714.6, "m"), (6781.4, "m"))
    ridge = 1714.6e12 / 6781.4e9
    lo, other, inten, r = bench.binding_roofline(128.0 * 1e6, 1e6, 1e-3, cpeak, hbm)
    assert r == ridge and inten == 128.0 and lo["bound"] == "hbm" and other["bound"] == "tensor"
    assert abs(lo["achieved"] - 1.0) < 1e-12 and abs(lo["frac"] - 1.0 / 6781.4) < 1e-15
    hi, other, _, _ = bench.binding_roofline(400.0 * 1e6, 1e6, 1e-3, cpeak, hbm)
    assert hi["bound"] == "tensor" and abs(hi["achieved"] - 0.4) < 1e-12 and other["bound"] == "hbm"
