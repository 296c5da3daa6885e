"""tests/golden/float32_spread.json, from which the GPU parity bounds are derived, is
complete and self-consistent: every figure the GPU tests read is present, finite and
positive, every top-level maximum is the maximum over its rounding orders, and every
case carries all of the orders that tests/golden/make_float32_spread.py defines."""
import json
import math
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SPREAD = json.load(open(os.path.join(HERE, "golden", "float32_spread.json")))
sys.path.insert(0, os.path.join(HERE, "golden"))

FLOAT32_CASES = ("sweep_ratios_bond_decay_8x8", "sweep_ratios_iid_8x8_sampled")
SPLIT_CASES = ("split_bf16_bond_decay_8x8", "split_bf16_bond_decay_24x24")
SPLIT_KEYS = ("sweep_ratio_max", "eloc_rel_scale_max", "logpsi_abs_max", "grad_norm_max", "grad_elementwise_max")


def _orders():
    import make_float32_spread as m
    return {"%s/%s" % o for o in m.ORDERS}


@pytest.mark.parametrize("case", FLOAT32_CASES)
def test_float32_sweep_figures(case):
    c = SPREAD[case]
    assert set(c["per_order"]) == _orders()
    assert math.isfinite(c["max"]) and c["max"] > 0
    assert c["max"] == max(v["max"] for v in c["per_order"].values())
    assert c["median"] == max(v["median"] for v in c["per_order"].values())


def test_float32_gradient_figure():
    c = SPREAD["grad_iid_8x8_sampled"]
    assert set(c["per_order"]) == _orders()
    assert c["max"] == max(c["per_order"].values()) > 0


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_split_figures(case):
    c = SPREAD[case]
    assert set(c["per_order"]) == _orders()
    for k in SPLIT_KEYS:
        assert math.isfinite(c[k]) and c[k] > 0, k
        assert c[k] == max(v[k] for v in c["per_order"].values()), k


def test_24x24_figures_cover_the_tested_chains():
    """The 24x24 bounds come from the chains tests/test_gpu_parity_24x24.py checks."""
    import make_float32_spread as m
    src = open(os.path.join(HERE, "test_gpu_parity_24x24.py")).read()
    assert "SWEEP_CHAINS = %r" % (m.SWEEP_CHAINS_24,) in src
    assert "MEASURE_CHAINS = %r" % (m.MEASURE_CHAINS_24,) in src
