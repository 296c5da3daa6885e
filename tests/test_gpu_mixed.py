"""The whole hot path in the tensor-core precisions against the FP64 oracle.

Each mode's error is stated and bounded here (tensors with simple-update-like bond
spectra, lambda_i = exp(-i), at the 8x8 workload shapes; random starts):
  * MIXED_BF16X3 (split BF16, x = hi + lo, three BF16 products): per operand ~2^-16;
    measured E_loc <= 1e-4 of the term scale, ln|Psi| <= 4e-4, G <= 2e-5 norm-wise,
    Metropolis decisions identical to FP32.  Bounds: 5e-4, 5e-3, 1e-3, >= 99 %.
  * MIXED_TF32: per operand 2^-11; measured E_loc <= 1e-2, ln|Psi| <= 3e-2.
    Bounds: 5e-2 and 1e-1.
  * MIXED_BF16: per operand 2^-9; measured E_loc <= 3e-2, ln|Psi| <= 0.2.
    Bounds: 1e-1 and 0.5 (at 24x24 a third of the sweep decisions differ from FP32,
    so this mode is a throughput reference, not a sampling mode).
"""
import json
import os

import numpy as np
import pytest

from oracle import vmc
from paper_1908_09359_gb300 import inputs

pytestmark = pytest.mark.gpu

BOUNDS = {3: (5e-4, 5e-3, 1e-3), 2: (5e-2, 1e-1, None), 1: (1e-1, 0.5, None)}
# twice the deviation of the oracle itself in emulated split BF16 at the 8x8 shapes
# (tests/golden/float32_spread.json, written by tests/golden/make_float32_spread.py)
SPLIT = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "float32_spread.json")))["split_bf16_bond_decay_8x8"]


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import api as a
    from paper_1908_09359_gb300 import build
    build.build()
    return a


def structured_8x8(n):
    w = inputs.workload("peps_8x8", n_chains=n)
    w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
    return w


@pytest.mark.parametrize("precision", [3, 2, 1])
def test_measure_in_mixed_precision(api, precision):
    w = structured_8x8(4)
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    sp = inputs.start_spins(4, 8, 8, 21, "random")
    ctx = api.PepsVMC(8, 8, 4, 16, 4, w["tensors"], w["sketch"], seed=3, precision=precision)
    ctx.set_spins(sp)
    e, lp, sg = ctx.measure()
    e_tol, lp_tol, g_tol = BOUNDS[precision]
    for c in range(4):
        r = vmc.measure(g, sp[c], 16, w["sketch"], 3, 1.0, 0.0, want_grad=g_tol is not None)
        assert abs(e[c] - r["eloc"]) <= e_tol * r["eloc_scale"], (c, e[c], r["eloc"])
        assert abs(lp[c] - r["logpsi"]) <= lp_tol
        if g_tol is not None:
            G = np.concatenate([x.ravel() for row in r["G"] for x in row])
            assert np.linalg.norm(ctx.chain_grad(c) - G) <= g_tol * np.linalg.norm(G)
    ctx.close()


def test_split_bf16_sweep_decisions_match_fp32(api):
    w = structured_8x8(32)
    sp = inputs.start_spins(32, 8, 8, 5, "random")
    dec = {}
    for precision in (0, 3):
        ctx = api.PepsVMC(8, 8, 4, 16, 32, w["tensors"], w["sketch"], seed=9, precision=precision)
        ctx.set_spins(sp)
        ctx.set_sweep_counter(2)
        ctx.enable_trace(True)
        ctx.sample_sweep(1)
        dec[precision] = ctx.get_trace()[1]
        ctx.close()
    assert np.mean(dec[0] == dec[3]) >= 0.99


@pytest.mark.parametrize("form", ["fused", "separate tcgen05 products"])
def test_split_bf16_whole_path_elementwise(api, form):
    """The chosen form (split BF16) through a whole sample step at the 8x8 shapes on
    bond-decay tensors, once with the fused column steps (the bench's form) and once with
    every product forced onto the separate tcgen05 kernel: one sweep's ratios and
    decisions, then E_loc, ln|Psi| and G element-wise against the FP64 oracle, each within
    twice the oracle's own deviation in emulated split BF16."""
    w = structured_8x8(6)
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    sp = inputs.start_spins(6, 8, 8, 31, "random")
    ctx = api.PepsVMC(8, 8, 4, 16, 6, w["tensors"], w["sketch"], seed=11, precision=3)
    if form != "fused":
        ctx.set_contraction_kernel("tc", 64)
    ctx.set_spins(sp)
    ctx.set_sweep_counter(3)
    ctx.enable_trace(True)
    ctx.sample_sweep(1)
    ratio, dec = ctx.get_trace()
    final = ctx.get_spins()
    for c in range(6):
        follow = {b: int(dec[c, b]) for b in range(ctx.n_bonds) if dec[c, b] >= 0}
        tr = vmc.Trace(follow=follow, tie=1e-5)
        new, _, _ = vmc.sweep(g, sp[c], 16, w["sketch"], 3, 11, c, 3, trace=tr)
        for bond, rho, _, acc in tr.rows:
            assert abs(ratio[c, bond] - rho) <= 2 * SPLIT["sweep_ratio_max"] * max(abs(rho), 1.0), (c, bond)
            assert int(acc) == int(dec[c, bond])
        assert np.array_equal(new, final[c])
    e, lp, sg = ctx.measure()
    for c in range(6):
        r = vmc.measure(g, final[c], 16, w["sketch"], 3, 1.0, 0.0)
        assert abs(e[c] - r["eloc"]) <= 2 * SPLIT["eloc_rel_scale_max"] * r["eloc_scale"], (c, e[c], r["eloc"])
        assert sg[c] == r["sign"] and abs(lp[c] - r["logpsi"]) <= 2 * SPLIT["logpsi_abs_max"]
        G = np.concatenate([x.ravel() for row in r["G"] for x in row])
        got = ctx.chain_grad(c)
        assert np.linalg.norm(got - G) <= 2 * SPLIT["grad_norm_max"] * np.linalg.norm(G)
        assert np.max(np.abs(got - G)) <= 2 * SPLIT["grad_elementwise_max"] * np.max(np.abs(G))
    ctx.close()
