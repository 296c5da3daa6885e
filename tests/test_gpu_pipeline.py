"""The batched pipeline: CUDA-graph replay of the sample step and the autotuner.

A replayed step must do exactly what the eager step does (the same launches with the
same arguments), so samples, spins and gradients agree bit for bit; the autotuner only
chooses among kernels that compute the same products, so results agree within FP32
rounding (1e-5 relative on E_loc)."""
import numpy as np
import pytest

from paper_1908_09359_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import api as a
    from paper_1908_09359_gb300 import build
    build.build()
    return a


def run(api, graphs, autotune, precision=0, steps=3):
    w = inputs.workload("peps_8x8", n_chains=16)
    t = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
    ctx = api.PepsVMC(8, 8, 4, 16, 16, t, w["sketch"], seed=4, precision=precision)
    ctx.set_graphs(graphs)
    ctx.set_autotune(autotune)
    ctx.set_spins(inputs.start_spins(16, 8, 8, 7, "random"))
    r = ctx.energy_and_grad(steps)
    out = dict(r, spins=ctx.get_spins(), tuning=ctx.get_tuning(), launches=ctx.launches)
    ctx.close()
    return out


@pytest.mark.parametrize("precision", [0, 3])
def test_graph_replay_is_bitwise_identical(api, precision):
    a = run(api, graphs=False, autotune=False, precision=precision)
    b = run(api, graphs=True, autotune=False, precision=precision)
    assert np.array_equal(a["spins"], b["spins"])
    assert np.array_equal(a["eloc"], b["eloc"])
    assert np.array_equal(a["grad"], b["grad"])
    assert a["launches"] == b["launches"]


def test_autotuned_kernels_agree_within_fp32(api):
    a = run(api, graphs=False, autotune=False)
    b = run(api, graphs=True, autotune=True)
    assert len(b["tuning"]) > 5 and all(len(t["candidate_ms"]) >= 6 for t in b["tuning"])
    assert np.array_equal(a["spins"], b["spins"])
    scale = np.abs(a["eloc"]).max()
    assert np.max(np.abs(a["eloc"] - b["eloc"])) <= 1e-5 * scale
