"""The gradient-sum exchange of a chain-sharded job through the C ABI, on one GPU: two
contexts holding chains 0-7 and 8-15 (chain offsets 0 and 8) against one context holding
all 16.  Per-chain results do not depend on the sharding; the sums of the shards add up
to the sums of the whole (up to float64 association); after writing the totals back
(pepsvmc_set_sums, or an in-place reduction of the device sums and
pepsvmc_finalize_sums) both shards apply the identical sign-SGD update, equal to the
whole job's wherever the gradient's sign is not decided by rounding."""
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


def make(api, w, n, offset):
    ctx = api.PepsVMC(8, 8, 4, 16, n, w["tensors"], w["sketch"], seed=w["seed"], chain_offset=offset)
    ctx.set_autotune(False)  # fixed kernel choices: per-chain results identical across contexts
    ctx.set_graphs(False)
    return ctx


@pytest.mark.parametrize("route", ["host", "device"])
def test_sharded_sums_and_update_match_the_whole_job(api, route):
    import torch

    from paper_1908_09359_gb300 import dist
    w = inputs.workload("peps_8x8", n_chains=16)
    whole = make(api, w, 16, 0)
    shards = [make(api, w, 8, 0), make(api, w, 8, 8)]
    whole.set_spins(w["spins"])
    shards[0].set_spins(w["spins"][:8])
    shards[1].set_spins(w["spins"][8:])
    rw = whole.energy_and_grad(2)
    rs = [s.energy_and_grad(2) for s in shards]
    el_w = rw["eloc"].reshape(2, 16)
    el_s = np.concatenate([r["eloc"].reshape(2, 8) for r in rs], axis=1)
    assert np.array_equal(el_w, el_s)
    assert np.array_equal(whole.get_spins(), np.concatenate([s.get_spins() for s in shards]))
    sw = whole.get_sums()
    parts = [s.get_sums() for s in shards]
    tot = [parts[0][i] + parts[1][i] for i in range(3)]
    assert tot[0][2] == 32.0
    for a, b in zip(tot, sw):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-13 * np.abs(b).max())
    if route == "host":
        for s in shards:
            s.set_sums(*tot)
    else:
        views = [dist.device_sums(s) for s in shards]
        torch.cuda.synchronize()
        totals = [views[0][i] + views[1][i] for i in range(3)]
        for v in views:
            for i in range(3):
                v[i].copy_(totals[i])
        torch.cuda.synchronize()
        for s in shards:
            s.finalize_sums()
    grad_w = rw["grad"]
    for s in shards:
        s.update(0.01, 5)
    whole.update(0.01, 5)
    t0, t1, tw = shards[0].get_tensors(), shards[1].get_tensors(), whole.get_tensors()
    assert np.array_equal(t0, t1)
    clear = np.abs(grad_w) > 1e-10 * np.abs(grad_w).max()
    assert np.array_equal(t0[clear], tw[clear])
    for c in shards + [whole]:
        c.close()
