"""Failure statuses of the C ABI (the conventions of include/pepsvmc.h): every one is
produced here on the host or by a bounded device wait, never by a GPU fault.

* ETIMEOUT: a context whose device wait budget is one clock cycle; the first wait of a
  tensor-core product expires, the kernel records the status, lets its products in
  flight finish (with the default budget), frees its tensor memory and returns; the call
  returns ETIMEOUT and the context works again once the budget is restored.
* ENONFINITE: a NaN written into the tensors by the host.
* EZEROPSI: a spin slot of a site set to zero on the host while every chain uses it, so
  Psi(S) = 0 exactly (the root cause is reported even though 0/0 follows downstream).
"""
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


def ctx_8x8(api, precision, **kw):
    w = inputs.workload("peps_8x8", n_chains=16)
    ctx = api.PepsVMC(8, 8, 4, 16, 16, w["tensors"], w["sketch"], seed=3, precision=precision, **kw)
    ctx.set_autotune(False)  # fixed kernel choices: two contexts compute bit-identical results
    ctx.set_spins(w["spins"])
    return ctx, w


@pytest.mark.parametrize("form", ["fused", "separate"])
def test_expired_device_wait_returns_etimeout_and_context_recovers(api, form):
    from paper_1908_09359_gb300 import PepsvmcError, _lib
    ref, w = ctx_8x8(api, 3)
    if form == "separate":
        ref.set_contraction_kernel("tc", 64)
    e_ref, lp_ref, _ = ref.measure()
    ctx, _ = ctx_8x8(api, 3, wait_budget_cycles=1)
    if form == "separate":
        ctx.set_contraction_kernel("tc", 64)
    with pytest.raises(PepsvmcError) as err:
        ctx.measure()
    assert err.value.code == _lib.ETIMEOUT
    with pytest.raises(PepsvmcError) as err:
        ctx.sample_sweep(1)
    assert err.value.code == _lib.ETIMEOUT
    ctx.set_wait_budget(0)
    ctx.set_spins(w["spins"])
    e, lp, _ = ctx.measure()
    assert np.array_equal(e, e_ref) and np.array_equal(lp, lp_ref)
    ctx.close()
    ref.close()


@pytest.mark.parametrize("precision", [0, 3])
def test_nan_tensor_returns_enonfinite(api, precision):
    from paper_1908_09359_gb300 import PepsvmcError, _lib
    ctx, w = ctx_8x8(api, precision)
    bad = w["tensors"].copy()
    bad[len(bad) // 2] = np.nan
    ctx.set_tensors(bad)
    with pytest.raises(PepsvmcError) as err:
        ctx.measure()
    assert err.value.code == _lib.ENONFINITE
    ctx.set_tensors(w["tensors"])
    e, lp, _ = ctx.measure()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(lp))
    ctx.close()


@pytest.mark.parametrize("precision", [0, 3])
def test_zero_amplitude_returns_ezeropsi(api, precision):
    from paper_1908_09359_gb300 import PepsvmcError, _lib
    ctx, w = ctx_8x8(api, precision)
    # site (0,0) has shape (2, 1, D, 1, D); zero its spin-up slot and put every chain's
    # spin (0,0) up (its down partner elsewhere keeps S^z = 0)
    D = 4
    bad = w["tensors"].copy()
    bad[:D * D] = 0.0
    sp = inputs.start_spins(16, 8, 8, 5, "neel")
    assert np.all(sp[:, 0, 0] == 1)
    ctx.set_tensors(bad)
    ctx.set_spins(sp)
    with pytest.raises(PepsvmcError) as err:
        ctx.measure()
    assert err.value.code == _lib.EZEROPSI
    with pytest.raises(PepsvmcError) as err:
        ctx.sample_sweep(1)
    assert err.value.code == _lib.EZEROPSI
    ctx.set_tensors(w["tensors"])
    e, _, _ = ctx.measure()
    assert np.all(np.isfinite(e))
    ctx.close()
