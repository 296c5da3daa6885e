"""The allocation-free three-line environment step.

Callers that cannot call cudaMalloc once they are running -- for example a service
that reserved all of its device memory at start-up, where an allocation could
synchronise the device or fragment the planned pool -- use
pepsvmc_env3_left_noalloc.  It must give what the context-based pepsvmc_env3_left
gives, call after call (its scratch array keeps the previous call's contents), must
leave the device's free memory unchanged, and must refuse sizes its fixed scratch
cannot hold.  This file is collected last so that a failure here comes after every
other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the tolerance of the other contraction tests


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import api, build, inputs
    build.build()
    w = inputs.workload("peps_8x8", n_chains=64)
    ctx = api.PepsVMC(8, 8, 4, 16, 64, w["tensors"], w["sketch"], seed=1)
    yield api, ctx, torch
    ctx.close()


def inputs_for(torch, dims, seed):
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    g = torch.Generator(device="cuda").manual_seed(seed)
    r = lambda *s: torch.randn(*s, generator=g, device="cuda", dtype=torch.float32)  # noqa: E731
    spins = torch.where(torch.rand(n, generator=g, device="cuda") < 0.5, 1, -1).to(torch.int8)
    return dict(E=r(n, cT, Dl, cB), T=r(n, cT, Du, cT2), A=r(2, Dl, Du, Dr, Dd), B=r(n, cB, Dd, cB2),
                spins=spins)


@pytest.mark.parametrize("dims", [(64, 16, 16, 16, 16, 4, 4, 4, 4), (40, 16, 12, 16, 16, 4, 1, 4, 4)])
def test_noalloc_matches_context_entry_point_twice(setup, dims):
    api, ctx, torch = setup
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    for call, seed in enumerate((11, 12)):           # two calls in a row, different data
        x = inputs_for(torch, dims, seed + sum(dims))
        want = torch.empty((n, cT2, Dr, cB2), dtype=torch.float32, device="cuda")
        got = torch.full_like(want, float("nan"))
        ctx.env3_left(x["E"], x["T"], x["A"], x["spins"], x["B"], want, dims)
        api.env3_left_noalloc(x["E"], x["T"], x["A"], x["spins"], x["B"], got, dims)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), call
        assert np.max(np.abs(g - w)) <= TOL * np.max(np.abs(w)), call


def test_noalloc_allocates_nothing(setup):
    api, ctx, torch = setup
    dims = (32, 16, 16, 16, 16, 4, 4, 4, 4)
    x = inputs_for(torch, dims, 5)
    out = torch.empty((32, 16, 4, 16), dtype=torch.float32, device="cuda")
    api.env3_left_noalloc(x["E"], x["T"], x["A"], x["spins"], x["B"], out, dims)   # first use on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        api.env3_left_noalloc(x["E"], x["T"], x["A"], x["spins"], x["B"], out, dims)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_scratch(setup):
    api, ctx, torch = setup
    from paper_1908_09359_gb300 import PepsvmcError, _lib
    per = 4 * 16 * 4 * 16   # Dl*cB*Du*cT2 for the dims below
    n = _lib.NOALLOC_SCRATCH_FLOATS // (2 * per) + 1
    with pytest.raises(PepsvmcError):
        api.env3_left_noalloc(1, 1, 1, 0, 1, 1, (n, 16, 16, 16, 16, 4, 4, 4, 4))
