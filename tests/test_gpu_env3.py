"""pepsvmc_env3_left, the batched three-line environment step (App. C), against the
oracle's env3_left on the same seeded float32-representable inputs."""
import numpy as np
import pytest

from oracle import vmc

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import api, build, inputs
    build.build()
    w = inputs.workload("peps_8x8", n_chains=64)
    ctx = api.PepsVMC(8, 8, 4, 16, 64, w["tensors"], w["sketch"], seed=1)
    yield ctx, torch
    ctx.close()


def case(dims, seed):
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    rng = np.random.default_rng(seed)
    f32 = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    return dict(E=f32(n, cT, Dl, cB), T=f32(n, cT, Du, cT2), A=f32(2, Dl, Dr, Du, Dd), B=f32(n, cB, Dd, cB2),
                spins=rng.choice(np.array([1, -1], dtype=np.int8), n))


def run_gpu(ctx, torch, c, dims):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    A_lurd = c["A"].transpose(0, 1, 3, 2, 4)  # the entry point takes each slot as (l, u, r, d)
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    out = torch.empty((n, cT2, Dr, cB2), dtype=torch.float32, device="cuda")
    ctx.env3_left(dev(c["E"]), dev(c["T"]), dev(A_lurd), dev(c["spins"]), dev(c["B"]), out, dims)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def reference(c, n):
    return np.stack([vmc.env3_left(c["E"][i].astype(np.float64), c["T"][i].astype(np.float64),
                                   c["A"][0 if c["spins"][i] > 0 else 1].astype(np.float64),
                                   c["B"][i].astype(np.float64)) for i in range(n)])


@pytest.mark.parametrize("dims", [(64, 16, 16, 16, 16, 4, 4, 4, 4), (37, 1, 1, 4, 3, 1, 4, 1, 4),
                                  (64, 16, 12, 16, 16, 4, 1, 4, 4), (5, 9, 7, 11, 13, 3, 2, 4, 2)])
def test_env3_left_matches_oracle(env, dims):
    ctx, torch = env
    c = case(dims, sum(dims))
    got = run_gpu(ctx, torch, c, dims)
    ref = reference(c, dims[0])
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


def test_env3_left_rejects_oversize(env):
    ctx, torch = env
    from paper_1908_09359_gb300 import PepsvmcError
    with pytest.raises(PepsvmcError):
        ctx.env3_left(1, 1, 1, 0, 1, 1, (65, 16, 16, 16, 16, 4, 4, 4, 4))
