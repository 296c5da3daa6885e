"""The tcgen05 tensor-core contraction path (MIXED_BF16 / MIXED_TF32) against the
oracle.  Operands are rounded to nearest BF16 (8-bit significand, unit roundoff 2^-9)
or TF32 (11-bit, 2^-11) with FP32 accumulation; a three-line step rounds the operands
of its three products (six roundings on the path of every term), so the norm-wise
error is a few unit roundoffs: bounds 1e-2 (BF16) and 3e-3 (TF32).  Split BF16 (x = hi +
lo, three products, lo*lo dropped) carries ~2^-16 per operand: bound 2e-4.  Element-wise,
every entry is held to the same bound relative to the largest entry of its step (an
entry is a sum of products whose rounding errors scale with the largest terms, not with
the entry itself, which may cancel)."""
import numpy as np
import pytest

from oracle import vmc

pytestmark = pytest.mark.gpu

TOL = {1: 1e-2, 2: 3e-3, 3: 2e-4}
EL_TOL = {1: 2e-2, 2: 6e-3, 3: 2e-4}  # element-wise, relative to the step's largest entry


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("dims", [(64, 16, 16, 16, 16, 4, 4, 4, 4), (48, 32, 32, 32, 32, 8, 8, 8, 8),
                                  (40, 24, 20, 24, 24, 6, 6, 6, 6), (33, 9, 7, 11, 13, 3, 2, 4, 2)])
def test_env3_tensor_cores_match_oracle(torch_mod, precision, dims):
    torch = torch_mod
    from paper_1908_09359_gb300 import api, inputs
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    D = max(Dl, Dr, Du, Dd)
    chi = max(cT, cB, cT2, cB2)
    w = inputs.workload("peps_8x8", n_chains=1)
    ctx = api.PepsVMC(8, 8, D, chi, n, inputs.peps_tensors(8, 8, D, 1), inputs.sketch(8, chi, D, 1),
                      seed=1, precision=precision)
    rng = np.random.default_rng(sum(dims) + precision)
    f32 = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    E, T, A, B = f32(n, cT, Dl, cB), f32(n, cT, Du, cT2), f32(2, Dl, Dr, Du, Dd), f32(n, cB, Dd, cB2)
    spins = rng.choice(np.array([1, -1], dtype=np.int8), n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = torch.empty((n, cT2, Dr, cB2), dtype=torch.float32, device="cuda")
    ctx.env3_left(dev(E), dev(T), dev(A.transpose(0, 1, 3, 2, 4)), dev(spins), dev(B), out, dims)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.stack([vmc.env3_left(E[i].astype(np.float64), T[i].astype(np.float64),
                                  A[0 if spins[i] > 0 else 1].astype(np.float64), B[i].astype(np.float64))
                    for i in range(n)])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL[precision], err
    for i in range(n):
        assert np.max(np.abs(got[i] - ref[i])) <= EL_TOL[precision] * np.max(np.abs(ref[i])), i
    ctx.close()


@pytest.mark.parametrize("precision,kind,bn", [(p, "tc", b) for p in (1, 2, 3) for b in (32, 64, 128, 256)]
                         + [(3, "tc2", 32), (3, "tc2", 64)])
def test_env3_every_tile_width_matches_oracle(torch_mod, precision, kind, bn):
    """Each tcgen05 kernel form and tile width fixed for all three products of the step
    (the autotuner would otherwise pick per shape), at the 24x24 bulk shapes with 300
    chains; "tc2" is the split-BF16 form with two shared-memory stages."""
    torch = torch_mod
    from paper_1908_09359_gb300 import api, inputs
    dims = (300, 32, 32, 32, 32, 8, 8, 8, 8)
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    ctx = api.PepsVMC(8, 8, 8, 32, n, inputs.peps_tensors(8, 8, 8, 1), inputs.sketch(8, 32, 8, 1),
                      seed=1, precision=precision)
    ctx.set_contraction_kernel(kind, bn)
    rng = np.random.default_rng(bn + precision)
    f32 = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    E, T, A, B = f32(n, cT, Dl, cB), f32(n, cT, Du, cT2), f32(2, Dl, Dr, Du, Dd), f32(n, cB, Dd, cB2)
    spins = rng.choice(np.array([1, -1], dtype=np.int8), n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = torch.empty((n, cT2, Dr, cB2), dtype=torch.float32, device="cuda")
    ctx.env3_left(dev(E), dev(T), dev(A.transpose(0, 1, 3, 2, 4)), dev(spins), dev(B), out, dims)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in list(range(0, n, 25)) + [n - 1]:
        ref = vmc.env3_left(E[i].astype(np.float64), T[i].astype(np.float64),
                            A[0 if spins[i] > 0 else 1].astype(np.float64), B[i].astype(np.float64))
        err = np.linalg.norm(got[i] - ref) / np.linalg.norm(ref)
        assert err <= TOL[precision], (i, err)
        assert np.max(np.abs(got[i] - ref)) <= EL_TOL[precision] * np.max(np.abs(ref)), i
    with pytest.raises(Exception):
        ctx.set_contraction_kernel("tc", 48)
    ctx.close()
