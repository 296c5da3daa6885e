"""The fused three-line column step (App. C, Fig. "contraction" (c)): all three products
in one tcgen05 kernel with the intermediates on chip, against the FP64 oracle element by
element and against the same precision computed as three separate products.

Error model (per operand: BF16 unit roundoff 2^-9; split BF16 x = hi + lo carries
2^-18 per operand plus the dropped lo*lo term, ~2^-17 per product): every output entry
is a sum of products of four operands through three roundings to the operand type, so
its error is a few unit roundoffs of the largest terms entering it.  Bounds, relative to
the largest entry of the step: split BF16 2e-4 element-wise and norm-wise; BF16 2e-2
element-wise, 1e-2 norm-wise.
"""
import numpy as np
import pytest

from oracle import vmc
from paper_1908_09359_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {1: (2e-2, 1e-2), 3: (2e-4, 2e-4)}  # precision: (element-wise vs max |ref|, norm-wise)


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    return torch


def step(torch, ctx, dims, seed, fused=True):
    n, cT, cB, cT2, cB2, Dl, Dr, Du, Dd = dims
    rng = np.random.default_rng(seed)
    f32 = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    E, T, A, B = f32(n, cT, Dl, cB), f32(n, cT, Du, cT2), f32(2, Dl, Dr, Du, Dd), f32(n, cB, Dd, cB2)
    spins = rng.choice(np.array([1, -1], dtype=np.int8), n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = torch.full((n, cT2, Dr, cB2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.set_fused(fused)
    ctx.env3_left(dev(E), dev(T), dev(A.transpose(0, 1, 3, 2, 4)), dev(spins), dev(B), out, dims)
    torch.cuda.synchronize()
    return dict(E=E, T=T, A=A, B=B, spins=spins), out.cpu().numpy()


def oracle_step(c, i):
    return vmc.env3_left(c["E"][i].astype(np.float64), c["T"][i].astype(np.float64),
                         c["A"][0 if c["spins"][i] > 0 else 1].astype(np.float64), c["B"][i].astype(np.float64))


@pytest.mark.parametrize("precision", [3, 1])
@pytest.mark.parametrize("dims", [
    (300, 32, 32, 32, 32, 8, 8, 8, 8),   # 24x24 bulk column: four a' tiles, one CTA per chain
    (64, 16, 16, 16, 16, 4, 4, 4, 4),    # 8x8 bulk column, zero-padded on chip
    (17, 32, 32, 20, 32, 8, 8, 8, 8),    # ragged last a' tile
    (33, 9, 7, 11, 13, 3, 2, 4, 2),      # every bond different and ragged
    (37, 1, 1, 4, 3, 1, 4, 1, 4),        # left edge of a top row (trivial legs)
    (5, 24, 24, 24, 24, 6, 6, 6, 6),     # 16x16 bulk shapes
])
def test_fused_env3_matches_oracle_elementwise(torch_mod, precision, dims):
    from paper_1908_09359_gb300 import api
    n = dims[0]
    D, chi = max(dims[5:]), max(dims[1:5])
    ctx = api.PepsVMC(8, 8, D, chi, n, inputs.peps_tensors(8, 8, D, 1), inputs.sketch(8, chi, D, 1),
                      seed=1, precision=precision)
    ctx.set_profiling(True)
    c, got = step(torch_mod, ctx, dims, sum(dims) + precision)
    shapes = [r["shape"] for r in ctx.get_profile_shapes()]
    assert any(s.startswith("fused3") for s in shapes), shapes
    el_tol, nrm_tol = TOL[precision]
    for i in sorted(set(list(range(0, n, max(1, n // 12))) + [n - 1])):
        ref = oracle_step(c, i)
        assert np.all(np.isfinite(got[i])), i
        assert np.max(np.abs(got[i] - ref)) <= el_tol * np.max(np.abs(ref)), i
        assert np.linalg.norm(got[i] - ref) <= nrm_tol * np.linalg.norm(ref), i
    ctx.close()


def test_fused_equals_separate_products_within_rounding(torch_mod):
    """The fused step and the three separate tensor-core products (split BF16) compute the
    same contraction in another rounding order."""
    from paper_1908_09359_gb300 import api
    dims = (152, 32, 32, 32, 32, 8, 8, 8, 8)
    ctx = api.PepsVMC(8, 8, 8, 32, 152, inputs.peps_tensors(8, 8, 8, 1), inputs.sketch(8, 32, 8, 1),
                      seed=1, precision=3)
    _, fused = step(torch_mod, ctx, dims, 7, fused=True)
    _, sep = step(torch_mod, ctx, dims, 7, fused=False)
    scale = np.max(np.abs(sep), axis=(1, 2, 3))
    assert np.all(np.max(np.abs(fused - sep), axis=(1, 2, 3)) <= 4e-4 * scale)
    ctx.close()


def test_fused_whole_path_matches_oracle(torch_mod):
    """Sweep and measurement of the 8x8 shapes in split BF16 with the fused steps (bond
    spectra lambda_i = exp(-i)): E_loc, ln|Psi| and G against the oracle, and the sweep's
    decisions against the separate-product form."""
    from paper_1908_09359_gb300 import api
    w = inputs.workload("peps_8x8", n_chains=8)
    w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    sp = inputs.start_spins(8, 8, 8, 21, "random")
    ctx = api.PepsVMC(8, 8, 4, 16, 8, w["tensors"], w["sketch"], seed=3, precision=3)
    ctx.set_spins(sp)
    ctx.set_profiling(True)
    e, lp, sg = ctx.measure()
    assert any(r["shape"].startswith("fused3") for r in ctx.get_profile_shapes())
    for c in range(0, 8, 2):
        r = vmc.measure(g, sp[c], 16, w["sketch"], 3, 1.0, 0.0)
        assert abs(e[c] - r["eloc"]) <= 5e-4 * r["eloc_scale"], (c, e[c], r["eloc"])
        assert sg[c] == r["sign"] and abs(lp[c] - r["logpsi"]) <= 5e-3
        G = np.concatenate([x.ravel() for row in r["G"] for x in row])
        assert np.linalg.norm(ctx.chain_grad(c) - G) <= 1e-3 * np.linalg.norm(G)
    dec = {}
    for fused in (True, False):
        ctx.set_fused(fused)
        ctx.set_spins(sp)
        ctx.set_sweep_counter(4)
        ctx.enable_trace(True)
        ctx.sample_sweep(1)
        dec[fused] = ctx.get_trace()[1]
    assert np.mean(dec[True] == dec[False]) >= 0.99
    ctx.close()


# ------------------------------------------------------------------ four-line step

def step4(torch, ctx, dims, seed, fused=True, bmajor=False):
    n, cT, cB, cT2, cB2, D1l, D1r, Du1, Dd1, D2l, D2r, Dd2 = dims
    rng = np.random.default_rng(seed)
    f32 = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    c = dict(E=f32(n, cT, D1l, D2l, cB), T=f32(n, cT, Du1, cT2), A1=f32(2, D1l, D1r, Du1, Dd1),
             A2=f32(2, D2l, D2r, Dd1, Dd2), B=f32(n, cB, Dd2, cB2),
             s1=rng.choice(np.array([1, -1], dtype=np.int8), n), s2=rng.choice(np.array([1, -1], dtype=np.int8), n))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ctx.set_fused(fused)
    if bmajor:  # E at [b][a][l1][l2], out at [b'][a'][r1][r2]
        out = torch.full((n, cB2, cT2, D1r, D2r), float("nan"), dtype=torch.float32, device="cuda")
        ctx.env4_left(dev(c["E"].transpose(0, 4, 1, 2, 3)), dev(c["T"]), dev(c["A1"].transpose(0, 1, 3, 2, 4)),
                      dev(c["s1"]), dev(c["A2"].transpose(0, 1, 3, 2, 4)), dev(c["s2"]), dev(c["B"]), out, dims,
                      bmajor=True)
        torch.cuda.synchronize()
        return c, out.cpu().numpy().transpose(0, 2, 3, 4, 1)
    out = torch.full((n, cT2, D1r, D2r, cB2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.env4_left(dev(c["E"]), dev(c["T"]), dev(c["A1"].transpose(0, 1, 3, 2, 4)), dev(c["s1"]),
                  dev(c["A2"].transpose(0, 1, 3, 2, 4)), dev(c["s2"]), dev(c["B"]), out, dims)
    torch.cuda.synchronize()
    return c, out.cpu().numpy()


def oracle_step4(c, i):
    f = lambda a: a.astype(np.float64)  # noqa: E731
    return vmc.env4_left(f(c["E"][i]), f(c["T"][i]), f(c["A1"][0 if c["s1"][i] > 0 else 1]),
                         f(c["A2"][0 if c["s2"][i] > 0 else 1]), f(c["B"][i]))


@pytest.mark.parametrize("bmajor", [False, True])
@pytest.mark.parametrize("precision", [3, 1])
@pytest.mark.parametrize("dims", [
    (160, 32, 32, 32, 32, 8, 8, 8, 8, 8, 8, 8),   # 24x24 bulk row pair: four a' tiles, 16 b tiles
    (40, 16, 16, 16, 16, 4, 4, 4, 4, 4, 4, 4),    # 8x8 bulk, zero-padded on chip
    (9, 32, 31, 27, 30, 8, 8, 8, 8, 8, 8, 8),     # ragged last a' and b tiles
    (11, 9, 7, 11, 13, 3, 2, 4, 2, 3, 2, 2),      # every bond different
    (13, 1, 1, 4, 3, 1, 4, 1, 4, 1, 4, 4),        # left edge of the top row pair
])
def test_fused_env4_matches_oracle_elementwise(torch_mod, precision, dims, bmajor):
    from paper_1908_09359_gb300 import api
    n = dims[0]
    D, chi = max(dims[5:]), max(dims[1:5])
    ctx = api.PepsVMC(8, 8, D, chi, n, inputs.peps_tensors(8, 8, D, 1), inputs.sketch(8, chi, D, 1),
                      seed=1, precision=precision)
    c, got = step4(torch_mod, ctx, dims, sum(dims) + precision, bmajor=bmajor)
    el_tol, nrm_tol = TOL[precision]
    for i in sorted(set(list(range(0, n, max(1, n // 6))) + [n - 1])):
        ref = oracle_step4(c, i)
        assert np.all(np.isfinite(got[i])), i
        assert np.max(np.abs(got[i] - ref)) <= el_tol * np.max(np.abs(ref)), i
        assert np.linalg.norm(got[i] - ref) <= nrm_tol * np.linalg.norm(ref), i
    ctx.close()


def test_fused_env4_equals_separate_products_within_rounding(torch_mod):
    from paper_1908_09359_gb300 import api
    dims = (152, 32, 32, 32, 32, 8, 8, 8, 8, 8, 8, 8)
    ctx = api.PepsVMC(8, 8, 8, 32, 152, inputs.peps_tensors(8, 8, 8, 1), inputs.sketch(8, 32, 8, 1),
                      seed=1, precision=3)
    _, fused = step4(torch_mod, ctx, dims, 5, fused=True)
    _, sep = step4(torch_mod, ctx, dims, 5, fused=False)
    scale = np.max(np.abs(sep), axis=(1, 2, 3, 4))
    assert np.all(np.max(np.abs(fused - sep), axis=(1, 2, 3, 4)) <= 4e-4 * scale)
    ctx.close()


def test_fused_j1j2_measurement_matches_oracle(torch_mod):
    """E_loc of the J1-J2 model (vertical and diagonal terms from the fused four-line
    steps) at 6x6, D = 3, Dc = 9 on tensors with bond spectra exp(-i), split BF16."""
    from paper_1908_09359_gb300 import api
    t = inputs.peps_tensors(6, 6, 3, 4, False, bond_decay=1.0)
    sk = inputs.sketch(6, 9, 3, 4)
    g = vmc.unpack(t, 6, 6, 3)
    sp = inputs.start_spins(4, 6, 6, 21, "random")
    ctx = api.PepsVMC(6, 6, 3, 9, 4, t, sk, J1=1.0, J2=0.5, seed=3, precision=3)
    ctx.set_spins(sp)
    ctx.set_profiling(True)
    e, lp, sg = ctx.measure()
    assert any(r["shape"].startswith("fused4") for r in ctx.get_profile_shapes())
    for c in range(4):
        r = vmc.measure(g, sp[c], 9, sk, 3, 1.0, 0.5)
        assert abs(e[c] - r["eloc"]) <= 5e-4 * r["eloc_scale"], (c, e[c], r["eloc"])
        G = np.concatenate([x.ravel() for row in r["G"] for x in row])
        assert np.linalg.norm(ctx.chain_grad(c) - G) <= 1e-3 * np.linalg.norm(G)
    ctx.close()
