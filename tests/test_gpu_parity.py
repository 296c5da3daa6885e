"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances (FP32 contractions against the FP64 oracle at equal Dc, same truncation
and the same configurations):
  * amplitude ratios and E_loc: 1e-5 relative; E_loc relative to the sum of the
    magnitudes of its terms, ratios relative to max(|ratio|, 1);
  * G = Delta/Psi and the energy gradient: 1e-4 relative, norm-wise per chain,
    and element-wise against 1e-4 of the largest entry;
  * ln|Psi|: 1e-4 absolute (Psi is a product over every truncated row, so its
    rounding error is larger than that of ratios, in which it cancels);
  * Metropolis decisions: identical except at near-ties |ln r - ln rho^2| < 1e-5,
    where the oracle takes the GPU's decision (it is then replaying the same chain);
  * spins and integer decisions: bit-exact; sign-SGD update: same float64 arithmetic.
"""
import numpy as np
import pytest

from oracle import exact, philox, vmc
from paper_1908_09359_gb300 import inputs

pytestmark = pytest.mark.gpu

RATIO_TOL = 1e-5
ELOC_TOL = 1e-5
GRAD_TOL = 1e-4
LOGPSI_TOL = 1e-4


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    from paper_1908_09359_gb300 import api as a
    return a


def ctx_for(api, w, n_chains, n_fit=3, seed=5):
    return api.PepsVMC(w["Ly"], w["Lx"], w["D"], w["chi"], n_chains, w["tensors"], w["sketch"],
                       J1=w["J1"], J2=w["J2"], seed=seed, n_fit=n_fit)


def small_workload(Ly, Lx, D, chi, J2=0.0, seed=1, normalise=False):
    return dict(Ly=Ly, Lx=Lx, D=D, chi=chi, J1=1.0, J2=J2,
                tensors=inputs.peps_tensors(Ly, Lx, D, seed, normalise),
                sketch=inputs.sketch(max(Ly, Lx), chi, D, seed))


def grid_of(w):
    return vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])


def flat_G(G):
    return np.concatenate([g.ravel() for row in G for g in row])


def check_grad(g, ref, tol=GRAD_TOL):
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err <= tol, err
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))
    return err


# ------------------------------------------------------------------- amplitudes (a2, a3)

def test_amplitude_exact_dc_matches_brute_force(api):
    """4x4, D=2, Dc=4 = D^(L/2): every row's contraction equals Psi by brute force."""
    w = small_workload(4, 4, 2, 4, seed=3)
    g = grid_of(w)
    sp = inputs.start_spins(8, 4, 4, 11, "random")
    ctx = ctx_for(api, w, 8)
    ctx.set_spins(sp)
    ref = np.array([exact.amplitude_transfer(g, c) for c in sp])
    for row in range(4):
        lp, sg = ctx.amplitude(row)
        assert np.all(sg == np.sign(ref))
        assert np.allclose(lp, np.log(np.abs(ref)), rtol=0, atol=1e-5)
    ctx.close()


@pytest.mark.parametrize("row", [0, 3, 7])
def test_amplitude_parity_finite_dc(api, row):
    """8x8, D=4, Dc=16 (truncated): Psi of chosen chains equals the oracle's."""
    w = inputs.workload("peps_8x8", n_chains=16)
    g = grid_of(w)
    ctx = ctx_for(api, w, 16)
    ctx.set_spins(w["spins"])
    lp, sg = ctx.amplitude(row)
    for c in (0, 9, 15):
        s = w["spins"][c]
        Ts, lT = vmc.top_envs(g, s, w["chi"], w["sketch"], 3)
        Bs, lB = vmc.bottom_envs(g, s, w["chi"], w["sketch"], 3)
        ref, rsg = vmc.row_psi(Ts[row], vmc.row_tensors(g, s, row), Bs[row], lT[row], lB[row])
        assert sg[c] == rsg
        assert abs(lp[c] - ref) <= LOGPSI_TOL, (c, lp[c], ref)
    ctx.close()


# ------------------------------------------------------------ measurement (a6, a7, a8)

@pytest.mark.parametrize("case", ["4x4_exact", "8x8_heisenberg", "6x6_j1j2"])
def test_measure_parity(api, case):
    if case == "4x4_exact":
        w, chains = small_workload(4, 4, 2, 4, seed=8), [0, 1, 2, 3]
        n = 4
    elif case == "8x8_heisenberg":
        w, chains = inputs.workload("peps_8x8", n_chains=8), [0, 5]
        n = 8
    else:
        w, chains = small_workload(6, 6, 3, 9, J2=0.5, seed=4), [0, 2]
        n = 4
    g = grid_of(w)
    sp = inputs.start_spins(n, w["Ly"], w["Lx"], 21, "random")
    ctx = ctx_for(api, w, n)
    ctx.set_spins(sp)
    e, lp, sg = ctx.measure()
    for c in chains:
        r = vmc.measure(g, sp[c], w["chi"], w["sketch"], 3, w["J1"], w["J2"])
        assert abs(e[c] - r["eloc"]) <= ELOC_TOL * r["eloc_scale"], (c, e[c], r["eloc"])
        assert sg[c] == r["sign"]
        assert abs(lp[c] - r["logpsi"]) <= LOGPSI_TOL
        check_grad(ctx.chain_grad(c), flat_G(r["G"]))
    ctx.close()


# ------------------------------------------------------------------ sampler (a4, a5)

def test_sweep_parity_with_decisions(api):
    """One sequential sweep on 8x8 (Dc=16): every proposal's ratio matches the oracle,
    every decision matches except at near-ties, the final spins are identical."""
    w = inputs.workload("peps_8x8", n_chains=6)
    g = grid_of(w)
    seed, t = 77, 3
    ctx = ctx_for(api, w, 6, seed=seed)
    ctx.set_spins(w["spins"])
    ctx.set_sweep_counter(t)
    ctx.enable_trace(True)
    ctx.sample_sweep(1)
    ratio, dec = ctx.get_trace()
    final = ctx.get_spins()
    worst, ties, props = 0.0, 0, 0
    for c in (0, 3, 5):
        follow = {b: int(dec[c, b]) for b in range(ctx.n_bonds) if dec[c, b] >= 0}
        tr = vmc.Trace(follow=follow, tie=1e-5)
        new, _, _ = vmc.sweep(g, w["spins"][c], w["chi"], w["sketch"], 3, seed, c, t, trace=tr)
        for bond, rho, u, acc in tr.rows:
            props += 1
            assert dec[c, bond] >= 0, "GPU made no proposal where the oracle did"
            worst = max(worst, abs(ratio[c, bond] - rho) / max(abs(rho), 1.0))
            if abs(np.log(max(u, 1e-300)) - np.log(rho * rho)) < 1e-5:
                ties += 1
            assert int(acc) == int(dec[c, bond]), (c, bond, rho, ratio[c, bond], u)
        assert np.count_nonzero(dec[c] >= 0) == len(tr.rows)
        assert np.array_equal(new, final[c])
        assert int(final[c].sum()) == 0
    assert props > 0
    assert worst <= RATIO_TOL, worst
    ctx.close()


def test_metropolis_uniforms_are_philox(api):
    """The GPU's decisions are reproduced from the oracle's Philox uniforms alone
    (no ties): accept iff r < min(1, ratio^2) with r = Philox(chain, sweep, bond)."""
    w = small_workload(4, 4, 2, 4, seed=13)
    ctx = ctx_for(api, w, 32, seed=991)
    ctx.set_spins(inputs.start_spins(32, 4, 4, 2, "random"))
    ctx.set_sweep_counter(12)
    ctx.enable_trace(True)
    ctx.sample_sweep(1)
    ratio, dec = ctx.get_trace()
    n = 0
    for c in range(32):
        for b in range(ctx.n_bonds):
            if dec[c, b] < 0:
                continue
            u = philox.metropolis_uniform(991, c, 12, b)
            if abs(np.log(u) - np.log(ratio[c, b] ** 2)) < 1e-6:
                continue
            assert int(dec[c, b]) == int(u < min(1.0, ratio[c, b] ** 2))
            n += 1
    assert n > 100
    ctx.close()


# --------------------------------------------------------- gradient and update (a9, a10)

def test_energy_and_grad_and_update_parity(api):
    w = inputs.workload("peps_8x8", n_chains=4)
    g = grid_of(w)
    seed = 31
    ctx = ctx_for(api, w, 4, seed=seed)
    ctx.set_spins(w["spins"])
    ctx.set_sweep_counter(0)
    r = ctx.energy_and_grad(1)
    after = ctx.get_spins()
    acc = vmc.Accumulator(g)
    scale = []
    for c in range(4):
        m = vmc.measure(g, after[c], w["chi"], w["sketch"], 3, w["J1"], w["J2"])
        assert abs(r["eloc"][c] - m["eloc"]) <= ELOC_TOL * m["eloc_scale"]
        acc.add(after[c], m["eloc"], m["G"])
        scale.append(m["eloc_scale"])
    grad_ref, E = acc.gradient()
    assert abs(r["E_mean"] - E) <= ELOC_TOL * np.mean(scale)
    check_grad(r["grad"], vmc.pack(grad_ref))
    t0 = ctx.get_tensors()
    ctx.update(0.01, step=7)
    t1 = ctx.get_tensors()
    ref = vmc.sign_sgd(t0, r["grad"], 0.01, seed, 7)
    assert np.array_equal(t1, ref) or np.max(np.abs(t1 - ref)) <= 1e-15
    ctx.close()


# ------------------------------------------------ full-size launch, sampled outputs

@pytest.mark.parametrize("name,chains", [("peps_8x8", (0, 1023)), ("peps_24x24", (0,))])
def test_full_size_sampled_parity(api, name, chains):
    """The bench's launch configuration (all chains of the workload in one context);
    the oracle recomputes sampled chains one by one."""
    w = inputs.workload(name)
    g = grid_of(w)
    ctx = ctx_for(api, w, w["n_chains"])
    ctx.set_spins(w["spins"])
    e, lp, sg = ctx.measure()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(lp))
    for c in chains:
        r = vmc.measure(g, w["spins"][c], w["chi"], w["sketch"], 3, w["J1"], w["J2"], want_grad=False)
        assert abs(e[c] - r["eloc"]) <= ELOC_TOL * r["eloc_scale"], (c, e[c], r["eloc"])
        assert sg[c] == r["sign"]
        assert abs(lp[c] - r["logpsi"]) <= LOGPSI_TOL * max(1.0, abs(r["logpsi"]) / 100.0)
    ctx.close()
