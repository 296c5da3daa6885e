"""Spin-inversion symmetrised sampling and measurement on the GPU against the oracle
(Phi(S) = Psi(S) + Psi(S-bar), end of Sec. II B; oracle/spin_inversion.py).

Chains p and p + P of a symmetrised context hold S and S-bar.  Checked through the C ABI:
one traced sweep (both chains' ratios against the oracle's rho and rho-bar, one decision
per pair, final pairs still inverted), E^Phi and w of a measurement, the |Phi|^2-weighted
gradient of a whole sample step with its sign-SGD update, and at exact Dc on 4x4 the mean
of E^Phi over long runs against <Phi|H|Phi>/<Phi|Phi> from the S^z = 0 enumeration.

Tolerances.  The ratios and E_loc, ln|Psi| and G of each configuration carry the FP32
errors bounded in tests/test_gpu_parity.py (twice the float32 spread of the oracle in
six rounding orders, tests/golden/float32_spread.json).  w = exp(lnPsi(S-bar) -
lnPsi(S)) then has relative error <= 2 LOGPSI_TOL, and E^Phi = (E + w E-bar)/(1 + w)
has error <= [ELOC_TOL (scale(S) + |w| scale(S-bar)) + |E-bar - E^Phi| |dw|] / |1 + w|.
Decisions near a tie (|ln u - ln q| below the FP32 uncertainty of ln q, 1e-4 here since w
enters q) follow the GPU's decision.
"""
import json
import os

import numpy as np
import pytest

from oracle import exact, spin_inversion, vmc
from paper_1908_09359_gb300 import autocorr, inputs

pytestmark = pytest.mark.gpu

ELOC_TOL = 1e-5
LOGPSI_TOL = 1e-4
GRAD_TOL = 1e-4
TIE = 1e-4
_SPREAD = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "float32_spread.json")))
RATIO_TOL_SWEEP = 2 * _SPREAD["sweep_ratios_bond_decay_8x8"]["max"]


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    from paper_1908_09359_gb300 import api as a
    return a


def structured_8x8(J2=0.5):
    """The 8x8 shapes (D = 4, Dc = 16) with simple-update-like bond spectra."""
    w = inputs.workload("peps_8x8", n_chains=6)
    w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], w["normalise"], bond_decay=1.0)
    w["J2"] = J2
    return w


def pairs_of(sp):
    return np.concatenate([sp, -sp]).astype(np.int8)


def make_ctx(api, w, n_pairs, seed, precision=0):
    return api.PepsVMC(w["Ly"], w["Lx"], w["D"], w["chi"], 2 * n_pairs, w["tensors"], w["sketch"],
                       J1=w["J1"], J2=w["J2"], seed=seed, n_fit=3, precision=precision, symmetrize=True)


def test_symmetrised_sweep_parity(api):
    """One sweep of three S, S-bar pairs on the 8x8 shapes (Dc = 16, J2 = 0.5): both chains'
    ratios match the oracle's rho and rho-bar, each pair takes the oracle's decision
    (near-ties excepted), and every final S-bar is still the inversion of its S."""
    w = structured_8x8()
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    P, seed, t = 3, 91, 4
    start = inputs.start_spins(P, 8, 8, 17, "random")
    ctx = make_ctx(api, w, P, seed)
    ctx.set_spins(pairs_of(start))
    ctx.set_sweep_counter(t)
    ctx.enable_trace(True)
    rate = ctx.sample_sweep(1)
    ratio, dec = ctx.get_trace()
    final = ctx.get_spins()
    assert np.array_equal(final[P:], -final[:P])
    assert 0.0 < rate < 1.0
    dev = []
    for p in range(P):
        assert np.array_equal(dec[p], dec[p + P])
        follow = {b: int(dec[p, b]) for b in range(ctx.n_bonds) if dec[p, b] >= 0}
        tr = spin_inversion.PairTrace(follow=follow, tie=TIE)
        new = spin_inversion.sweep(g, start[p], w["chi"], w["sketch"], 3, seed, p, t, trace=tr)
        for bond, rho, rho_b, wv, u, acc in tr.rows:
            dev.append(abs(ratio[p, bond] - rho) / max(abs(rho), 1.0))
            dev.append(abs(ratio[p + P, bond] - rho_b) / max(abs(rho_b), 1.0))
            assert int(acc) == int(dec[p, bond]), (p, bond, rho, rho_b, wv, u)
        assert np.count_nonzero(dec[p] >= 0) == len(tr.rows)
        assert np.array_equal(new, final[p])
    assert max(dev) <= RATIO_TOL_SWEEP, max(dev)
    ctx.close()


def test_symmetrised_measure_parity(api):
    """E^Phi and w of every pair against the oracle (8x8 shapes, J2 = 0.5)."""
    w = structured_8x8()
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    P = 3
    sp = inputs.start_spins(P, 8, 8, 29, "random")
    ctx = make_ctx(api, w, P, 5)
    ctx.set_spins(pairs_of(sp))
    e, lp, sg = ctx.measure()
    ephi, wv = ctx.phi()
    for p in range(P):
        r = spin_inversion.measure(g, sp[p], w["chi"], w["sketch"], 3, w["J1"], w["J2"], want_grad=False)
        dw = 2 * LOGPSI_TOL * abs(r["w"])
        assert abs(wv[p] - r["w"]) <= dw, (p, wv[p], r["w"])
        bound = (ELOC_TOL * (r["plain"]["eloc_scale"] + abs(r["w"]) * r["bar"]["eloc_scale"])
                 + abs(r["eloc_bar"] - r["eloc_phi"]) * dw) / abs(1.0 + r["w"])
        assert abs(ephi[p] - r["eloc_phi"]) <= bound, (p, ephi[p], r["eloc_phi"], bound)
        assert abs(e[p] - r["eloc"]) <= ELOC_TOL * r["plain"]["eloc_scale"]
        assert abs(e[p + P] - r["eloc_bar"]) <= ELOC_TOL * r["bar"]["eloc_scale"]
    ctx.close()


def test_symmetrised_step_gradient_and_update(api):
    """energy_and_grad(1) of three pairs: the gradient of <Phi|H|Phi>/<Phi|Phi> from the
    |Phi|^2-weighted sums matches the oracle's accumulation over the same final pairs,
    E_mean is the mean of E^Phi over pairs, and sign-SGD follows the GPU's gradient."""
    w = structured_8x8()
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    P, seed = 3, 13
    ctx = make_ctx(api, w, P, seed)
    ctx.set_spins(pairs_of(inputs.start_spins(P, 8, 8, 41, "random")))
    ctx.set_sweep_counter(2)
    r = ctx.energy_and_grad(1)
    after = ctx.get_spins()
    assert np.array_equal(after[P:], -after[:P])
    acc = spin_inversion.Accumulator(g)
    scale = []
    for p in range(P):
        m = spin_inversion.measure(g, after[p], w["chi"], w["sketch"], 3, w["J1"], w["J2"])
        acc.add(m)
        scale.append(m["scale"] / abs(1.0 + m["w"]))
        assert r["eloc"][p] == r["eloc"][p + P]
    grad_ref, E = acc.gradient()
    assert abs(r["E_mean"] - E) <= 10 * ELOC_TOL * np.mean(scale)
    ref = vmc.pack(grad_ref)
    assert np.linalg.norm(r["grad"] - ref) <= GRAD_TOL * np.linalg.norm(ref)
    t0 = ctx.get_tensors()
    ctx.update(0.01, step=3)
    assert np.max(np.abs(ctx.get_tensors() - vmc.sign_sgd(t0, r["grad"], 0.01, seed, 3))) <= 1e-15
    ctx.close()


def test_symmetrised_split_bf16_runs_and_agrees(api):
    """The bench's precision (split BF16, fused column steps) in symmetrised mode: a sample
    step runs and keeps the pairs inverted, and E^Phi of a measurement agrees with the
    oracle's within the split-BF16 bounds of the 8x8 shapes (twice the oracle's own
    deviation in emulated split BF16, propagated through w as above)."""
    split = _SPREAD["split_bf16_bond_decay_8x8"]
    w = structured_8x8(J2=0.0)   # the couplings the split-BF16 bounds were derived at
    P = 3
    sp = pairs_of(inputs.start_spins(P, 8, 8, 57, "random"))
    out = {}
    for precision in (0, 3):
        ctx = make_ctx(api, w, P, 7, precision)
        ctx.set_spins(sp)
        ctx.measure()
        out[precision] = ctx.phi()
        ctx.set_spins(sp)
        ctx.energy_and_grad(1, want_samples=False)
        assert np.array_equal(ctx.get_spins()[P:], -ctx.get_spins()[:P])
        ctx.close()
    g = vmc.unpack(w["tensors"], 8, 8, 4)
    for p in range(P):
        r = spin_inversion.measure(g, sp[p], w["chi"], w["sketch"], 3, w["J1"], w["J2"], want_grad=False)
        dw = 2 * split["logpsi_abs_max"] * 2 * abs(r["w"])
        bound = (2 * split["eloc_rel_scale_max"] * (r["plain"]["eloc_scale"] + abs(r["w"]) * r["bar"]["eloc_scale"])
                 + abs(r["eloc_bar"] - r["eloc_phi"]) * dw) / abs(1.0 + r["w"])
        assert abs(out[3][0][p] - r["eloc_phi"]) <= bound, (p, out[3][0][p], r["eloc_phi"], bound)


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_mean_eloc_phi_matches_exact_symmetrised_energy(api, J2):
    """4x4, D = 2, exact Dc: the mean of E^Phi over 1024 pairs x 60 sweeps equals
    <Phi|H|Phi>/<Phi|Phi> from the S^z = 0 enumeration within five tau-corrected standard
    errors.  (That the chains follow |Phi|^2 and not |Psi|^2 is pinned decision by decision
    by the sweep parity test: the two energies differ by less than the error bar here.)"""
    t = inputs.peps_tensors(4, 4, 2, 11, True)
    sk = inputs.sketch(4, 4, 2, 11)
    g = vmc.unpack(t, 4, 4, 2)
    _, cfg, psi = exact.energy_exact(g, 1.0, J2)
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    phi = np.array([psi[n] + psi[index[(-c).tobytes()]] for n, c in enumerate(flat)])
    Hphi = np.zeros_like(phi)
    for n, c in enumerate(flat):
        for i, j, J in exact.bonds(4, 4, 1.0, J2):
            Hphi[n] += J * c[i] * c[j] / 4.0 * phi[n]
            if c[i] != c[j]:
                c2 = c.copy()
                c2[i], c2[j] = c[j], c[i]
                Hphi[index[c2.tobytes()]] += 0.5 * J * phi[n]
    E_phi = float(phi @ Hphi / (phi @ phi))
    P, therm, sweeps = 1024, 20, 60
    ctx = api.PepsVMC(4, 4, 2, 4, 2 * P, t, sk, J1=1.0, J2=J2, seed=3, n_fit=1, symmetrize=True)
    ctx.set_spins(pairs_of(inputs.start_spins(P, 4, 4, 7, "random")))
    ctx.sample_sweep(therm)
    el = ctx.energy_and_grad(sweeps, want_grad=False)["eloc"].reshape(sweeps, 2 * P)[:, :P]
    mean, err = autocorr.mean_and_error(el)
    assert err > 0
    assert abs(mean - E_phi) <= 5 * err, (mean, E_phi, err)
    ctx.close()
