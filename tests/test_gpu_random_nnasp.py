"""The random-NNASP scheme on the GPU (Sec. II A, Eq. (prob_r)): the paper's reference
sampler for its sequential sweep.

* Parity with the oracle (oracle/random_nnasp.py), draw for draw: every attempt of one
  sweep picks the same antiparallel pair from the same Philox word, its ratio
  Psi(S_b)/Psi(S_a) (two full boundary-MPS contractions) agrees within 1e-4 relative to
  max(|rho|, 1) (exact cutoff) or 2e-4 (truncated, bond-decay tensors), every decision is
  the same except at near-ties |ln r - ln P| < 1e-5 (replayed with the GPU's decision), and
  the final spins are identical.
* The equivalence the paper shows in Fig. SweepScheme, at exact Dc on 4x4: from the same
  starts, the random scheme's chains and the sequential sweep's chains both give a mean
  E_loc equal to the enumerated <H> within five tau_int-corrected standard errors (for the
  Heisenberg and the J1-J2 model), and so agree with each other.
"""
import numpy as np
import pytest

from oracle import exact, philox, random_nnasp, vmc
from paper_1908_09359_gb300 import autocorr, inputs

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


@pytest.mark.parametrize("case", ["4x4_exact", "6x6_truncated"])
def test_random_sweep_matches_oracle_draw_for_draw(api, case):
    if case == "4x4_exact":
        Ly = Lx = 4
        D, chi, n_fit, tol = 2, 4, 1, 1e-4
        t = inputs.peps_tensors(4, 4, 2, 19)
    else:
        Ly = Lx = 6
        D, chi, n_fit, tol = 3, 6, 3, 2e-4
        t = inputs.peps_tensors(6, 6, 3, 23, bond_decay=1.0)
    sk = inputs.sketch(Ly, chi, D, 5)
    g = vmc.unpack(t, Ly, Lx, D)
    n, seed, sweep = 8, 4242, 9
    start = inputs.start_spins(n, Ly, Lx, 61, "random")
    ctx = api.PepsVMC(Ly, Lx, D, chi, n, t, sk, seed=seed, n_fit=n_fit)
    ctx.set_spins(start)
    ctx.set_sweep_counter(sweep)
    ctx.enable_trace(True)
    rate = ctx.random_sweep(1)
    bond, ratio, dec = ctx.get_random_trace()
    final = ctx.get_spins()
    assert 0.0 < rate < 1.0
    accepted = 0
    for c in range(n):
        s = start[c].copy()
        cur = random_nnasp.boundary_psi(g, s, chi, sk, n_fit)
        for a in range(Ly * Lx):
            word, r = philox.random_attempt_words(seed, c, sweep, a)
            rec = []
            s2, cur2 = random_nnasp.attempt_with(g, s, chi, sk, n_fit, word, r, cur, rec)
            b, rho, Ka, Kb, acc = rec[0]
            assert bond[c, a] == b, (c, a)
            if b < 0:
                continue
            assert abs(ratio[c, a] - rho) <= tol * max(abs(rho), 1.0), (c, a, ratio[c, a], rho)
            if int(acc) != int(dec[c, a]):
                p = min(1.0, rho * rho * Ka / Kb)
                assert abs(np.log(r) - np.log(p)) < 1e-5, (c, a, r, p)
                rec = []
                s2, cur2 = random_nnasp.attempt_with(g, s, chi, sk, n_fit, word, r, cur, rec, force=bool(dec[c, a]))
            accepted += int(dec[c, a])
            s, cur = s2, cur2
        assert np.array_equal(s, final[c]), c
    assert accepted > 0
    ctx.close()


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_random_and_sequential_schemes_sample_the_same_energy(api, J2):
    chains, therm, sweeps = 512, 8, 24
    t = inputs.peps_tensors(4, 4, 2, 11, True)
    sk = inputs.sketch(4, 4, 2, 11)
    E, _, _ = exact.energy_exact(vmc.unpack(t, 4, 4, 2), 1.0, J2)
    means = {}
    for scheme in ("random", "sequential"):
        ctx = api.PepsVMC(4, 4, 2, 4, chains, t, sk, J1=1.0, J2=J2, seed=13, n_fit=1)
        ctx.set_spins(inputs.start_spins(chains, 4, 4, 3, "random"))
        step = ctx.random_sweep if scheme == "random" else ctx.sample_sweep
        step(therm)
        el = np.empty((sweeps, chains))
        for i in range(sweeps):
            step(1)
            el[i] = ctx.measure()[0]
        mean, err = autocorr.mean_and_error(el)
        assert err > 0 and abs(mean - E) <= 5 * err, (scheme, mean, E, err)
        means[scheme] = (mean, err)
        ctx.close()
    (m1, e1), (m2, e2) = means["random"], means["sequential"]
    assert abs(m1 - m2) <= 5 * np.hypot(e1, e2)
