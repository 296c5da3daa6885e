"""Pins of the learned-proposal oracle (CPU): convolution gradients against finite
differences, proposal probabilities normalised and matching the sampler's draws, band
ratios against brute force, and exact detailed balance of the learned MH kernel on a
lattice small enough to enumerate every configuration and move."""
import itertools

import numpy as np
import pytest

from oracle import exact, proposal, vmc
from paper_1908_09359_gb300 import inputs


def test_conv_net_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = proposal.init_params(3)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]
    spins = rng.choice([-1, 1], size=(3, 4, 5))
    ratios_h = np.exp(rng.standard_normal((3, 4, 4)))
    ratios_v = np.exp(rng.standard_normal((3, 3, 5)))
    tgt, mask = proposal.bond_targets(spins, ratios_h, ratios_v)
    loss, grads = proposal.loss_and_grad(params, spins, tgt, mask)
    h = 1e-6
    for i, p in enumerate(params):
        for _ in range(4):
            idx = tuple(rng.integers(n) for n in p.shape)
            pp = [q.copy() for q in params]
            pp[i][idx] += h
            lp, _ = proposal.loss_and_grad(pp, spins, tgt, mask)
            pp[i][idx] -= 2 * h
            lm, _ = proposal.loss_and_grad(pp, spins, tgt, mask)
            assert grads[i][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def _all_moves(cand):
    keys = [(c[0], c[1]) for c in cand]
    ones = [(k,) for k in keys]
    twos = [(a, b) for (i, a), (j, b) in itertools.combinations(enumerate(keys), 2)
            if not ({a[0], a[1]} & {b[0], b[1]})]
    return ones, twos


def test_move_probabilities_are_normalised_and_match_draws():
    rng = np.random.default_rng(1)
    params = proposal.init_params(5)
    spins = inputs.start_spins(1, 4, 5, 3, "random")[0] if (4 * 5) % 2 == 0 else None
    logits = proposal.forward(params, spins[None])[0][0]
    k = 1
    cand = proposal.candidates(spins, k)
    ones, twos = _all_moves(cand)
    probs = {m: np.exp(proposal.move_logprob(logits, spins, k, m)) for m in ones + twos}
    lg = np.array([logits[c[2], c[3][0], c[3][1]] for c in cand])
    p1 = np.exp(lg - lg.max()) / np.exp(lg - lg.max()).sum()
    p_null = 0.5 * sum(p1[i] for i, c in enumerate(cand) if not any(
        not ({c[0], c[1]} & {d[0], d[1]}) for d in cand if d is not c))
    assert sum(probs.values()) + p_null == pytest.approx(1.0, abs=1e-12)
    counts = {}
    n = 40000
    for _ in range(n):
        m = proposal.propose(logits, spins, k, *rng.random(3))
        if m is not None and len(m) == 2 and m not in probs:
            m = (m[1], m[0])
        counts[m] = counts.get(m, 0) + 1
    for m, p in probs.items():
        if p > 0.01:
            assert counts.get(m, 0) / n == pytest.approx(p, abs=4 * np.sqrt(p / n) + 1e-3)


def test_band_ratio_is_exact_amplitude_ratio():
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = vmc.unpack(inputs.peps_tensors(Ly, Lx, D, 17), Ly, Lx, D)
    W = inputs.sketch(4, chi, D, 3)
    s = inputs.start_spins(1, Ly, Lx, 9, "random")[0]
    Ts, _ = vmc.top_envs(g, s, chi, W, 1)
    Bs, _ = vmc.bottom_envs(g, s, chi, W, 1)
    for k in range(Ly - 1):
        cand = proposal.candidates(s, k)
        move = ((cand[0][0], cand[0][1]), (cand[-1][0], cand[-1][1]))
        if {move[0][0], move[0][1]} & {move[1][0], move[1][1]}:
            move = move[:1]
        new = proposal.apply_move(s, move)
        ref = exact.amplitude_transfer(g, new) / exact.amplitude_transfer(g, s)
        assert proposal.band_psi_ratio(g, s, new, k, Ts[k], Bs[k + 1]) == pytest.approx(ref, rel=1e-10)


def test_learned_mh_kernel_satisfies_detailed_balance_exactly():
    """Every configuration and every move of the learned kernel on 2x4 (one band, exact
    Dc): pi(S) P(S -> S') = pi(S') P(S' -> S) with pi = |Psi|^2, for an untrained
    network -- the acceptance min[1, |Psi'/Psi|^2 q(S|S')/q(S'|S)] (Eq. (8) with a
    learned q) makes the chain exact whatever q is."""
    Ly, Lx, D, chi = 2, 4, 2, 2
    g = vmc.unpack(inputs.peps_tensors(Ly, Lx, D, 23), Ly, Lx, D)
    W = inputs.sketch(4, chi, D, 1)
    params = proposal.init_params(11)
    params = [p_ + 0.3 * np.random.default_rng(2).standard_normal(p_.shape) for p_ in params]
    _, cfg, psi = exact.energy_exact(g, 1.0, 0.0)
    pi = psi ** 2 / np.sum(psi ** 2)
    index = {c.tobytes(): i for i, c in enumerate(cfg.reshape(len(cfg), -1))}
    n = len(cfg)
    P = np.zeros((n, n))
    for i, s in enumerate(cfg):
        Ts, _ = vmc.top_envs(g, s, chi, W, 1)
        Bs, _ = vmc.bottom_envs(g, s, chi, W, 1)
        logits = proposal.forward(params, s[None])[0][0]
        ones, twos = _all_moves(proposal.candidates(s, 0))
        for m in ones + twos:
            q = np.exp(proposal.move_logprob(logits, s, 0, m))
            new = proposal.apply_move(s, m)
            q_rev = np.exp(proposal.move_logprob(proposal.forward(params, new[None])[0][0], new, 0, m))
            rho = proposal.band_psi_ratio(g, s, new, 0, Ts[0], Bs[1])
            P[i, index[new.reshape(-1).tobytes()]] += q * min(1.0, rho * rho * q_rev / q)
    flow = pi[:, None] * P
    assert np.max(np.abs(flow - flow.T)) <= 1e-12 * np.max(flow)
    assert np.count_nonzero(flow > 1e-9) > 3 * n   # the kernel actually moves
