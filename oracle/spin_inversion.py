"""Spin-inversion symmetrised amplitude Phi(S) = Psi(S) + Psi(S-bar) (end of Sec. II B).

Test infrastructure only (see the package header).  S-bar is S with every spin
reversed.  Sampling follows |Phi|^2 and every observable is taken with that weight.

Built from the boundary-MPS pieces of ``vmc``; the quantities are:

* w(S) = Psi(S-bar) / Psi(S).  Since the Heisenberg Hamiltonian commutes with the
  global spin inversion, <S|H|S'> = <S-bar|H|S'-bar>, so the local energy of Phi is
  E^Phi(S) = (E_loc(S) + w E_loc(S-bar)) / (1 + w), and its log-derivative is
  G^Phi(S) = (G(S) + w G(S-bar)) / (1 + w), where G(S) sits in the slots s_i of S and
  G(S-bar) in the opposite slots.
* A pair exchange S -> S' on an antiparallel bond is the same exchange on S-bar, and
  Phi(S') / Phi(S) = (rho + w rho-bar) / (1 + w) with rho = Psi(S')/Psi(S) and
  rho-bar = Psi(S-bar')/Psi(S-bar); after an accepted move w <- w rho-bar / rho.

Readings of points the paper leaves open:
* The sweep is the sequential sweep of ``vmc.sweep`` run on S and S-bar in lockstep:
  each configuration keeps its own environments, both take the same decision, drawn
  from the uniform of (chain, sweep, bond) with the pair's index as the chain.
* w is taken afresh at the start of each phase (vertical, then horizontal) from the
  two amplitudes closed at row 0 of that phase's lattice with the phase's bottom
  environments (cutoff Dc of the sampler), then carried through the phase by the
  ratios of the accepted moves.
* The measurement takes w from the two measured amplitudes (row Ly//2, cutoff of
  the measurement).
"""
from __future__ import annotations

import numpy as np

from . import philox, vmc


def weight(logpsi, sign, logpsi_bar, sign_bar):
    """w = Psi(S-bar)/Psi(S) from the logs and signs of the two amplitudes."""
    return float(sign * sign_bar * np.exp(logpsi_bar - logpsi))


def phase_weight(grid, spins, Bs, logB, Bs_bar, logB_bar):
    """w of a phase: both amplitudes closed at row 0 (trivial top, bottom B_0)."""
    Lx = spins.shape[1]
    lp, sg = vmc.row_psi(vmc.trivial_mps(Lx), vmc.row_tensors(grid, spins, 0), Bs[0], 0.0, logB[0])
    lpb, sgb = vmc.row_psi(vmc.trivial_mps(Lx), vmc.row_tensors(grid, -spins, 0), Bs_bar[0], 0.0,
                           logB_bar[0])
    return weight(lp, sg, lpb, sgb)


class PairTrace:
    """Records (bond, rho, rho_bar, w, u, decision).  With ``follow`` set to a dict
    bond -> decision, near-ties (|ln u - ln q| < tie, q the |Phi|^2 ratio) take that
    decision."""

    def __init__(self, follow=None, tie=1e-5):
        self.rows, self.follow, self.tie = [], follow, tie

    def decide(self, bond, rho, rho_bar, w, u, q, accept):
        if self.follow is not None and bond in self.follow and q > 0.0:
            if abs(np.log(u if u > 0 else 1e-300) - np.log(q)) < self.tie:
                accept = bool(self.follow[bond])
        self.rows.append((bond, rho, rho_bar, w, u, bool(accept)))
        return accept


def _right_envs(a, spins, k, T, B):
    """Normalised R(m) of the current spins and R_f(m) of column m flipped (same norm)."""
    Lx = spins.shape[1]
    R, Rf = [None] * (Lx + 1), [None] * (Lx + 1)
    R[Lx] = np.ones((1, 1, 1))
    for m in range(Lx - 1, 0, -1):
        s = vmc.sidx(spins[k, m])
        raw = vmc.env3_right(R[m + 1], T[m], a[m][s], B[m])
        nrm = np.linalg.norm(raw)
        R[m] = raw / nrm
        Rf[m] = vmc.env3_right(R[m + 1], T[m], a[m][1 - s], B[m]) / nrm
    return R, Rf


def _sample_row_pair(grid, spins, k, T, B, Tb, Bb, w, seed, pair, sweep, bond_base, trace):
    """Metropolis visits of the horizontal bonds of row k for S (``spins``) and S-bar
    (its negation, environments Tb, Bb), accepting with min[1, |Phi(S')/Phi(S)|^2].
    Mutates ``spins``; returns w at the end of the row."""
    Lx = spins.shape[1]
    a = grid[k]
    R, Rf = _right_envs(a, spins, k, T, B)
    Rb, Rfb = _right_envs(a, -spins, k, Tb, Bb)
    E, Eb = np.ones((1, 1, 1)), np.ones((1, 1, 1))
    for m in range(Lx - 1):
        s = vmc.sidx(spins[k, m])
        cur = vmc.env3_left(E, T[m], a[m][s], B[m])
        cur_b = vmc.env3_left(Eb, Tb[m], a[m][1 - s], Bb[m])
        if spins[k, m] != spins[k, m + 1]:
            flip = vmc.env3_left(E, T[m], a[m][1 - s], B[m])
            flip_b = vmc.env3_left(Eb, Tb[m], a[m][s], Bb[m])
            rho = float(np.vdot(flip, Rf[m + 1]) / np.vdot(cur, R[m + 1]))
            rho_b = float(np.vdot(flip_b, Rfb[m + 1]) / np.vdot(cur_b, Rb[m + 1]))
            q = ((rho + w * rho_b) / (1.0 + w)) ** 2
            bond = bond_base + k * (Lx - 1) + m
            u = philox.metropolis_uniform(seed, pair, sweep, bond)
            accept = u < min(1.0, q)
            if trace is not None:
                accept = trace.decide(bond, rho, rho_b, w, u, q, accept)
            if accept:
                spins[k, m] = -spins[k, m]
                spins[k, m + 1] = -spins[k, m + 1]
                cur, cur_b = flip, flip_b
                w = w * rho_b / rho
        E, _ = vmc._normalised(cur)
        Eb, _ = vmc._normalised(cur_b)
    return w


def _row_phase_pair(grid, spins, chi, W, n_fit, seed, pair, sweep, bond_base, trace):
    """The row phase of ``vmc`` for S and S-bar in lockstep (mutates ``spins``)."""
    Ly, Lx = spins.shape
    Bs, logB = vmc.bottom_envs(grid, spins, chi, W, n_fit)
    Bsb, logBb = vmc.bottom_envs(grid, -spins, chi, W, n_fit)
    w = phase_weight(grid, spins, Bs, logB, Bsb, logBb)
    T, Tb = vmc.trivial_mps(Lx), vmc.trivial_mps(Lx)
    for k in range(Ly):
        w = _sample_row_pair(grid, spins, k, T, Bs[k], Tb, Bsb[k], w, seed, pair, sweep, bond_base, trace)
        if k < Ly - 1:
            T, _ = vmc.compress(vmc.mpo_times_mps(T, vmc.row_tensors(grid, spins, k)), chi, W, n_fit)
            Tb, _ = vmc.compress(vmc.mpo_times_mps(Tb, vmc.row_tensors(grid, -spins, k)), chi, W, n_fit)
    return w


def sweep(grid, spins, chi, W, n_fit, seed, pair, sweep_index, trace=None):
    """One sequential sweep sampling |Phi|^2 (bond ids and order as ``vmc.sweep``).
    Returns the new S (S-bar is its negation)."""
    spins = np.array(spins, dtype=np.int8)
    Ly, Lx = spins.shape
    st = np.ascontiguousarray(spins.T)
    _row_phase_pair(vmc.transpose_lattice(grid), st, chi, W, n_fit, seed, pair, sweep_index, 0, trace)
    spins = np.ascontiguousarray(st.T)
    _row_phase_pair(grid, spins, chi, W, n_fit, seed, pair, sweep_index, Lx * (Ly - 1), trace)
    return spins


def measure(grid, spins, chi, W, n_fit, J1, J2, want_grad=True):
    """E^Phi, w and G^Phi of one configuration.  G^Phi is a list of lists of arrays of
    the site tensors' full shape (2, Dl, Dr, Du, Dd): G(S) / (1 + w) in the slots of
    S and w G(S-bar) / (1 + w) in the slots of S-bar."""
    spins = np.asarray(spins)
    m = vmc.measure(grid, spins, chi, W, n_fit, J1, J2, want_grad=want_grad)
    mb = vmc.measure(grid, -spins, chi, W, n_fit, J1, J2, want_grad=want_grad)
    w = weight(m["logpsi"], m["sign"], mb["logpsi"], mb["sign"])
    out = dict(w=w, eloc_phi=(m["eloc"] + w * mb["eloc"]) / (1.0 + w), eloc=m["eloc"], eloc_bar=mb["eloc"],
               scale=m["eloc_scale"] + abs(w) * mb["eloc_scale"], plain=m, bar=mb)
    if want_grad:
        Ly, Lx = spins.shape
        G = [[np.zeros_like(t) for t in row] for row in grid]
        for k in range(Ly):
            for mm in range(Lx):
                s = vmc.sidx(spins[k, mm])
                G[k][mm][s] += m["G"][k][mm] / (1.0 + w)
                G[k][mm][1 - s] += w * mb["G"][k][mm] / (1.0 + w)
        out["G"] = G
    return out


class Accumulator:
    """Algorithm 1's sums with the weight |Phi|^2: one sample per pair."""

    def __init__(self, grid):
        self.n, self.sE, self.sE2 = 0, 0.0, 0.0
        self.P1 = [[np.zeros_like(t) for t in row] for row in grid]
        self.P2 = [[np.zeros_like(t) for t in row] for row in grid]

    def add(self, r):
        e = r["eloc_phi"]
        self.n += 1
        self.sE += e
        self.sE2 += e * e
        for k, row in enumerate(r["G"]):
            for m, g in enumerate(row):
                self.P1[k][m] += g * e
                self.P2[k][m] += g

    def gradient(self):
        E = self.sE / self.n
        return [[p1 / self.n - (p2 / self.n) * E for p1, p2 in zip(r1, r2)]
                for r1, r2 in zip(self.P1, self.P2)], E
