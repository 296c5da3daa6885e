"""Random-NNASP sampling of Sec. II A -- FP64 oracle.

Test infrastructure only (see the package header).  The paper validates its sequential
sweep against the usual scheme: pick one of the K(S) nearest-neighbour antiparallel
spin pairs (NNASPs) of S uniformly at random, swap it to get S', and accept with
min[1, (|Psi(S')|^2 / K(S')) / (|Psi(S)|^2 / K(S))] -- the 1/K factors are the
proposal probabilities, so the rule is Metropolis-Hastings and samples |Psi|^2 even
though K changes from configuration to configuration.  The sequential scheme instead
visits every bond in lattice order and accepts a swap of an antiparallel pair with
min[1, |Psi(S')|^2 / |Psi(S)|^2].

This module writes both schemes as exact transition matrices over the S^z = 0 sector
of a small lattice, for any amplitude function, so that their stationary
distributions can be compared with |Psi|^2 and with each other; and the random scheme
as a sampler on the boundary-MPS amplitude (App. B) with Philox uniforms, one sweep being
N attempts (N = Ly Lx, Sec. II A), which the GPU sampler reproduces draw for draw.
"""
from __future__ import annotations

import numpy as np

from . import exact, philox, vmc


def nn_bonds(Ly, Lx):
    """Nearest-neighbour bonds (i, j) of the flattened lattice in the sequential sweep's
    order: vertical bonds (columns left to right, top to bottom), then horizontal bonds
    (rows top to bottom, left to right)."""
    vert = [(k * Lx + m, (k + 1) * Lx + m) for m in range(Lx) for k in range(Ly - 1)]
    horiz = [(k * Lx + m, k * Lx + m + 1) for k in range(Ly) for m in range(Lx - 1)]
    return vert + horiz


def nnasps(flat, bonds):
    """The antiparallel pairs among `bonds` for the flattened configuration `flat`."""
    return [(i, j) for i, j in bonds if flat[i] != flat[j]]


def _swap(flat, i, j):
    out = flat.copy()
    out[i], out[j] = flat[j], flat[i]
    return out


def random_scheme_matrix(cfg, psi, Ly, Lx, with_k=True):
    """Transition matrix P[a, b] of one random-NNASP attempt over the configurations
    `cfg` (n, Ly, Lx) with amplitudes psi.  with_k=False drops the 1/K factors from the
    acceptance (a plausible mistake the tests must catch)."""
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    bonds = nn_bonds(Ly, Lx)
    K = np.array([len(nnasps(c, bonds)) for c in flat], dtype=np.float64)
    P = np.zeros((len(cfg), len(cfg)))
    for a, c in enumerate(flat):
        pairs = nnasps(c, bonds)
        for i, j in pairs:
            b = index[_swap(c, i, j).tobytes()]
            ratio = psi[b] ** 2 / psi[a] ** 2
            if with_k:
                ratio *= K[a] / K[b]
            P[a, b] += min(1.0, ratio) / K[a]
        P[a, a] += 1.0 - P[a].sum()
    return P


def sequential_sweep_matrix(cfg, psi, Ly, Lx):
    """Transition matrix of one sequential sweep: the product, in visiting order, of the
    single-bond kernels (swap an antiparallel pair with probability min[1, psi'^2/psi^2])."""
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    n = len(cfg)
    P = np.eye(n)
    for i, j in nn_bonds(Ly, Lx):
        Pb = np.zeros((n, n))
        for a, c in enumerate(flat):
            if c[i] != c[j]:
                b = index[_swap(c, i, j).tobytes()]
                acc = min(1.0, psi[b] ** 2 / psi[a] ** 2)
                Pb[a, b] += acc
                Pb[a, a] += 1.0 - acc
            else:
                Pb[a, a] = 1.0
        P = P @ Pb
    return P


def stationary(P):
    """The stationary distribution of a row-stochastic matrix (left eigenvector of
    eigenvalue 1, normalised)."""
    w, v = np.linalg.eig(P.T)
    x = np.real(v[:, np.argmin(np.abs(w - 1.0))])
    return x / x.sum()


def sector(grid):
    """(configurations of the S^z = 0 sector, exact amplitudes) of a small lattice."""
    Ly, Lx = len(grid), len(grid[0])
    cfg = exact.sz0_configs(Ly, Lx)
    return cfg, np.array([exact.amplitude_transfer(grid, c) for c in cfg])


def boundary_psi(grid, spins, chi, W, n_fit):
    """(ln|Psi|, sign) of a configuration by the boundary-MPS contraction closed at row
    Ly // 2 (the amplitude the measurement reports)."""
    Ly = len(grid)
    k = Ly // 2
    Ts, logT = vmc.top_envs(grid, spins, chi, W, n_fit, upto=k)
    Bs, logB = vmc.bottom_envs(grid, spins, chi, W, n_fit)
    return vmc.row_psi(Ts[k], vmc.row_tensors(grid, spins, k), Bs[k], logT[k], logB[k])


def random_attempt(grid, spins, chi, W, n_fit, seed, chain, sweep, attempt, cur=None, record=None):
    """One attempt of the random-NNASP scheme (Eq. (prob_r)) from configuration `spins`
    with the Philox uniforms of (chain, sweep, attempt); see attempt_with."""
    word, r = philox.random_attempt_words(seed, chain, sweep, attempt)
    return attempt_with(grid, spins, chi, W, n_fit, word, r, cur, record)


def attempt_with(grid, spins, chi, W, n_fit, word, r, cur=None, record=None, force=None):
    """The attempt for a given pick word and acceptance uniform r: the K_a antiparallel
    NN pairs of S_a are listed in the sweep's bond order, the pair with index
    pick(word, K_a) is swapped, and the trial S_b is accepted when
    r < min[1, (|Psi(S_b)|^2 / K_b) / (|Psi(S_a)|^2 / K_a)].  `cur` = (ln|Psi|, sign) of
    `spins` (computed when None).  Returns (new spins, (ln|Psi|, sign) of them); `record`
    (list) receives (bond id, ratio Psi(S_b)/Psi(S_a), K_a, K_b, decision).  `force`
    (True / False) replaces the decision (replaying another implementation's decision at
    a near-tie)."""
    spins = np.asarray(spins)
    Ly, Lx = spins.shape
    flat = spins.ravel()
    bonds = nn_bonds(Ly, Lx)
    if cur is None:
        cur = boundary_psi(grid, spins, chi, W, n_fit)
    pairs = [(n, i, j) for n, (i, j) in enumerate(bonds) if flat[i] != flat[j]]
    if not pairs:
        if record is not None:
            record.append((-1, 0.0, 0, 0, False))
        return spins.copy(), cur
    bond, i, j = pairs[philox.pick(word, len(pairs))]
    trial = _swap(flat, i, j).reshape(Ly, Lx)
    new = boundary_psi(grid, trial, chi, W, n_fit)
    Ka = len(pairs)
    Kb = len(nnasps(trial.ravel(), bonds))
    rho = new[1] * cur[1] * np.exp(new[0] - cur[0])
    accept = r < min(1.0, rho * rho * Ka / Kb) if force is None else bool(force)
    if record is not None:
        record.append((bond, rho, Ka, Kb, bool(accept)))
    return (trial, new) if accept else (spins.copy(), cur)


def random_sweep(grid, spins, chi, W, n_fit, seed, chain, sweep, record=None):
    """One sweep of the random scheme: N = Ly Lx attempts (Sec. II A)."""
    spins = np.asarray(spins).copy()
    cur = boundary_psi(grid, spins, chi, W, n_fit)
    for t in range(spins.size):
        spins, cur = random_attempt(grid, spins, chi, W, n_fit, seed, chain, sweep, t, cur, record)
    return spins
