"""Brute-force references for small lattices (no truncation anywhere).

Test infrastructure only (see the package header).  These are the plain definitions
the boundary-MPS oracle is pinned to:

* Psi(S) = Tr(A_1^{s_1} ... A_N^{s_N}) (Sec. II A, Eq. (4)) by a row transfer vector
  over all D^Lx values of the cut, and by one einsum over every bond index;
* the S^z = 0 sector and <Psi|H|Psi>/<Psi|Psi> (Eq. (2)) by applying H to the full
  amplitude vector;
* E_tot(A) as a function of the tensors, for finite-difference gradients.
"""
from __future__ import annotations

import itertools
import string

import numpy as np

from .vmc import sidx


def amplitude_transfer(grid, spins):
    """Psi(S) by a transfer vector over the vertical legs, one site at a time."""
    Ly, Lx = len(grid), len(grid[0])
    v = np.ones((1,) * Lx)
    for k in range(Ly):
        S = v[np.newaxis]
        for m in range(Lx):
            a = grid[k][m][sidx(spins[k][m])]          # (l, r, u, d)
            S = np.tensordot(S, a, axes=([0, 1 + m], [0, 2]))
            S = np.moveaxis(S, [-2, -1], [0, 1 + m])
        v = S[0]
    return float(v.reshape(()))


def amplitude_einsum(grid, spins):
    """Psi(S) as one einsum over all bond indices (every bond gets its own letter)."""
    Ly, Lx = len(grid), len(grid[0])
    letters = iter(string.ascii_letters)
    h = {(k, m): next(letters) for k in range(Ly) for m in range(Lx - 1)}
    v = {(k, m): next(letters) for k in range(Ly - 1) for m in range(Lx)}
    one = next(letters)  # dimension-1 open legs share a summed letter of extent 1
    terms, ops = [], []
    for k in range(Ly):
        for m in range(Lx):
            l = h[(k, m - 1)] if m > 0 else one
            r = h[(k, m)] if m < Lx - 1 else one
            u = v[(k - 1, m)] if k > 0 else one
            d = v[(k, m)] if k < Ly - 1 else one
            terms.append(l + r + u + d)
            ops.append(grid[k][m][sidx(spins[k][m])])
    return float(np.einsum(",".join(terms) + "->", *ops, optimize="greedy"))


def sz0_configs(Ly, Lx):
    """All configurations with sum sigma = 0, as an int8 array (n, Ly, Lx)."""
    N = Ly * Lx
    out = []
    for ups in itertools.combinations(range(N), N // 2):
        c = -np.ones(N, dtype=np.int8)
        c[list(ups)] = 1
        out.append(c.reshape(Ly, Lx))
    return np.array(out)


def bonds(Ly, Lx, J1, J2):
    """(site i, site j, J) for NN bonds and, if J2 != 0, both plaquette diagonals."""
    out = []
    for k in range(Ly):
        for m in range(Lx):
            i = k * Lx + m
            if m + 1 < Lx:
                out.append((i, i + 1, J1))
            if k + 1 < Ly:
                out.append((i, i + Lx, J1))
            if J2 != 0.0 and k + 1 < Ly and m + 1 < Lx:
                out.append((i, i + Lx + 1, J2))
                out.append((i + 1, i + Lx, J2))
    return out


def energy_exact(grid, J1, J2):
    """(<Psi|H|Psi>/<Psi|Psi>, configs, psi) over the S^z = 0 sector, H applied directly."""
    Ly, Lx = len(grid), len(grid[0])
    cfg = sz0_configs(Ly, Lx)
    psi = np.array([amplitude_transfer(grid, c) for c in cfg])
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    Hpsi = np.zeros_like(psi)
    for n, c in enumerate(flat):
        for i, j, J in bonds(Ly, Lx, J1, J2):
            Hpsi[n] += J * c[i] * c[j] / 4.0 * psi[n]
            if c[i] != c[j]:
                c2 = c.copy()
                c2[i], c2[j] = c[j], c[i]
                Hpsi[index[c2.tobytes()]] += 0.5 * J * psi[n]
    return float(psi @ Hpsi / (psi @ psi)), cfg, psi
