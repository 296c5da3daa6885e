"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module draws random numbers and lays them out; it holds none of the method's
arithmetic.  Everything the method later draws itself (Metropolis uniforms, sign-SGD
uniforms) comes from the counter-based Philox generator that each side implements
on its own.

Workloads (square open lattices, spin-1/2, physical dimension P = 2):

* ``peps_4x4``   : 4x4 Heisenberg, D=2, Dc=4 (exact), 1 chain, Neel start.
* ``peps_8x8``   : 8x8 Heisenberg, D=4, Dc=16, 1024 chains, tensors normalised per site.
* ``peps_16x16`` : 16x16 Heisenberg, D=6, Dc=24, 2048 chains.
* ``peps_24x24`` : 24x24 J1-J2 (J2/J1 = 0.5), D=8, Dc=32, 512 chains.
* ``peps_32x32`` : 32x32 Heisenberg, D=8, Dc=32, 256 chains.

Tensor entries are iid N(0,1) (the paper's workloads are optimised ground-state
PEPS, which are not available; iid Gaussian tensors of the same shapes stand in for
them).  Seeds are ``1908093590 + workload index``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1908093590

WORKLOADS = {
    "peps_4x4": dict(index=0, Ly=4, Lx=4, D=2, chi=4, n_chains=1, J1=1.0, J2=0.0,
                     normalise=False, start="neel"),
    "peps_8x8": dict(index=1, Ly=8, Lx=8, D=4, chi=16, n_chains=1024, J1=1.0, J2=0.0,
                     normalise=True, start="random"),
    "peps_16x16": dict(index=2, Ly=16, Lx=16, D=6, chi=24, n_chains=2048, J1=1.0, J2=0.0,
                       normalise=False, start="random"),
    "peps_24x24": dict(index=3, Ly=24, Lx=24, D=8, chi=32, n_chains=512, J1=1.0, J2=0.5,
                       normalise=False, start="random"),
    "peps_32x32": dict(index=4, Ly=32, Lx=32, D=8, chi=32, n_chains=256, J1=1.0, J2=0.0,
                       normalise=False, start="random"),
}


def site_shape(Ly: int, Lx: int, D: int, k: int, m: int) -> tuple:
    """(P, Dl, Dr, Du, Dd) of site (row k, column m); legs on the open edge have dimension 1."""
    return (2,
            1 if m == 0 else D,
            1 if m == Lx - 1 else D,
            1 if k == 0 else D,
            1 if k == Ly - 1 else D)


def n_params(Ly: int, Lx: int, D: int) -> int:
    return int(sum(np.prod(site_shape(Ly, Lx, D, k, m)) for k in range(Ly) for m in range(Lx)))


def peps_tensors(Ly: int, Lx: int, D: int, seed: int, normalise: bool = False,
                 bond_decay: float = 0.0) -> np.ndarray:
    """Flat float64 array, site-major (k, then m), each site (s, l, r, u, d) row-major.

    ``bond_decay`` > 0 scales virtual index i of every leg by exp(-bond_decay * i / 2),
    i.e. bond weights lambda_i = exp(-bond_decay * i) split evenly between the two
    tensors of a bond, as after a simple-update initialisation (App. A absorbs
    lambda^(1/2) into each tensor).  0 gives the plain iid N(0,1) tensors.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(Ly):
        for m in range(Lx):
            shp = site_shape(Ly, Lx, D, k, m)
            t = rng.standard_normal(shp)
            if bond_decay > 0.0:
                for axis in range(1, 5):
                    w = np.exp(-bond_decay * np.arange(shp[axis]) / 2.0)
                    t = t * w.reshape([-1 if a == axis else 1 for a in range(5)])
            if normalise:
                t = t / np.sqrt(np.sum(t * t))
            parts.append(t.ravel())
    return np.concatenate(parts)


def sketch(L: int, chi: int, D: int, seed: int) -> np.ndarray:
    """Raw Gaussian sketch tensors, shape (L, chi, D, chi), float64.

    They seed the variational fit of every boundary-MPS truncation; each side slices
    and orthonormalises them itself.
    """
    rng = np.random.default_rng(seed ^ 0x5CE7C4)
    return rng.standard_normal((L, chi, D, chi))


def start_spins(n_chains: int, Ly: int, Lx: int, seed: int, kind: str = "random") -> np.ndarray:
    """int8 spins (n_chains, Ly, Lx) of +-1 with total S^z = 0 (Ly*Lx must be even).

    ``neel``: s(k, m) = (-1)^(k+m).  ``random``: a seeded permutation of half ups.
    """
    N = Ly * Lx
    if N % 2:
        raise ValueError("S^z = 0 needs an even number of sites")
    if kind == "neel":
        k, m = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
        one = np.where((k + m) % 2 == 0, 1, -1).astype(np.int8)
        return np.broadcast_to(one, (n_chains, Ly, Lx)).copy()
    rng = np.random.default_rng(seed ^ 0x5B1A5)
    base = np.array([1] * (N // 2) + [-1] * (N // 2), dtype=np.int8)
    out = np.empty((n_chains, N), dtype=np.int8)
    for c in range(n_chains):
        out[c] = rng.permutation(base)
    return out.reshape(n_chains, Ly, Lx)


def proposal_params(seed: int) -> np.ndarray:
    """Initial weights of the proposal network as one float64 array in the order
    w1 (32,1,3,3), b1 (32), w2 (32,32,3,3), b2 (32), w3 (2,32,3,3), b3 (2): Gaussian
    entries scaled by sqrt(2 / fan-in) (He initialisation), the last layer by a further
    0.1, zero biases."""
    rng = np.random.default_rng(seed ^ 0xC0DE)
    parts = []
    for shape, extra in (((32, 1, 3, 3), 1.0), ((32, 32, 3, 3), 1.0), ((2, 32, 3, 3), 0.1)):
        parts.append(rng.standard_normal(shape).ravel() * np.sqrt(2.0 / (shape[1] * 9)) * extra)
        parts.append(np.zeros(shape[0]))
    return np.concatenate(parts)


def workload(name: str, n_chains: int | None = None) -> dict:
    """Everything a run of workload ``name`` needs, as plain arrays and numbers."""
    w = dict(WORKLOADS[name])
    seed = SEED_BASE + w["index"]
    nc = w["n_chains"] if n_chains is None else n_chains
    w.update(
        name=name, seed=seed, n_chains=nc,
        tensors=peps_tensors(w["Ly"], w["Lx"], w["D"], seed, w["normalise"]),
        sketch=sketch(max(w["Ly"], w["Lx"]), w["chi"], w["D"], seed),
        spins=start_spins(nc, w["Ly"], w["Lx"], seed, w["start"]),
    )
    return w
