"""Pins of the simple-update oracle (App. A, oracle/simple_update.py), CPU only.

* the gate's closed form against the matrix exponential of J S1.S2;
* without truncation an NN update and an NNN update (every direction, every corner path)
  change the state represented by the lambda-weighted network exactly into G|Psi>, with
  |Psi> and G|Psi> built by brute force over all 2^N configurations;
* with truncation the new lambdas are unit vectors of length D and every tensor stays
  finite;
* imaginary-time evolution lowers the energy to within a few tenths of a percent of the
  exact ground-state energy (diagonalisation of H in the S^z = 0 sector) on 2x2 and, with
  J2 = 0.5, on 2x4, and never below it (variational).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg

from oracle import exact, simple_update as su


def full_vector(grid):
    Ly, Lx = len(grid), len(grid[0])
    return {bits: exact.amplitude_transfer(grid, np.array(bits, dtype=np.int8).reshape(Ly, Lx))
            for bits in itertools.product([1, -1], repeat=Ly * Lx)}


def apply_gate(v, i, j, g):
    out = {b: 0.0 for b in v}
    for bits, a in v.items():
        s1, s2 = (0 if bits[i] == 1 else 1), (0 if bits[j] == 1 else 1)
        for u in range(2):
            for w in range(2):
                nb = list(bits)
                nb[i], nb[j] = (1 if u == 0 else -1), (1 if w == 0 else -1)
                out[tuple(nb)] += g[u, w, s1, s2] * a
    return out


def same_ray(a, b):
    x = np.array([a[k] for k in sorted(a)])
    y = np.array([b[k] for k in sorted(b)])
    x, y = x / np.linalg.norm(x), y / np.linalg.norm(y)
    return np.max(np.abs(x - np.sign(x @ y) * y))


def random_lambdas(st, seed):
    rng = np.random.default_rng(seed)
    for row in st.lh + st.lv:
        for i in range(len(row)):
            row[i] = rng.uniform(0.3, 1.0, size=row[i].shape)
    return st


def ground_energy(Ly, Lx, J1, J2):
    cfg = exact.sz0_configs(Ly, Lx)
    flat = cfg.reshape(len(cfg), -1)
    idx = {c.tobytes(): n for n, c in enumerate(flat)}
    H = np.zeros((len(cfg), len(cfg)))
    for n, c in enumerate(flat):
        for i, j, J in exact.bonds(Ly, Lx, J1, J2):
            H[n, n] += J * c[i] * c[j] / 4
            if c[i] != c[j]:
                c2 = c.copy()
                c2[i], c2[j] = c[j], c[i]
                H[idx[c2.tobytes()], n] += 0.5 * J
    return np.linalg.eigvalsh(H)[0]


def test_gate_is_the_matrix_exponential():
    h = np.diag([0.25, -0.25, -0.25, 0.25])
    h[1, 2] = h[2, 1] = 0.5
    for J, tau in ((1.0, 0.01), (0.5, 0.3), (1.7, -0.2)):
        ref = scipy.linalg.expm(-tau * J * h).reshape(2, 2, 2, 2)
        assert np.max(np.abs(su.heisenberg_gate(J, tau) - ref)) < 1e-14


@pytest.mark.parametrize("bond", [((0, 1), (0, 2)), ((0, 0), (1, 0)), ((1, 1), (1, 2)), ((0, 2), (1, 2))])
def test_nn_update_without_truncation_is_exact(bond):
    st = random_lambdas(su.init_state(2, 3, 2, 5), 1)
    g = su.heisenberg_gate(1.0, 0.4)
    v0 = full_vector(su.to_peps(st))
    p1, p2 = bond
    su.nn_update(st, p1, p2, g, 64)
    i, j = p1[0] * 3 + p1[1], p2[0] * 3 + p2[1]
    assert same_ray(full_vector(su.to_peps(st)), apply_gate(v0, i, j, g)) < 1e-12


@pytest.mark.parametrize("triple", [((0, 0), (0, 1), (1, 1)), ((0, 0), (1, 0), (1, 1)), ((0, 1), (0, 0), (1, 0)),
                                    ((0, 1), (1, 1), (1, 0)), ((1, 1), (1, 2), (2, 2)), ((1, 1), (2, 1), (2, 2)),
                                    ((1, 2), (1, 1), (2, 1)), ((1, 2), (2, 2), (2, 1))])
def test_nnn_update_without_truncation_is_exact(triple):
    st = random_lambdas(su.init_state(3, 3, 2, 5), 2)
    g = su.heisenberg_gate(0.7, 0.3)
    v0 = full_vector(su.to_peps(st))
    p1, c, p3 = triple
    su.nnn_update(st, p1, c, p3, g, 64)
    i, j = p1[0] * 3 + p1[1], p3[0] * 3 + p3[1]
    assert same_ray(full_vector(su.to_peps(st)), apply_gate(v0, i, j, g)) < 1e-12


def test_truncated_updates_keep_unit_lambdas_of_length_D():
    D = 3
    st = random_lambdas(su.init_state(4, 4, D, 9), 3)
    su.trotter_step(st, 1.0, 0.5, 0.1, D)
    for lam in st.links():
        assert len(lam) == D and abs(np.linalg.norm(lam) - 1.0) < 1e-12 and np.all(lam >= 0)
    for row in st.B:
        for t in row:
            assert np.all(np.isfinite(t))


@pytest.mark.parametrize("Ly,Lx,D,J2,rel", [(2, 2, 2, 0.0, 5e-3), (2, 4, 4, 0.5, 5e-3)])
def test_evolution_approaches_the_ground_state(Ly, Lx, D, J2, rel):
    st = su.init_state(Ly, Lx, D, 3)
    su.evolve(st, 1.0, J2, D, [(0.05, 300), (0.01, 300)], tol=1e-9)
    E = exact.energy_exact(su.to_peps(st), 1.0, J2)[0]
    E0 = ground_energy(Ly, Lx, 1.0, J2)
    assert E >= E0 - 1e-10
    assert (E - E0) <= rel * abs(E0), (E, E0)
