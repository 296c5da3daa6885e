"""Pins of the spin-inversion oracle (Phi(S) = Psi(S) + Psi(S-bar), end of Sec. II B).

Each test pins a piece of ``oracle/spin_inversion.py`` to something other than itself:
brute force over the S^z = 0 sector at exact Dc (Phi built from exact amplitudes, H
applied to the full Phi vector), finite differences of the exact symmetrised energy,
exact amplitude ratios of every sweep proposal, and a symmetric special case where
Phi = 2 Psi and everything reduces to the plain method.
"""
import numpy as np
import pytest

from oracle import exact, philox, spin_inversion, vmc
from paper_1908_09359_gb300 import inputs


def peps(Ly, Lx, D, seed):
    return vmc.unpack(inputs.peps_tensors(Ly, Lx, D, seed, False), Ly, Lx, D)


def phi_table(g):
    """(configs, Phi, index) over the S^z = 0 sector from exact amplitudes."""
    _, cfg, psi = exact.energy_exact(g, 1.0, 0.0)
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    phi = np.array([psi[n] + psi[index[(-c).tobytes()]] for n, c in enumerate(flat)])
    return cfg, phi, index


def exact_phi_energy(g, J1, J2):
    """<Phi|H|Phi>/<Phi|Phi> with H applied to the full Phi vector."""
    Ly, Lx = len(g), len(g[0])
    cfg, phi, index = phi_table(g)
    flat = cfg.reshape(len(cfg), -1)
    Hphi = np.zeros_like(phi)
    for n, c in enumerate(flat):
        for i, j, J in exact.bonds(Ly, Lx, J1, J2):
            Hphi[n] += J * c[i] * c[j] / 4.0 * phi[n]
            if c[i] != c[j]:
                c2 = c.copy()
                c2[i], c2[j] = c[j], c[i]
                Hphi[index[c2.tobytes()]] += 0.5 * J * phi[n]
    return float(phi @ Hphi / (phi @ phi))


def direct_eloc_phi(g, c, phi, index, J1, J2):
    """sum_S' <S|H|S'> Phi(S')/Phi(S) straight from the Phi table."""
    Ly, Lx = len(g), len(g[0])
    f = c.reshape(-1)
    n = index[f.tobytes()]
    e = 0.0
    for a, b, J in exact.bonds(Ly, Lx, J1, J2):
        e += J * f[a] * f[b] / 4.0
        if f[a] != f[b]:
            f2 = f.copy()
            f2[a], f2[b] = f[b], f[a]
            e += 0.5 * J * phi[index[f2.tobytes()]] / phi[n]
    return e


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_eloc_phi_equals_brute_force_and_mean_equals_exact_energy(J2):
    """On 2x4 at exact Dc every E^Phi(S) equals its brute-force value from the Phi table,
    and the |Phi|^2-weighted mean over the whole sector equals <Phi|H|Phi>/<Phi|Phi>."""
    Ly, Lx, D, chi = 2, 4, 2, 2
    g = peps(Ly, Lx, D, 41)
    W = inputs.sketch(4, chi, D, 7)
    cfg, phi, index = phi_table(g)
    wts = phi ** 2 / np.sum(phi ** 2)
    mean = 0.0
    for wt, c in zip(wts, cfg):
        r = spin_inversion.measure(g, c, chi, W, 1, 1.0, J2, want_grad=False)
        assert r["eloc_phi"] == pytest.approx(direct_eloc_phi(g, c, phi, index, 1.0, J2), rel=1e-9, abs=1e-9)
        n, nb = index[c.reshape(-1).tobytes()], index[(-c).reshape(-1).tobytes()]
        psi_n = exact.amplitude_transfer(g, c)
        assert r["w"] == pytest.approx((phi[n] - psi_n) / psi_n, rel=1e-9)
        assert phi[n] == pytest.approx(phi[nb], rel=1e-12)   # Phi(S-bar) = Phi(S)
        mean += wt * r["eloc_phi"]
    assert mean == pytest.approx(exact_phi_energy(g, 1.0, J2), rel=1e-10)


def test_eloc_phi_4x4_heaviest_configurations():
    """4x4, D = 2, exact Dc = 4: E^Phi of the heaviest configurations against brute force."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 31)
    W = inputs.sketch(4, chi, D, 7)
    cfg, phi, index = phi_table(g)
    for i in np.argsort(-phi ** 2)[:24]:
        r = spin_inversion.measure(g, cfg[i], chi, W, 1, 1.0, 0.5, want_grad=False)
        assert r["eloc_phi"] == pytest.approx(direct_eloc_phi(g, cfg[i], phi, index, 1.0, 0.5),
                                              rel=1e-9, abs=1e-9)


def test_gradient_matches_fd_of_exact_phi_energy():
    """2(<G^Phi E^Phi> - <G^Phi><E^Phi>) under exact |Phi|^2 weights equals the finite
    difference of <Phi|H|Phi>/<Phi|Phi> in every sampled tensor element (both slots)."""
    Ly, Lx, D, chi = 2, 4, 2, 2
    g = peps(Ly, Lx, D, 77)
    W = inputs.sketch(4, chi, D, 7)
    cfg, phi, _ = phi_table(g)
    wts = phi ** 2 / np.sum(phi ** 2)
    acc = spin_inversion.Accumulator(g)
    P1 = [[np.zeros_like(t) for t in row] for row in g]
    P2 = [[np.zeros_like(t) for t in row] for row in g]
    Ebar = 0.0
    for wt, c in zip(wts, cfg):
        r = spin_inversion.measure(g, c, chi, W, 1, 1.0, 0.5)
        Ebar += wt * r["eloc_phi"]
        for k in range(Ly):
            for m in range(Lx):
                P1[k][m] += wt * r["G"][k][m] * r["eloc_phi"]
                P2[k][m] += wt * r["G"][k][m]
        if wt > 0.01:
            acc.add(r)
    E0 = exact_phi_energy(g, 1.0, 0.5)
    assert Ebar == pytest.approx(E0, rel=1e-10)
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(10):
        k, m = rng.integers(Ly), rng.integers(Lx)
        idx = tuple(rng.integers(n) for n in g[k][m].shape)
        grad = P1[k][m][idx] - P2[k][m][idx] * Ebar
        vals = []
        for sgn in (1, -1):
            g2 = [[t.copy() for t in row] for row in g]
            g2[k][m][idx] += sgn * h
            vals.append(exact_phi_energy(g2, 1.0, 0.5))
        assert 2 * grad == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=1e-5, abs=1e-8)
    # the accumulator's formula is the same sums divided by the sample count
    gr, E = acc.gradient()
    assert acc.n > 0 and np.isfinite(E) and all(np.all(np.isfinite(x)) for row in gr for x in row)


def test_sweep_ratios_are_exact_phi_ratios():
    """4x4 at exact Dc: every proposal's rho and rho-bar equal exact amplitude ratios, w
    equals Psi(S-bar)/Psi(S) of the configuration before the move, the uniform is the
    pair's Philox draw, and the decision is u < min(1, |Phi(S')/Phi(S)|^2)."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 19)
    W = inputs.sketch(4, chi, D, 7)
    c = inputs.start_spins(1, Ly, Lx, 3, "random")[0]
    tr = spin_inversion.PairTrace()
    new = spin_inversion.sweep(g, c, chi, W, 1, seed=321, pair=5, sweep_index=2, trace=tr)
    assert int(new.sum()) == 0 and len(tr.rows) > 0
    cur = c.copy()
    amp = exact.amplitude_transfer
    n_acc = 0
    for bond, rho, rho_b, w, u, acc in tr.rows:
        if bond < Lx * (Ly - 1):
            m, k = divmod(bond, Ly - 1)
            pts = ((k, m), (k + 1, m))
        else:
            k, m = divmod(bond - Lx * (Ly - 1), Lx - 1)
            pts = ((k, m), (k, m + 1))
        prop = cur.copy()
        for p in pts:
            prop[p] = -prop[p]
        a, ab, pa, pab = amp(g, cur), amp(g, -cur), amp(g, prop), amp(g, -prop)
        assert rho == pytest.approx(pa / a, rel=1e-9)
        assert rho_b == pytest.approx(pab / ab, rel=1e-9)
        assert w == pytest.approx(ab / a, rel=1e-8)
        assert u == philox.metropolis_uniform(321, 5, 2, bond)
        q = ((pa + pab) / (a + ab)) ** 2
        assert acc == (u < min(1.0, q))
        if acc:
            cur = prop
            n_acc += 1
    assert n_acc > 0 and np.array_equal(cur, new)


def z2_symmetric_peps(Ly, Lx, D, seed):
    """Tensors with A^{down} = (Z x Z x Z x Z) A^{up}, Z = diag(+1, -1, +1, ...) on every
    leg: Z appears twice on each inner bond, so Psi(S-bar) = Psi(S) for every S."""
    g = peps(Ly, Lx, D, seed)
    for row in g:
        for t in row:
            z = [np.array([(-1.0) ** i for i in range(n)]) for n in t.shape[1:]]
            t[1] = np.einsum("lrud,l,r,u,d->lrud", t[0], *z)
    return g


def test_symmetric_peps_reduces_to_the_plain_method():
    """With Psi(S-bar) = Psi(S): w = 1, E^Phi = E_loc, G^Phi puts G/2 in both slots, and
    the symmetrised sweep takes exactly the plain sweep's decisions."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = z2_symmetric_peps(Ly, Lx, D, 13)
    W = inputs.sketch(4, chi, D, 7)
    c = inputs.start_spins(1, Ly, Lx, 8, "random")[0]
    assert exact.amplitude_transfer(g, -c) == pytest.approx(exact.amplitude_transfer(g, c), rel=1e-12)
    r = spin_inversion.measure(g, c, chi, W, 1, 1.0, 0.5)
    assert r["w"] == pytest.approx(1.0, rel=1e-10)
    assert r["eloc_phi"] == pytest.approx(r["eloc"], rel=1e-10, abs=1e-12)
    k, m = 1, 2
    s = vmc.sidx(c[k, m])
    assert np.allclose(r["G"][k][m][s], r["plain"]["G"][k][m] / 2, rtol=1e-9, atol=1e-12)
    tp, ts = vmc.Trace(), spin_inversion.PairTrace()
    plain, _, _ = vmc.sweep(g, c, chi, W, 1, 77, 4, 1, trace=tp)
    sym = spin_inversion.sweep(g, c, chi, W, 1, 77, 4, 1, trace=ts)
    assert [row[3] for row in tp.rows] == [row[5] for row in ts.rows]
    assert np.array_equal(plain, sym)


@pytest.mark.slow
def test_sampled_histogram_matches_phi_squared():
    """Long symmetrised chain on 2x3: visit frequencies approach |Phi(S)|^2 / sum |Phi|^2
    (total variation)."""
    Ly, Lx, D, chi = 2, 3, 2, 2
    g = peps(Ly, Lx, D, 61)
    W = inputs.sketch(3, chi, D, 7)
    cfg, phi, index = phi_table(g)
    p = phi ** 2 / np.sum(phi ** 2)
    c = inputs.start_spins(1, Ly, Lx, 0, "neel")[0]
    hist = np.zeros(len(cfg))
    n = 3000
    for t in range(n):
        c = spin_inversion.sweep(g, c, chi, W, 1, 99, 0, t)
        hist[index[c.reshape(-1).tobytes()]] += 1
    tv = 0.5 * np.sum(np.abs(hist / n - p))
    assert tv < 0.06, tv
