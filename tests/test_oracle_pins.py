"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test names the pin it provides: brute force, closed forms, invariants, finite
differences, published known-answer vectors, and exactness of boundary-MPS
contraction once Dc >= D^(L/2) (App. B).
"""
import os

import numpy as np
import pytest

from oracle import exact, philox, vmc
from paper_1908_09359_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def peps(Ly, Lx, D, seed, normalise=False):
    return vmc.unpack(inputs.peps_tensors(Ly, Lx, D, seed, normalise), Ly, Lx, D)


def sk(L, chi, D, seed=7):
    return inputs.sketch(L, chi, D, seed)


def rand_cfg(Ly, Lx, seed):
    if (Ly * Lx) % 2:   # odd lattices: any +-1 pattern
        return np.random.default_rng(seed).choice(np.array([1, -1], dtype=np.int8), (Ly, Lx))
    return inputs.start_spins(1, Ly, Lx, seed, "random")[0]


# ------------------------------------------------------------------------ Philox (KAT)

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])
        out = philox.philox4x32_10_np(*[np.array([x], dtype=np.uint64) for x in v[0:6]])
        assert tuple(int(o[0]) for o in out) == tuple(v[6:10])


def test_uniform24_range_and_exactness():
    w = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.uniform24(w)
    assert list(u[:3]) == [0.0, 0.0, 2.0 ** -24]
    assert u[3] == 1.0 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


# ------------------------------------------------------------ P1 / P13: exact amplitudes

@pytest.mark.parametrize("Ly,Lx,D", [(2, 2, 3), (3, 3, 2), (2, 4, 2), (3, 2, 3)])
def test_transfer_equals_full_einsum(Ly, Lx, D):
    g = peps(Ly, Lx, D, 11 + D)
    for seed in range(3):
        c = rand_cfg(Ly, Lx, seed)
        a, b = exact.amplitude_transfer(g, c), exact.amplitude_einsum(g, c)
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


def test_single_row_is_matrix_product():
    """Ly = 1: Psi = l^T a_1 ... a_Lx r, a plain product of D x D matrices (P13)."""
    Lx, D = 6, 3
    g = peps(1, Lx, D, 5)
    c = rand_cfg(1, Lx, 1)
    mats = [g[0][m][vmc.sidx(c[0, m])][:, :, 0, 0] for m in range(Lx)]
    ref = np.linalg.multi_dot(mats)[0, 0]
    assert exact.amplitude_transfer(g, c) == pytest.approx(ref, rel=1e-12)
    for chi in (1, 2, 5):
        Ts, lT = vmc.top_envs(g, c, chi, sk(Lx, chi, 1), 1)
        Bs, lB = vmc.bottom_envs(g, c, chi, sk(Lx, chi, 1), 1)
        lp, s = vmc.row_psi(Ts[0], vmc.row_tensors(g, c, 0), Bs[0], lT[0], lB[0])
        assert s * np.exp(lp) == pytest.approx(ref, rel=1e-12)


# --------------------------------------------- P2 / P3: exactness at Dc >= D^(L/2), App. B

@pytest.mark.parametrize("Ly,Lx,D,chi,n_fit", [(4, 4, 2, 4, 1), (4, 4, 2, 4, 3),
                                               (3, 3, 3, 3, 1), (4, 3, 2, 4, 1),
                                               (5, 4, 2, 4, 3), (4, 4, 3, 9, 1)])
def test_boundary_mps_exact_every_row(Ly, Lx, D, chi, n_fit):
    g = peps(Ly, Lx, D, 100 + Ly * Lx + D)
    W = sk(max(Ly, Lx), chi, D)
    for seed in range(2):
        c = rand_cfg(Ly, Lx, seed)
        ref = exact.amplitude_transfer(g, c)
        Ts, lT = vmc.top_envs(g, c, chi, W, n_fit)
        Bs, lB = vmc.bottom_envs(g, c, chi, W, n_fit)
        for k in range(Ly):
            lp, s = vmc.row_psi(Ts[k], vmc.row_tensors(g, c, k), Bs[k], lT[k], lB[k])
            assert s * np.exp(lp) == pytest.approx(ref, rel=1e-10), k


def test_three_and_four_line_closures_agree():
    """Tr[L0(m) R0(m+1)] is the same for every m (App. C) and equals the four-line
    closure of every row pair and the exact amplitude."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 3)
    W = sk(4, chi, D)
    c = rand_cfg(Ly, Lx, 9)
    ref = exact.amplitude_transfer(g, c)
    Ts, lT = vmc.top_envs(g, c, chi, W, 1)
    Bs, lB = vmc.bottom_envs(g, c, chi, W, 1)
    for k in range(Ly):
        T, B = Ts[k], Bs[k]
        row = vmc.row_tensors(g, c, k)
        Ls = [np.ones((1, 1, 1))]
        for m in range(Lx):
            Ls.append(vmc.env3_left(Ls[-1], T[m], row[m], B[m]))
        Rs = [np.ones((1, 1, 1))]
        for m in range(Lx - 1, -1, -1):
            Rs.insert(0, vmc.env3_right(Rs[0], T[m], row[m], B[m]))
        scale = np.exp(lT[k] + lB[k])
        for m in range(Lx + 1):
            assert np.vdot(Ls[m], Rs[m]) * scale == pytest.approx(ref, rel=1e-10)
    for k in range(Ly - 1):
        T, B = Ts[k], Bs[k + 1]
        E = np.ones((1, 1, 1, 1))
        for m in range(Lx):
            a1 = g[k][m][vmc.sidx(c[k, m])]
            a2 = g[k + 1][m][vmc.sidx(c[k + 1, m])]
            E = vmc.env4_left(E, T[m], a1, a2, B[m])
        assert float(E.reshape(())) * np.exp(lT[k] + lB[k + 1]) == pytest.approx(ref, rel=1e-10)


# ------------------------------------------------------------- truncated regime, App. B

def _dense(mps):
    v = mps[0]
    for t in mps[1:]:
        v = np.tensordot(v, t, axes=([-1], [0]))
    return v.reshape(-1)


def _svd_truncate_dense(vec, phys, r):
    """Successive SVD truncation of a dense vector to an MPS with bonds r (textbook TT-SVD)."""
    L = len(phys)
    sites, rest, left = [], vec.reshape(1, -1), 1
    for m in range(L - 1):
        M = rest.reshape(left * phys[m], -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        k = min(r[m], len(S))
        sites.append(U[:, :k].reshape(left, phys[m], k))
        rest = S[:k, None] * Vt[:k]
        left = k
    sites.append(rest.reshape(left, phys[-1], 1))
    return sites


def test_fit_between_optimal_bound_and_tt_svd():
    """At finite Dc the fit error lies between the Eckart-Young bound (no MPS of bond r
    can do better at any cut) and the error of plain TT-SVD truncation."""
    rng = np.random.default_rng(4)
    L, p, chiX, chi = 6, 2, 6, 3
    X = [rng.standard_normal((1 if m == 0 else chiX, p, 1 if m == L - 1 else chiX))
         for m in range(L)]
    x = _dense(X)
    r = vmc.bond_caps([chiX] * (L - 1), [p] * L, chi)
    W = sk(L, chi, p, 21)
    errs = []
    for n_fit in (1, 3, 9, 21):
        V, ln = vmc.compress(X, chi, W, n_fit)
        v = _dense(V) * np.exp(ln)
        # the fit output is the orthogonal projection of X on its final basis
        errs.append(np.linalg.norm(x - v) / np.linalg.norm(x))
    lower = 0.0
    for m in range(L - 1):
        S = np.linalg.svd(x.reshape(p ** (m + 1), -1), compute_uv=False)
        lower = max(lower, np.sqrt(np.sum(S[r[m]:] ** 2)) / np.linalg.norm(x))
    tt = _dense(_svd_truncate_dense(x, [p] * L, r))
    upper = np.linalg.norm(x - tt) / np.linalg.norm(x)
    assert all(e >= lower * (1 - 1e-9) for e in errs)
    assert errs[-1] <= upper * (1 + 1e-6)
    assert errs[2] <= errs[0] + 1e-12


def test_svd_truncation_is_right_to_left_tt_svd():
    """The SVD truncation mode (App. B's truncation done by SVD instead of the fit) equals
    textbook TT-SVD of the dense vector run from the right end, its output is
    left-orthonormal and normalised, and at Dc >= the exact bonds it reproduces X."""
    rng = np.random.default_rng(6)
    L, p, chiX, chi = 6, 2, 6, 3
    X = [rng.standard_normal((1 if m == 0 else chiX, p, 1 if m == L - 1 else chiX)) for m in range(L)]
    x = _dense(X)
    r = vmc.bond_caps([chiX] * (L - 1), [p] * L, chi)
    V, ln = vmc.compress_svd(X, chi)
    v = _dense(V) * np.exp(ln)
    xr = x.reshape((p,) * L).transpose(tuple(range(L - 1, -1, -1))).reshape(-1)
    tt = _dense(_svd_truncate_dense(xr, [p] * L, r[::-1]))
    ref = tt.reshape((p,) * L).transpose(tuple(range(L - 1, -1, -1))).reshape(-1)
    assert np.linalg.norm(v - ref) <= 1e-10 * np.linalg.norm(ref)
    for t in V[:-1]:
        M = t.reshape(-1, t.shape[2])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-12)
    assert np.linalg.norm(V[-1]) == pytest.approx(1.0, rel=1e-14)
    V, ln = vmc.compress(X, 64, None, 0)
    assert np.linalg.norm(_dense(V) * np.exp(ln) - x) <= 1e-10 * np.linalg.norm(x)


def test_svd_mode_boundary_mps_exact_at_full_dc():
    """Both truncation modes give the exact amplitude through the whole contraction once
    Dc >= D^(L/2) (4x4, D = 2, Dc = 4), and agree with each other there."""
    g = peps(4, 4, 2, 12)
    W = sk(4, 4, 2)
    for seed in range(3):
        c = rand_cfg(4, 4, seed)
        ref = exact.amplitude_transfer(g, c)
        for n_fit in (0, 1):
            r = vmc.measure(g, c, 4, W, n_fit, 1.0, 0.5, want_grad=False)
            assert r["sign"] * np.exp(r["logpsi"]) == pytest.approx(ref, rel=1e-10)


def test_fit_output_left_orthonormal_and_normalised():
    rng = np.random.default_rng(2)
    X = [rng.standard_normal((1 if m == 0 else 8, 3, 1 if m == 4 else 8)) for m in range(5)]
    V, _ = vmc.compress(X, 5, sk(5, 5, 3), 3)
    for t in V[:-1]:
        M = t.reshape(-1, t.shape[2])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-12)
    assert np.linalg.norm(V[-1]) == pytest.approx(1.0, rel=1e-14)


# -------------------------------------------------- P4: E_loc against direct enumeration

@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_mean_eloc_equals_exact_energy(J2):
    """sum_S |Psi|^2 E_loc(S) / Z (Eq. (2)) with the boundary-MPS E_loc at exact Dc equals
    <Psi|H|Psi>/<Psi|Psi> from H applied to the full amplitude vector."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 31)
    W = sk(4, chi, D)
    E_ref, cfg, psi = exact.energy_exact(g, 1.0, J2)
    w = psi ** 2 / np.sum(psi ** 2)
    idx = np.argsort(-w)[:400]   # the heaviest configurations carry almost all weight
    el = np.array([vmc.measure(g, cfg[i], chi, W, 1, 1.0, J2, want_grad=False)["eloc"]
                   for i in idx])
    # E_loc of the same configurations straight from exact amplitudes of every S'
    flat = cfg.reshape(len(cfg), -1)
    index = {c.tobytes(): n for n, c in enumerate(flat)}
    direct = []
    for i in idx:
        c = flat[i]
        e = 0.0
        for a, b, J in exact.bonds(Ly, Lx, 1.0, J2):
            e += J * c[a] * c[b] / 4.0
            if c[a] != c[b]:
                c2 = c.copy()
                c2[a], c2[b] = c[b], c[a]
                e += 0.5 * J * psi[index[c2.tobytes()]] / psi[i]
        direct.append(e)
    assert np.allclose(el, direct, rtol=1e-9, atol=1e-9)
    # E_tot from all configurations with the direct E_loc equals the H-apply route
    full = 0.0
    for i, c in enumerate(flat):
        e = 0.0
        for a, b, J in exact.bonds(Ly, Lx, 1.0, J2):
            e += J * c[a] * c[b] / 4.0
            if c[a] != c[b]:
                c2 = c.copy()
                c2[a], c2[b] = c[b], c[a]
                e += 0.5 * J * psi[index[c2.tobytes()]] / psi[i]
        full += w[i] * e
    assert full == pytest.approx(E_ref, rel=1e-10)


# ------------------------------------------------------------ P5: D = 1 product states

def test_product_state_closed_forms():
    Ly, Lx = 3, 4
    g = peps(Ly, Lx, 1, 8)
    c = rand_cfg(Ly, Lx, 2)
    W = sk(4, 2, 1)
    r = vmc.measure(g, c, 2, W, 1, 1.0, 0.5)
    amp = lambda k, m, s: g[k][m][vmc.sidx(s)].reshape(())
    psi = np.prod([amp(k, m, c[k, m]) for k in range(Ly) for m in range(Lx)])
    assert r["sign"] * np.exp(r["logpsi"]) == pytest.approx(psi, rel=1e-12)
    e = 0.0
    for a, b, J in exact.bonds(Ly, Lx, 1.0, 0.5):
        (ka, ma), (kb, mb) = divmod(a, Lx), divmod(b, Lx)
        sa, sb = c[ka, ma], c[kb, mb]
        e += J * sa * sb / 4
        if sa != sb:
            e += 0.5 * J * amp(ka, ma, sb) * amp(kb, mb, sa) / (amp(ka, ma, sa) * amp(kb, mb, sb))
    assert r["eloc"] == pytest.approx(e, rel=1e-12)
    for k in range(Ly):
        for m in range(Lx):
            assert r["G"][k][m].reshape(()) == pytest.approx(1.0 / amp(k, m, c[k, m]), rel=1e-12)


# ------------------------------------------------- P6 / P7: G against Euler and FD of ln Psi

def test_euler_identity_at_finite_dc():
    """Psi is linear in each tensor, so <G_k, a_k> = 1 at every site, truncated or not."""
    Ly, Lx, D, chi = 5, 5, 3, 4
    g = peps(Ly, Lx, D, 12)
    c = rand_cfg(Ly, Lx, 1)
    r = vmc.measure(g, c, chi, sk(5, chi, D), 3, 1.0, 0.5)
    for k in range(Ly):
        for m in range(Lx):
            a = g[k][m][vmc.sidx(c[k, m])]
            assert np.sum(r["G"][k][m] * a) == pytest.approx(1.0, abs=1e-10)


def test_G_equals_finite_difference_of_ln_psi():
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 44)
    c = rand_cfg(Ly, Lx, 5)
    r = vmc.measure(g, c, chi, sk(4, chi, D), 1, 1.0, 0.0)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(12):
        k, m = rng.integers(Ly), rng.integers(Lx)
        s = vmc.sidx(c[k, m])
        shp = g[k][m].shape[1:]
        idx = tuple(rng.integers(n) for n in shp)
        vals = []
        for sgn in (1, -1):
            g2 = [[t.copy() for t in row] for row in g]
            g2[k][m][(s,) + idx] += sgn * h
            vals.append(np.log(abs(exact.amplitude_transfer(g2, c))))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert r["G"][k][m][idx] == pytest.approx(fd, rel=1e-6, abs=1e-7)


# ----------------------------------------------------- P8: energy gradient (Alg. 1, Eq. (5))

def test_gradient_matches_fd_of_exact_energy():
    """2(<G E_loc> - <G><E_loc>) with exact |Psi|^2 weights equals dE_tot/dA by FD."""
    Ly, Lx, D, chi = 2, 4, 2, 2
    g = peps(Ly, Lx, D, 77)
    W = sk(4, chi, D)
    E0, cfg, psi = exact.energy_exact(g, 1.0, 0.5)
    wts = psi ** 2 / np.sum(psi ** 2)
    acc = [[np.zeros_like(t) for t in row] for row in g]
    accE = [[np.zeros_like(t) for t in row] for row in g]
    Ebar = 0.0
    for wgt, c in zip(wts, cfg):
        r = vmc.measure(g, c, chi, W, 1, 1.0, 0.5)
        Ebar += wgt * r["eloc"]
        for k in range(Ly):
            for m in range(Lx):
                s = vmc.sidx(c[k, m])
                acc[k][m][s] += wgt * r["G"][k][m]
                accE[k][m][s] += wgt * r["G"][k][m] * r["eloc"]
    assert Ebar == pytest.approx(E0, rel=1e-10)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(10):
        k, m = rng.integers(Ly), rng.integers(Lx)
        idx = tuple(rng.integers(n) for n in g[k][m].shape)
        grad = accE[k][m][idx] - acc[k][m][idx] * Ebar
        vals = []
        for sgn in (1, -1):
            g2 = [[t.copy() for t in row] for row in g]
            g2[k][m][idx] += sgn * h
            vals.append(exact.energy_exact(g2, 1.0, 0.5)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert 2 * grad == pytest.approx(fd, rel=1e-5, abs=1e-8)


# --------------------------------------------------------- sampler: ratios and rule, Eq. (9)

def test_sweep_ratios_are_exact_amplitude_ratios():
    """Every proposal's ratio equals Psi(S_b)/Psi(S_a) by brute force at exact Dc, the
    decision is r < min(1, ratio^2), and S^z is conserved (P14)."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 19)
    W = sk(4, chi, D)
    c = inputs.start_spins(1, Ly, Lx, 0, "neel")[0]
    tr = vmc.Trace()
    new, Ts, lT = vmc.sweep(g, c, chi, W, 1, seed=123, chain=0, sweep_index=0, trace=tr)
    assert int(new.sum()) == 0 and len(tr.rows) > 0
    # replay: walk the bond list, rebuild each S_a and S_b, check ratio and decision
    cur = c.copy()
    for bond, rho, u, acc in tr.rows:
        if bond < Lx * (Ly - 1):
            m, k = divmod(bond, Ly - 1)
            pts = ((k, m), (k + 1, m))
        else:
            k, m = divmod(bond - Lx * (Ly - 1), Lx - 1)
            pts = ((k, m), (k, m + 1))
        prop = cur.copy()
        for p in pts:
            prop[p] = -prop[p]
        ref = exact.amplitude_transfer(g, prop) / exact.amplitude_transfer(g, cur)
        assert rho == pytest.approx(ref, rel=1e-9)
        assert u == philox.metropolis_uniform(123, 0, 0, bond)
        assert acc == (u < min(1.0, rho * rho))
        if acc:
            cur = prop
    assert np.array_equal(cur, new)
    # T_k returned by the sweep are environments of the final configuration
    ref = exact.amplitude_transfer(g, new)
    Bs, lB = vmc.bottom_envs(g, new, chi, W, 1)
    for k in range(Ly):
        lp, s = vmc.row_psi(Ts[k], vmc.row_tensors(g, new, k), Bs[k], lT[k], lB[k])
        assert s * np.exp(lp) == pytest.approx(ref, rel=1e-10)


def test_horizontal_only_moves_cannot_change_row_magnetisation():
    """Sweeping only one kind of bond is not ergodic (Sec. II A): horizontal swaps
    conserve the magnetisation of every row, so both kinds are needed."""
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 23)
    W = sk(4, chi, D)
    c = inputs.start_spins(1, Ly, Lx, 0, "neel")[0].copy()
    rows0 = c.sum(axis=1).copy()
    seen_change = False
    for t in range(6):
        vmc._row_phase(g, c, chi, W, 1, 5, 0, t, 1000, None)
        assert np.array_equal(c.sum(axis=1), rows0)
    for t in range(6):
        c, _, _ = vmc.sweep(g, c, chi, W, 1, 5, 0, 10 + t)
        seen_change |= not np.array_equal(c.sum(axis=1), rows0)
    assert seen_change


@pytest.mark.slow
def test_sampled_histogram_matches_psi_squared():
    """Long chain on 2x3: visit frequencies approach |Psi(S)|^2/Z (total variation)."""
    Ly, Lx, D, chi = 2, 3, 2, 2
    g = peps(Ly, Lx, D, 61)
    W = sk(3, chi, D)
    _, cfg, psi = exact.energy_exact(g, 1.0, 0.0)
    p = psi ** 2 / np.sum(psi ** 2)
    index = {cc.tobytes(): n for n, cc in enumerate(cfg.reshape(len(cfg), -1))}
    c = inputs.start_spins(1, Ly, Lx, 0, "neel")[0]
    hist = np.zeros(len(cfg))
    n = 3000
    for t in range(n):
        c, _, _ = vmc.sweep(g, c, chi, W, 1, 99, 0, t)
        hist[index[c.reshape(-1).tobytes()]] += 1
    tv = 0.5 * np.sum(np.abs(hist / n - p))
    assert tv < 0.06, tv


# ------------------------------------------------------- P10 / P12: symmetries, invariants

def test_transpose_invariance():
    Ly, Lx, D, chi = 4, 4, 2, 4
    g = peps(Ly, Lx, D, 90)
    W = sk(4, chi, D)
    c = rand_cfg(Ly, Lx, 3)
    a = vmc.measure(g, c, chi, W, 1, 1.0, 0.5, want_grad=False)
    b = vmc.measure(vmc.transpose_lattice(g), np.ascontiguousarray(c.T), chi, W, 1, 1.0, 0.5,
                    want_grad=False)
    assert a["eloc"] == pytest.approx(b["eloc"], rel=1e-10)
    assert a["logpsi"] == pytest.approx(b["logpsi"], rel=1e-12)


def test_scaling_one_tensor():
    """A_k -> c A_k: ratios and E_loc unchanged, G_k -> G_k/c, ln|Psi| -> ln|Psi| + ln c
    (finite Dc, because the fit is homogeneous in each row)."""
    Ly, Lx, D, chi = 5, 4, 3, 5
    g = peps(Ly, Lx, D, 15)
    W = sk(5, chi, D)
    c = rand_cfg(Ly, Lx, 8)
    a = vmc.measure(g, c, chi, W, 3, 1.0, 0.5)
    g2 = [[t.copy() for t in row] for row in g]
    g2[2][1] *= 3.0
    b = vmc.measure(g2, c, chi, W, 3, 1.0, 0.5)
    assert b["eloc"] == pytest.approx(a["eloc"], rel=1e-9)
    assert b["logpsi"] == pytest.approx(a["logpsi"] + np.log(3.0), rel=1e-12)
    assert np.allclose(b["G"][2][1], a["G"][2][1] / 3.0, rtol=1e-9, atol=1e-12)
    assert np.allclose(b["G"][0][0], a["G"][0][0], rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------- sign-SGD, Eq. (10)

def test_sign_sgd_step():
    rng = np.random.default_rng(0)
    A = rng.standard_normal(1000)
    gr = rng.standard_normal(1000)
    gr[::7] = 0.0
    new = vmc.sign_sgd(A, gr, 0.02, seed=5, step=3)
    d = new - A
    r = philox.update_uniforms(5, 3, 1000)
    assert np.all(np.abs(d) <= 0.02)
    assert np.all(d[gr > 0] <= 0) and np.all(d[gr < 0] >= 0) and np.all(d[gr == 0] == 0)
    assert np.allclose(np.abs(d[gr != 0]), 0.02 * r[gr != 0], rtol=0, atol=1e-15)
    w0 = philox.philox4x32_10((17, 0, 3, philox.TAG_UPDATE), philox.key_of(5))[0]
    assert r[17] == (w0 >> 8) * 2.0 ** -24


def test_accumulator_gradient_formula():
    """P1/M - (P2/M) E_tot/M of Algorithm 1 on two hand-made samples."""
    g = peps(1, 2, 1, 3)
    acc = vmc.Accumulator(g)
    G1 = [[np.full((1, 1, 1, 1), 2.0), np.full((1, 1, 1, 1), 3.0)]]
    G2 = [[np.full((1, 1, 1, 1), 5.0), np.full((1, 1, 1, 1), 7.0)]]
    acc.add(np.array([[1, -1]]), -1.0, G1)
    acc.add(np.array([[1, 1]]), -3.0, G2)
    grad, E = acc.gradient()
    assert E == -2.0
    # site 0 slot 0: <G E> = (2*-1 + 5*-3)/2 = -8.5 ; <G> = 3.5 ; grad = -8.5 + 7 = -1.5
    assert grad[0][0][0].item() == pytest.approx(-1.5)
    # site 1 slot 1 (sigma=-1) only in sample 1: <G E> = -1.5, <G> = 1.5, grad = -1.5 + 3 = 1.5
    assert grad[0][1][1].item() == pytest.approx(1.5)
    assert grad[0][1][0].item() == pytest.approx(-10.5 + 7.0)


# ------------------------------------------------ P11: sequential vs random-NNASP sampling

def test_random_nnasp_and_sequential_sweep_share_the_stationary_distribution():
    """Sec. II A: the random-NNASP rule with its 1/K proposal factors and the sequential
    sweep both leave |Psi|^2 invariant, so their stationary energies agree (the paper's
    validation of the sequential scheme).  Exact transition matrices over the S^z = 0
    sector of 2x4 (70 configurations); dropping the 1/K factors breaks detailed balance."""
    from oracle import random_nnasp as rn
    Ly, Lx = 2, 4
    g = peps(Ly, Lx, 2, 77)
    cfg, psi = rn.sector(g)
    pi = psi ** 2 / np.sum(psi ** 2)
    Pr = rn.random_scheme_matrix(cfg, psi, Ly, Lx)
    Ps = rn.sequential_sweep_matrix(cfg, psi, Ly, Lx)
    for P in (Pr, Ps):
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12) and np.all(P >= -1e-15)
        assert np.max(np.abs(pi @ P - pi)) <= 1e-12
    flow = pi[:, None] * Pr
    assert np.max(np.abs(flow - flow.T)) <= 1e-12                      # detailed balance
    assert np.max(np.abs(rn.stationary(Pr) - rn.stationary(Ps))) <= 1e-9
    E, _, _ = exact.energy_exact(g, 1.0, 0.0)
    eloc = np.array([vmc.measure(g, c, 4, sk(4, 4, 2), 1, 1.0, 0.0, want_grad=False)["eloc"] for c in cfg])
    assert float(rn.stationary(Pr) @ eloc) == pytest.approx(E, abs=1e-10)
    assert float(rn.stationary(Ps) @ eloc) == pytest.approx(E, abs=1e-10)
    wrong = rn.random_scheme_matrix(cfg, psi, Ly, Lx, with_k=False)
    assert np.max(np.abs(pi @ wrong - pi)) > 1e-4                      # the 1/K factors matter


# -------------------------------------------- P11: the random-NNASP sampler (Sec. II A)

def test_random_attempt_reproduces_the_transition_matrix():
    """The Philox-driven random-NNASP attempt (Eq. (prob_r)) on 2x4 at exact Dc: for every
    configuration and every pair index, the trial it builds and the acceptance probability
    min[1, |Psi_b|^2 K_a / (|Psi_a|^2 K_b)] it applies equal the transition matrix entry
    K_a P[a, b] of the exact random scheme, whose stationary law is |Psi|^2 (pinned above);
    and a uniform just below / above that probability is accepted / rejected."""
    from oracle import random_nnasp as rn
    g = peps(2, 4, 2, 17)
    W = inputs.sketch(4, 4, 2, 17)
    cfg, psi = rn.sector(g)
    P = rn.random_scheme_matrix(cfg, psi, 2, 4)
    index = {c.tobytes(): n for n, c in enumerate(cfg.reshape(len(cfg), -1))}
    for a in range(0, len(cfg), 7):
        pairs = rn.nnasps(cfg[a].ravel(), rn.nn_bonds(2, 4))
        K = len(pairs)
        for i in range(K):
            m = -(-(i << 24) // K)  # smallest 24-bit m with floor(m K / 2^24) = i
            word = m << 8
            assert philox.pick(word, K) == i
            rec = []
            new, _ = rn.attempt_with(g, cfg[a], 4, W, 1, word, 0.0, None, rec)
            bond, rho, Ka, Kb, acc = rec[0]
            b = index[new.tobytes()]
            p_acc = min(1.0, rho * rho * Ka / Kb)
            assert Ka == K and acc
            assert p_acc == pytest.approx(K * P[a, b], rel=1e-9, abs=1e-12)
            assert rho == pytest.approx(psi[b] / psi[a], rel=1e-9)
            if p_acc < 1.0:
                rec = []
                rn.attempt_with(g, cfg[a], 4, W, 1, word, p_acc * (1 + 1e-9), None, rec)
                assert not rec[0][4]
            assert int(new.sum()) == int(cfg[a].sum())


def test_random_sweep_keeps_sz_and_counts_attempts():
    from oracle import random_nnasp as rn
    g = peps(4, 4, 2, 3)
    W = inputs.sketch(4, 4, 2, 3)
    s0 = inputs.start_spins(1, 4, 4, 9, "random")[0]
    rec = []
    s1 = rn.random_sweep(g, s0, 4, W, 1, 5, 0, 0, record=rec)
    assert len(rec) == 16 and int(s1.sum()) == 0
    assert any(r[4] for r in rec)
