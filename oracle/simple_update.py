"""Simple-update imaginary-time evolution (App. A) -- the initialiser of the optimisation.

Test infrastructure only (see the package header).  The PEPS is held as site tensors
B[k][m] of shape (2, Dl, Dr, Du, Dd) (index order and spin slots as in ``vmc``) and one
diagonal matrix, a vector lambda, on every nearest-neighbour link; the environment of a
tensor is approximated by the lambdas on its legs.  One evolution operator exp(-tau h)
of a bond updates the tensors it touches:

* NN bond (sites 1, 2): each tensor with the lambdas of its three outer legs absorbed is
  reduced by a QR (rows: outer legs; columns: bond leg and spin), the gate acts on the
  two R factors joined by the bond's lambda, an SVD truncated to D gives the new bond
  lambda and the new R factors, and the outer lambdas are divided out again.
* NNN bond (sites 1 and 3, through the corner site 2 that shares a link with each):
  the steps of App. A's figure -- QR of B1 and of B3 with their outer lambdas, the gate
  contracted with R1, R3 and B2 (with B2's outer lambdas and both link lambdas) into
  T_a, a truncated SVD of T_a giving R1-tilde, lambda-tilde(1,2) and T_b, a truncated SVD
  of lambda-tilde(1,2) T_b giving T_c, lambda-tilde(2,3) and L3-tilde, then B1-tilde,
  B2-tilde and B3-tilde with the inverse lambdas divided out.
Each new lambda is normalised to unit 2-norm.  The final PEPS for the Monte Carlo
stage carries lambda^(1/2) of every link absorbed into each of its two tensors (App. A).

Readings of points the paper leaves open:
* Gates: h = J S_i.S_j with S = sigma/2 (the Hamiltonian of the energy, Eq. (2));
  exp(-tau J S.S) = e^{-tau J/4} P_triplet + e^{3 tau J/4} P_singlet.
* Trotter order (first order) of one step: horizontal NN bonds with m even, then m odd,
  vertical NN bonds with k even, then k odd (all with tau); then, when J2 != 0, for
  each plaquette diagonal (k,m)-(k+1,m+1) and (k,m+1)-(k+1,m) and each of its two
  corner paths, the plaquettes in four groups by (k mod 2, m mod 2), each NNN gate with
  tau/2 so that the two paths of a diagonal together make one step tau.  The bonds of a
  group share no site, so their order inside the group does not matter.
* Truncation keeps the min(D, r) largest singular values, r the number above 1e-7 of the
  largest; the bond dimension of an inner link is D from the start (random initial
  tensors, lambda = 1) and stays D: when r < D the missing lambda entries and the
  matching tensor slices are zero.
* QR with diag(R) >= 0 (``vmc.qr_pos``); SVD singular vectors with their largest-magnitude
  entry made positive (any fixed rule would do; this one makes the tensors a function of
  the input up to degenerate singular values).
* Inverse lambdas: 1/lambda for lambda > 1e-14 max(lambda), else 0.
* Convergence (App. A): mean over links of ||lambda(t+tau) - lambda(t)|| / ||lambda(t)||
  below ``tol``.
"""
from __future__ import annotations

import numpy as np

from .vmc import qr_pos

LEGS = {"l": 1, "r": 2, "u": 3, "d": 4}


def heisenberg_gate(J, tau):
    """G[s1', s2', s1, s2] = <s1' s2'| exp(-tau J S1.S2) |s1 s2>, slot 0 = spin up."""
    # S1.S2 in the basis (uu, ud, du, dd)
    h = np.array([[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]])
    p_singlet = 0.25 * np.eye(4) - h
    p_triplet = 0.75 * np.eye(4) + h
    g = np.exp(-tau * J / 4) * p_triplet + np.exp(3 * tau * J / 4) * p_singlet
    return g.reshape(2, 2, 2, 2)


class State:
    """Site tensors B[k][m] (2, Dl, Dr, Du, Dd) and link vectors lh[k][m] (link (k,m)-(k,m+1))
    and lv[k][m] (link (k,m)-(k+1,m))."""

    def __init__(self, B, lh, lv):
        self.B, self.lh, self.lv = B, lh, lv
        self.Ly, self.Lx = len(B), len(B[0])

    def copy(self):
        return State([[t.copy() for t in row] for row in self.B], [[x.copy() for x in r] for r in self.lh],
                     [[x.copy() for x in r] for r in self.lv])

    def lam(self, p, q):
        (k1, m1), (k2, m2) = sorted([p, q])
        return self.lh[k1][m1] if k1 == k2 else self.lv[k1][m1]

    def set_lam(self, p, q, v):
        (k1, m1), (k2, m2) = sorted([p, q])
        if k1 == k2:
            self.lh[k1][m1] = v
        else:
            self.lv[k1][m1] = v

    def links(self):
        return [x for r in self.lh for x in r] + [x for r in self.lv for x in r]


def init_state(Ly, Lx, D, seed):
    """Random start: iid N(0,1) site tensors, each of unit norm, every lambda = 1."""
    rng = np.random.default_rng(seed)
    B = []
    for k in range(Ly):
        row = []
        for m in range(Lx):
            shape = (2, 1 if m == 0 else D, 1 if m == Lx - 1 else D, 1 if k == 0 else D, 1 if k == Ly - 1 else D)
            t = rng.standard_normal(shape)
            row.append(t / np.linalg.norm(t))
        B.append(row)
    lh = [[np.ones(D) for _ in range(Lx - 1)] for _ in range(Ly)]
    lv = [[np.ones(D) for _ in range(Lx)] for _ in range(Ly - 1)]
    return State(B, lh, lv)


def direction(p, q):
    """Leg of site p that points to its neighbour q."""
    dk, dm = q[0] - p[0], q[1] - p[1]
    return {(0, 1): "r", (0, -1): "l", (1, 0): "d", (-1, 0): "u"}[(dk, dm)]


def neighbours(st, p):
    k, m = p
    out = {}
    if m > 0:
        out["l"] = (k, m - 1)
    if m < st.Lx - 1:
        out["r"] = (k, m + 1)
    if k > 0:
        out["u"] = (k - 1, m)
    if k < st.Ly - 1:
        out["d"] = (k + 1, m)
    return out


def _scale(t, leg, v):
    shape = [1] * 5
    shape[LEGS[leg]] = len(v)
    return t * v.reshape(shape)


def _inv(v):
    cut = 1e-14 * np.max(np.abs(v))
    return np.where(np.abs(v) > cut, 1.0 / np.where(np.abs(v) > cut, v, 1.0), 0.0)


def _svd(M):
    """SVD with each singular vector pair's sign fixed by the largest-magnitude entry of u."""
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    for i in range(len(S)):
        j = np.argmax(np.abs(U[:, i]))
        if U[j, i] < 0:
            U[:, i] *= -1
            Vt[i] *= -1
    return U, S, Vt


def _keep(S, D):
    """Kept count n and the normalised lambda, zero-padded to length D."""
    n = min(D, int(np.count_nonzero(S > 1e-7 * S[0]))) if S[0] > 0 else 0
    lam = np.zeros(D)
    if n:
        lam[:n] = S[:n] / np.linalg.norm(S[:n])
    return n, lam


def _pad_cols(U, n, D):
    out = np.zeros((U.shape[0], D))
    out[:, :n] = U[:, :n]
    return out


def _reduce(st, p, bond_leg):
    """(Q, R, outer legs, outer shape) of site p with the lambdas of its outer legs (all but
    bond_leg) absorbed: rows = outer legs in (l, r, u, d) order, columns = (bond leg, spin)."""
    t = st.B[p[0]][p[1]]
    nb = neighbours(st, p)
    outer = [g for g in "lrud" if g != bond_leg]
    for g in outer:
        if g in nb:
            t = _scale(t, g, st.lam(p, nb[g]))
    axes = [LEGS[g] for g in outer] + [LEGS[bond_leg], 0]
    tt = np.transpose(t, axes)
    oshape = tt.shape[:3]
    Q, R = qr_pos(tt.reshape(int(np.prod(oshape)), -1))
    return Q, R.reshape(R.shape[0], tt.shape[3], 2), outer, oshape


def _rebuild(st, p, Q, Rt, outer, oshape, bond_leg):
    """B(p) from Q (outer x k) and Rt[x, spin, bond]: outer lambdas divided out, legs
    back in (s, l, r, u, d) order."""
    M = (Q @ Rt.reshape(Rt.shape[0], -1)).reshape(*oshape, 2, Rt.shape[2])
    order = outer + ["s", bond_leg]
    t = np.transpose(M, [order.index(g) for g in ["s", "l", "r", "u", "d"]])
    nb = neighbours(st, p)
    for g in outer:
        if g in nb:
            t = _scale(t, g, _inv(st.lam(p, nb[g])))
    return t


def nn_update(st, p1, p2, gate, D):
    """Apply the two-site gate G[s1', s2', s1, s2] to the NN bond (p1, p2) in place."""
    g1, g2 = direction(p1, p2), direction(p2, p1)
    Q1, R1, o1, s1 = _reduce(st, p1, g1)
    Q2, R2, o2, s2 = _reduce(st, p2, g2)
    lam = st.lam(p1, p2)
    th = np.einsum("xas,a,yat,uvst->xuyv", R1, lam, R2, gate)
    k1, k2 = R1.shape[0], R2.shape[0]
    U, S, Vt = _svd(th.reshape(k1 * 2, k2 * 2))
    n, lam_new = _keep(S, D)
    Rt1 = _pad_cols(U, n, D).reshape(k1, 2, D)
    Rt2 = _pad_cols(Vt.T, n, D).reshape(k2, 2, D)
    st.set_lam(p1, p2, lam_new)
    st.B[p1[0]][p1[1]] = _rebuild(st, p1, Q1, Rt1, o1, s1, g1)
    st.B[p2[0]][p2[1]] = _rebuild(st, p2, Q2, Rt2, o2, s2, g2)


def nnn_update(st, p1, p2, p3, gate, D):
    """Apply the gate G[s1', s3', s1, s3] to the NNN pair (p1, p3) through the corner p2
    (App. A, steps (b)-(h) of its figure), in place."""
    a1, a2 = direction(p1, p2), direction(p2, p1)
    b2, b3 = direction(p2, p3), direction(p3, p2)
    Q1, R1, o1, s1 = _reduce(st, p1, a1)      # (b)
    Q3, R3, o3, s3 = _reduce(st, p3, b3)
    lam_a, lam_b = st.lam(p1, p2), st.lam(p2, p3)
    t2 = st.B[p2[0]][p2[1]]
    nb2 = neighbours(st, p2)
    outer2 = [g for g in "lrud" if g not in (a2, b2)]
    for g in outer2:
        if g in nb2:
            t2 = _scale(t2, g, st.lam(p2, nb2[g]))
    t2 = _scale(_scale(t2, a2, lam_a), b2, lam_b)
    M2 = np.transpose(t2, [0, LEGS[a2], LEGS[b2]] + [LEGS[g] for g in outer2])  # (s2, a, b, o, o')
    Ta = np.einsum("xas,tabop,zbu,vwsu->xvtopzw", R1, M2, R3, gate)             # (c)
    k1, k3 = R1.shape[0], R3.shape[0]
    o, op = M2.shape[3], M2.shape[4]
    U1, S1, V1t = _svd(Ta.reshape(k1 * 2, -1))                                   # (d)
    n1, la = _keep(S1, D)
    Tb = (la[:, None] * _pad_cols(V1t.T, n1, D).T).reshape(D * 2 * o * op, k3 * 2)  # (a', s2, o, o') x (z, s3')
    U2, S2, V2t = _svd(Tb)                                                       # (e)
    n2, lb = _keep(S2, D)
    Tc = _pad_cols(U2, n2, D).reshape(D, 2, o, op, D)                            # (a', s2, o, o', b')
    st.set_lam(p1, p2, la)
    st.set_lam(p2, p3, lb)
    st.B[p1[0]][p1[1]] = _rebuild(st, p1, Q1, _pad_cols(U1, n1, D).reshape(k1, 2, D), o1, s1, a1)   # (f)
    st.B[p3[0]][p3[1]] = _rebuild(st, p3, Q3, _pad_cols(V2t.T, n2, D).reshape(k3, 2, D), o3, s3, b3)  # (h)
    t = Tc.transpose(1, 0, 4, 2, 3)                                              # (s2, a', b', o, o')
    order = ["s", a2, b2] + outer2
    t = np.transpose(t, [order.index(g) for g in ["s", "l", "r", "u", "d"]])     # (g)
    t = _scale(t, a2, _inv(la))
    for g in outer2:
        if g in nb2:
            t = _scale(t, g, _inv(st.lam(p2, nb2[g])))
    st.B[p2[0]][p2[1]] = t


def nn_groups(Ly, Lx):
    """The four site-disjoint groups of NN bonds, in Trotter order."""
    return [[((k, m), (k, m + 1)) for k in range(Ly) for m in range(par, Lx - 1, 2)] for par in (0, 1)] + \
           [[((k, m), (k + 1, m)) for k in range(par, Ly - 1, 2) for m in range(Lx)] for par in (0, 1)]


def nnn_groups(Ly, Lx):
    """Site-disjoint groups of NNN updates (p1, corner, p3), in Trotter order."""
    out = []
    for diag in (0, 1):
        for path in (0, 1):
            for pk in (0, 1):
                for pm in (0, 1):
                    grp = []
                    for k in range(pk, Ly - 1, 2):
                        for m in range(pm, Lx - 1, 2):
                            if diag == 0:   # (k,m)-(k+1,m+1) through (k,m+1) or (k+1,m)
                                p1, p3 = (k, m), (k + 1, m + 1)
                                c = (k, m + 1) if path == 0 else (k + 1, m)
                            else:           # (k,m+1)-(k+1,m) through (k,m) or (k+1,m+1)
                                p1, p3 = (k, m + 1), (k + 1, m)
                                c = (k, m) if path == 0 else (k + 1, m + 1)
                            grp.append((p1, c, p3))
                    out.append(grp)
    return out


def trotter_step(st, J1, J2, tau, D):
    g1 = heisenberg_gate(J1, tau)
    for grp in nn_groups(st.Ly, st.Lx):
        for p1, p2 in grp:
            nn_update(st, p1, p2, g1, D)
    if J2 != 0.0:
        g2 = heisenberg_gate(J2, tau / 2)
        for grp in nnn_groups(st.Ly, st.Lx):
            for p1, c, p3 in grp:
                nnn_update(st, p1, c, p3, g2, D)


def lambda_change(old, new):
    """Mean over links of ||lambda_new - lambda_old|| / ||lambda_old||."""
    d = [np.linalg.norm(b - a) / np.linalg.norm(a) for a, b in zip(old.links(), new.links())]
    return float(np.mean(d))


def evolve(st, J1, J2, D, schedule, tol=1e-11):
    """Imaginary-time evolution: for each (tau, max_steps) of ``schedule``, Trotter steps
    until the lambdas change by less than ``tol`` (App. A).  Returns the steps taken."""
    steps = []
    for tau, n in schedule:
        done = 0
        for _ in range(n):
            old = st.copy()
            trotter_step(st, J1, J2, tau, D)
            done += 1
            if lambda_change(old, st) < tol:
                break
        steps.append(done)
    return steps


def to_peps(st):
    """Site tensors A = B with lambda^(1/2) of every link absorbed on both ends (App. A)."""
    out = []
    for k in range(st.Ly):
        row = []
        for m in range(st.Lx):
            t = st.B[k][m]
            for g, q in neighbours(st, (k, m)).items():
                t = _scale(t, g, np.sqrt(st.lam((k, m), q)))
            row.append(t)
        out.append(row)
    return out
