"""Plain FP64 oracle of the per-sample single-layer PEPS contraction inside VMC.

Test infrastructure only (see the package header).  Every function is written from
the paper (Liu, Huang, Gong, Gu, "Accurate simulation for finite projected entangled
pair states in two dimensions", arXiv:1908.09359); numpy einsum / QR are the only
library steps.  Nothing here is blocked, fused or reordered for speed.

Conventions
-----------
* Lattice: Ly rows (k = 0 top) x Lx columns (m = 0 left), open boundaries.
* Site tensor A[k][m] has shape (2, Dl, Dr, Du, Dd) (index order A(s,l,r,u,d) of
  Sec. II A, Eq. (1)); legs on the open edge have dimension 1.
* Spin sigma = +1 uses slot s = 0, sigma = -1 uses slot s = 1.
* Boundary MPS site tensors have shape (left bond, physical, right bond).
* Top environment T_k covers rows < k; its physical legs are the u legs of row k.
  Bottom environment B_k covers rows > k; its physical legs are the d legs of row k.
  (App. B: |U_k> = M_k |U_{k-1}>, <D_k| = <D_{k+1}| M_k.)

Readings of points the paper leaves open:
* Truncation (App. B): the variational fit min ||M|U> - |U'>||^2 by one-site
  sweeps.  Its initial guess is a fixed random MPS (the ``sketch``, an input) brought
  to right-orthonormal form site by site; the first left-to-right sweep is then a
  randomized range finder and later sweeps refine it.  ``n_fit`` (odd) half-sweeps
  are done; the result is left-orthonormal, normalised, its norm kept as a log.
  The second truncation mode, SVD (``n_fit = 0``), is the canonical two-pass
  compression of the exact product (``compress_svd``); the GPU path runs the fit.
* QR: Householder QR with the sign of each column chosen so that diag(R) >= 0.
* Sweep order (Sec. II A): vertical bonds first (columns left to right, bonds top
  to bottom, through the transposed lattice), then horizontal bonds (rows top to
  bottom, bonds left to right).  Only antiparallel pairs are proposed.
* Ratios on the vertical bonds and on the J2 diagonals in E_loc use four-line
  environments of a row pair (App. C works out only the horizontal case).
"""
from __future__ import annotations

import numpy as np

from . import philox

_PATHS = {}


def _einsum(spec, *ops):
    """np.einsum with a pairwise (greedy) contraction order and no cap on the size of
    intermediates; the order of a sum changes nothing but rounding."""
    key = (spec,) + tuple(o.shape for o in ops)
    path = _PATHS.get(key)
    if path is None:
        path = np.einsum_path(spec, *ops, optimize=("greedy", 1e15))[0]
        _PATHS[key] = path
    return np.einsum(spec, *ops, optimize=path)

# ----------------------------------------------------------------------------- lattice


def site_shape(Ly, Lx, D, k, m):
    return (2, 1 if m == 0 else D, 1 if m == Lx - 1 else D, 1 if k == 0 else D,
            1 if k == Ly - 1 else D)


def unpack(flat, Ly, Lx, D):
    """Flat site-major array -> grid[k][m] of (2, Dl, Dr, Du, Dd) arrays (copies)."""
    grid, off = [], 0
    for k in range(Ly):
        row = []
        for m in range(Lx):
            shp = site_shape(Ly, Lx, D, k, m)
            n = int(np.prod(shp))
            row.append(np.array(flat[off:off + n], dtype=np.float64).reshape(shp))
            off += n
        grid.append(row)
    if off != len(flat):
        raise ValueError("tensor array has the wrong length")
    return grid


def pack(grid):
    return np.concatenate([t.ravel() for row in grid for t in row])


def sidx(sigma):
    return 0 if sigma > 0 else 1


def transpose_lattice(grid):
    """Columns become rows: A'(s, l'=u, r'=d, u'=l, d'=r) at (m, k)."""
    Ly, Lx = len(grid), len(grid[0])
    return [[grid[k][m].transpose(0, 3, 4, 1, 2) for k in range(Ly)] for m in range(Lx)]


def vflip_lattice(grid):
    """Upside down: row k -> Ly-1-k, legs u and d swapped."""
    return [[t.transpose(0, 1, 2, 4, 3) for t in row] for row in grid[::-1]]


# ------------------------------------------------------------------ boundary-MPS (App. B)


def qr_pos(M):
    """Householder QR with diag(R) >= 0 (makes Q unique for full-rank M)."""
    Q, R = np.linalg.qr(M, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn, R * sgn[:, None]


def bond_caps(chiX, phys, chi):
    """Bond dimensions of the truncated MPS: min(chi, target bond), reduced so that no
    bond exceeds what the physical legs on either side can carry."""
    L = len(phys)
    r = [min(chi, chiX[i]) for i in range(L - 1)]
    prev = 1
    for i in range(L - 1):
        r[i] = min(r[i], prev * phys[i])
        prev = r[i]
    nxt = 1
    for i in range(L - 2, -1, -1):
        r[i] = min(r[i], nxt * phys[i + 1])
        nxt = r[i]
    return r


def sketch_mps(W, r, phys):
    """Initial guess of the fit: sketch site m sliced to (r[m-1], p_m, r[m]) and made
    right-orthonormal on its own (rows of the (r[m-1], p_m r[m]) matrix orthonormal)."""
    L = len(phys)
    b = [1] + list(r) + [1]
    V = []
    for m in range(L):
        w = np.array(W[m][:b[m], :phys[m], :b[m + 1]], dtype=np.float64)
        if m == 0:
            V.append(w)
            continue
        Q, _ = qr_pos(w.reshape(b[m], phys[m] * b[m + 1]).T)
        V.append(Q.T.reshape(b[m], phys[m], b[m + 1]))
    return V


def mpo_times_mps(T, row):
    """|X> = M_k |T_k>: X_m[(a,l), d, (a',r)] = sum_u T_m[a,u,a'] a_m[l,r,u,d] (App. B)."""
    X = []
    for Tm, a in zip(T, row):
        cl, _, cr = Tm.shape
        Dl, Dr, _, Dd = a.shape
        X.append(np.einsum("aub,lrud->aldbr", Tm, a).reshape(cl * Dl, Dd, cr * Dr))
    return X


def compress_svd(X, chi):
    """Truncation by SVD (canonical two-pass compression): X is brought to left-orthonormal
    form by QR (diag(R) >= 0), then, from the right, each site's (left bond, spin x right
    bond) matrix is truncated by an SVD to the bond caps; the result is brought back to
    left-orthonormal form and normalised.  Returns (V, log ||V||) like ``compress``."""
    L = len(X)
    phys = [x.shape[1] for x in X]
    r = bond_caps([X[m].shape[2] for m in range(L - 1)], phys, chi)
    Y = [np.array(x, dtype=np.float64) for x in X]
    logn = 0.0
    for sweep in range(2):
        if sweep == 1:
            for m in range(L - 1, 0, -1):   # right to left: truncated SVDs
                b0, p, b1 = Y[m].shape
                U, S, Vt = np.linalg.svd(Y[m].reshape(b0, p * b1), full_matrices=False)
                k = min(r[m - 1], len(S))
                Y[m] = Vt[:k].reshape(k, p, b1)
                Y[m - 1] = np.einsum("apb,bk->apk", Y[m - 1], U[:, :k] * S[:k])
        for m in range(L - 1):              # left to right: QR
            b0, p, b1 = Y[m].shape
            Q, R = qr_pos(Y[m].reshape(b0 * p, b1))
            Y[m] = Q.reshape(b0, p, Q.shape[1])
            Y[m + 1] = np.einsum("ab,bpc->apc", R, Y[m + 1])
        nrm = np.linalg.norm(Y[L - 1])
        Y[L - 1] = Y[L - 1] / nrm
        logn += float(np.log(nrm))
    return Y, logn


def compress(X, chi, W, n_fit):
    """Variational fit of App. B: minimise ||X - V||^2 over MPS V of bond <= chi.

    Returns (V, log ||V_fit||) with V normalised and left-orthonormal (centre at the
    last site).  ``n_fit`` is the number of one-site half-sweeps (odd); ``n_fit = 0``
    selects the SVD truncation of ``compress_svd`` instead of the fit.
    """
    if n_fit == 0:
        return compress_svd(X, chi)
    if n_fit < 1 or n_fit % 2 == 0:
        raise ValueError("n_fit must be odd")
    L = len(X)
    phys = [x.shape[1] for x in X]
    r = bond_caps([X[m].shape[2] for m in range(L - 1)], phys, chi)
    V = sketch_mps(W, r, phys)
    R = [None] * (L + 1)
    R[L] = np.ones((1, 1))
    for m in range(L - 1, 0, -1):  # R[m]: (X bond left of m, V bond left of m)
        R[m] = _einsum("xpy,bpc,yc->xb", X[m], V[m], R[m + 1])
    Le = [None] * (L + 1)
    Le[0] = np.ones((1, 1))
    for sweep in range(n_fit):
        order = range(L) if sweep % 2 == 0 else range(L - 1, -1, -1)
        for m in order:
            Y = _einsum("xb,xpy,yc->bpc", Le[m], X[m], R[m + 1])  # optimal site m
            b0, p, b1 = Y.shape
            if sweep % 2 == 0 and m < L - 1:
                Q, _ = qr_pos(Y.reshape(b0 * p, b1))
                V[m] = Q.reshape(b0, p, b1)
                Le[m + 1] = _einsum("xb,xpy,bpc->yc", Le[m], X[m], V[m])
            elif sweep % 2 == 1 and m > 0:
                Q, _ = qr_pos(Y.reshape(b0, p * b1).T)
                V[m] = Q.T.reshape(b0, p, b1)
                R[m] = _einsum("xpy,bpc,yc->xb", X[m], V[m], R[m + 1])
            else:
                V[m] = Y
    nrm = np.linalg.norm(V[L - 1])
    V[L - 1] = V[L - 1] / nrm
    return V, float(np.log(nrm))


def trivial_mps(L):
    return [np.ones((1, 1, 1)) for _ in range(L)]


def row_tensors(grid, spins, k):
    return [grid[k][m][sidx(spins[k][m])] for m in range(len(grid[k]))]


def top_envs(grid, spins, chi, W, n_fit, upto=None):
    """T_0 .. T_{upto} (default all Ly) and their log norms, rows fixed."""
    Ly, Lx = len(grid), len(grid[0])
    upto = Ly - 1 if upto is None else upto
    Ts, logs = [trivial_mps(Lx)], [0.0]
    for k in range(upto):
        V, ln = compress(mpo_times_mps(Ts[-1], row_tensors(grid, spins, k)), chi, W, n_fit)
        Ts.append(V)
        logs.append(logs[-1] + ln)
    return Ts, logs


def bottom_envs(grid, spins, chi, W, n_fit):
    """B_0 .. B_{Ly-1} via the top-down pass on the upside-down lattice."""
    Ly = len(grid)
    Tf, lf = top_envs(vflip_lattice(grid), np.asarray(spins)[::-1], chi, W, n_fit)
    return [Tf[Ly - 1 - k] for k in range(Ly)], [lf[Ly - 1 - k] for k in range(Ly)]


# ------------------------------------------------------- three-line environments (App. C)


def env3_left(E, T, a, B):
    """L(m) from L(m-1): columns of (T_k, row k, B_k) absorbed from the left."""
    return _einsum("xlb,xua,lrud,bdc->arc", E, T, a, B)


def env3_right(E, T, a, B):
    """R(m) from R(m+1)."""
    return _einsum("arc,xua,lrud,bdc->xlb", E, T, a, B)


def env4_left(E, T, a1, a2, B):
    """Four-line left environment of rows (k, k+1): E[a, l1, l2, b]."""
    return _einsum("xpqb,xua,prud,qsde,bec->arsc", E, T, a1, a2, B)


def env4_right(E, T, a1, a2, B):
    return _einsum("arsc,xua,prud,qsde,bec->xpqb", E, T, a1, a2, B)


def _normalised(E):
    n = np.linalg.norm(E)
    return E / n, n


def row_psi(T, row, B, logT, logB):
    """(log|Psi|, sign) of <B_k| M_k |T_k> contracted column by column."""
    E, ln = np.ones((1, 1, 1)), logT + logB
    for m in range(len(row)):
        E = env3_left(E, T[m], row[m], B[m])
        if m < len(row) - 1:
            E, n = _normalised(E)
            ln += np.log(n)
    v = float(E.reshape(()))
    return ln + np.log(abs(v)), float(np.sign(v))


# ------------------------------------------------------------- sequential sweep (Sec. II A)


def _row_phase(grid, spins, chi, W, n_fit, seed, chain, sweep, bond_base, trace):
    """Visit the horizontal bonds of every row of ``grid`` (rows top to bottom, bonds
    left to right) with the Metropolis rule P_s = min[1, |Psi(S_b)|^2/|Psi(S_a)|^2]
    (Eq. (9)).  Row k uses the fixed environments T_k (rebuilt after each row) and
    B_k (from the configuration at the start of the phase).  Mutates ``spins``.
    Returns the top environments T_0..T_{Ly-1} of the final configuration."""
    Ly, Lx = spins.shape
    Bs, _ = bottom_envs(grid, spins, chi, W, n_fit)
    Ts, logT = [trivial_mps(Lx)], [0.0]
    for k in range(Ly):
        T, B = Ts[k], Bs[k]
        _sample_row(grid, spins, k, T, B, seed, chain, sweep, bond_base, trace)
        if k < Ly - 1:
            V, ln = compress(mpo_times_mps(T, row_tensors(grid, spins, k)), chi, W, n_fit)
            Ts.append(V)
            logT.append(logT[-1] + ln)
    return Ts, logT


def _sample_row(grid, spins, k, T, B, seed, chain, sweep, bond_base, trace):
    """Metropolis visits of the horizontal bonds of row k, left to right, with the
    fixed environments T_k, B_k; the left three-line environment follows the
    accepted configuration (App. C, Fig. "contraction")."""
    Lx = spins.shape[1]
    a = grid[k]
    R = [None] * (Lx + 1)
    Rf = [None] * (Lx + 1)
    R[Lx] = np.ones((1, 1, 1))
    for m in range(Lx - 1, 0, -1):
        s = sidx(spins[k, m])
        raw = env3_right(R[m + 1], T[m], a[m][s], B[m])
        nrm = np.linalg.norm(raw)
        R[m] = raw / nrm
        Rf[m] = env3_right(R[m + 1], T[m], a[m][1 - s], B[m]) / nrm
    E = np.ones((1, 1, 1))
    for m in range(Lx - 1):
        s = sidx(spins[k, m])
        cur = env3_left(E, T[m], a[m][s], B[m])
        if spins[k, m] != spins[k, m + 1]:
            flip = env3_left(E, T[m], a[m][1 - s], B[m])
            rho = float(np.vdot(flip, Rf[m + 1]) / np.vdot(cur, R[m + 1]))
            bond = bond_base + k * (Lx - 1) + m
            u = philox.metropolis_uniform(seed, chain, sweep, bond)
            accept = u < min(1.0, rho * rho)
            if trace is not None:
                accept = trace.decide(bond, rho, u, accept)
            if accept:
                spins[k, m] = -spins[k, m]
                spins[k, m + 1] = -spins[k, m + 1]
                cur = flip
        E, _ = _normalised(cur)


class Trace:
    """Records every proposal (bond, ratio, uniform, decision).  With ``follow`` set to
    a dict bond -> decision, near-ties (|ln r - ln rho^2| < tie) take that decision."""

    def __init__(self, follow=None, tie=1e-5):
        self.rows, self.follow, self.tie = [], follow, tie

    def decide(self, bond, rho, u, accept):
        if self.follow is not None and bond in self.follow and rho != 0.0:
            if abs(np.log(u if u > 0 else 1e-300) - np.log(rho * rho)) < self.tie:
                accept = bool(self.follow[bond])
        self.rows.append((bond, rho, u, bool(accept)))
        return accept


def sweep(grid, spins, chi, W, n_fit, seed, chain, sweep_index, trace=None):
    """One sequential MC sweep (all vertical then all horizontal bonds once).

    Bond ids: vertical bond (k,m)-(k+1,m) is m*(Ly-1)+k; horizontal bond (k,m)-(k,m+1)
    is Lx*(Ly-1) + k*(Lx-1) + m.  Returns (new spins, T_k, log T_k) where the top
    environments are those of the final configuration.
    """
    spins = np.array(spins, dtype=np.int8)
    Ly, Lx = spins.shape
    st = np.ascontiguousarray(spins.T)
    _row_phase(transpose_lattice(grid), st, chi, W, n_fit, seed, chain, sweep_index, 0, trace)
    spins = np.ascontiguousarray(st.T)
    Ts, logT = _row_phase(grid, spins, chi, W, n_fit, seed, chain, sweep_index,
                          Lx * (Ly - 1), trace)
    return spins, Ts, logT


# --------------------------------------------------------- measurement (Eqs. (3)-(7), App. C)


def measure(grid, spins, chi, W, n_fit, J1, J2, Ts=None, logT=None, want_grad=True):
    """E_loc(S), log|Psi(S)|, sign Psi(S) and G(S) = Delta(S)/Psi(S) for one configuration.

    E_loc (App. C, Eq. (C1)) of H = J1 sum_NN S_i.S_j + J2 sum_NNN S_i.S_j with S = sigma/2:
    each bond gives J sigma_i sigma_j / 4 and, if antiparallel, J/2 Psi(S')/Psi(S).
    Horizontal ratios and G of row k use (T_k, row k, B_k); vertical and diagonal ratios
    of rows (k, k+1) use four-line environments between T_k and B_{k+1}.  log|Psi| and
    the sign are those of row Ly//2.  G is a list of (Dl, Dr, Du, Dd) arrays for the
    slot s(k, m) of every site.
    """
    spins = np.asarray(spins)
    Ly, Lx = spins.shape
    if Ts is None:
        Ts, logT = top_envs(grid, spins, chi, W, n_fit)
    Bs, logB = bottom_envs(grid, spins, chi, W, n_fit)
    e = 0.0
    scale = [0.0]   # sum of |terms| of E_loc (tolerance scale for comparisons)
    G = [[None] * Lx for _ in range(Ly)]
    logpsi = sign = None
    for k in range(Ly):
        if k == Ly // 2:
            logpsi, sign = row_psi(Ts[k], row_tensors(grid, spins, k), Bs[k], logT[k], logB[k])
        e += _row_terms(grid, spins, k, Ts[k], Bs[k], J1, G if want_grad else None, scale)
    for k in range(Ly - 1):
        e += _pair_terms(grid, spins, k, Ts[k], Bs[k + 1], J1, J2, scale)
    return dict(eloc=e, logpsi=logpsi, sign=sign, G=G if want_grad else None, eloc_scale=scale[0])


def _row_terms(grid, spins, k, T, B, J1, G, scale):
    """Horizontal NN terms of row k from its three-line environments (App. C, Fig.
    "contraction"); fills G[k][m] = Delta/Psi when G is given."""
    Lx = spins.shape[1]
    R = [None] * (Lx + 1)
    Rf = [None] * (Lx + 1)
    R[Lx] = np.ones((1, 1, 1))
    for m in range(Lx - 1, 0, -1):
        s = sidx(spins[k, m])
        raw = env3_right(R[m + 1], T[m], grid[k][m][s], B[m])
        nrm = np.linalg.norm(raw)
        R[m] = raw / nrm
        Rf[m] = env3_right(R[m + 1], T[m], grid[k][m][1 - s], B[m]) / nrm
    e = 0.0
    E = np.ones((1, 1, 1))
    for m in range(Lx):
        s = sidx(spins[k, m])
        cur = env3_left(E, T[m], grid[k][m][s], B[m])
        if G is not None:
            psi_km = np.vdot(cur, R[m + 1])   # Tr[L0(m) R0(m+1)], same scale as Delta
            delta = _einsum("xlb,xua,bdc,arc->lrud", E, T[m], B[m], R[m + 1])
            G[k][m] = delta / psi_km
        if m < Lx - 1:
            sg = spins[k, m] * spins[k, m + 1]
            e += J1 * sg / 4.0
            scale[0] += abs(J1) / 4.0
            if sg < 0:
                flip = env3_left(E, T[m], grid[k][m][1 - s], B[m])
                t = 0.5 * J1 * float(np.vdot(flip, Rf[m + 1]) / np.vdot(cur, R[m + 1]))
                e += t
                scale[0] += abs(t)
        E, _ = _normalised(cur)
    return e


def _col(grid, spins, k, m, flip_top=False, flip_bot=False):
    s1, s2 = sidx(spins[k, m]), sidx(spins[k + 1, m])
    return grid[k][m][1 - s1 if flip_top else s1], grid[k + 1][m][1 - s2 if flip_bot else s2]


def _pair_terms(grid, spins, k, T, B, J1, J2, scale):
    """Vertical NN terms (k,m)-(k+1,m) and both NNN diagonals of rows (k, k+1)."""
    Lx = spins.shape[1]
    R4 = [None] * (Lx + 1)
    R4[Lx] = np.ones((1, 1, 1, 1))
    for m in range(Lx - 1, -1, -1):
        a1, a2 = _col(grid, spins, k, m)
        R4[m], _ = _normalised(env4_right(R4[m + 1], T[m], a1, a2, B[m]))
    e = 0.0
    E = np.ones((1, 1, 1, 1))
    for m in range(Lx):
        cur = env4_left(E, T[m], *_col(grid, spins, k, m), B[m])
        den1 = np.vdot(cur, R4[m + 1])
        sg = spins[k, m] * spins[k + 1, m]
        e += J1 * sg / 4.0
        scale[0] += abs(J1) / 4.0
        if sg < 0:
            fl = env4_left(E, T[m], *_col(grid, spins, k, m, True, True), B[m])
            t = 0.5 * J1 * float(np.vdot(fl, R4[m + 1]) / den1)
            e += t
            scale[0] += abs(t)
        if J2 != 0.0 and m < Lx - 1:
            nxt = env4_left(cur, T[m + 1], *_col(grid, spins, k, m + 1), B[m + 1])
            den2 = np.vdot(nxt, R4[m + 2])
            # diagonal (k,m)-(k+1,m+1)
            sg = spins[k, m] * spins[k + 1, m + 1]
            e += J2 * sg / 4.0
            scale[0] += abs(J2) / 4.0
            if sg < 0:
                f = env4_left(E, T[m], *_col(grid, spins, k, m, True, False), B[m])
                f = env4_left(f, T[m + 1], *_col(grid, spins, k, m + 1, False, True), B[m + 1])
                t = 0.5 * J2 * float(np.vdot(f, R4[m + 2]) / den2)
                e += t
                scale[0] += abs(t)
            # anti-diagonal (k,m+1)-(k+1,m)
            sg = spins[k, m + 1] * spins[k + 1, m]
            e += J2 * sg / 4.0
            scale[0] += abs(J2) / 4.0
            if sg < 0:
                f = env4_left(E, T[m], *_col(grid, spins, k, m, False, True), B[m])
                f = env4_left(f, T[m + 1], *_col(grid, spins, k, m + 1, True, False), B[m + 1])
                t = 0.5 * J2 * float(np.vdot(f, R4[m + 2]) / den2)
                e += t
                scale[0] += abs(t)
        E, _ = _normalised(cur)
    return e


# ------------------------------------------------------ gradient and update (Alg. 1, Eq. (10))


class Accumulator:
    """Monte Carlo sums of Algorithm 1: E_tot, P1 = sum G E_loc, P2 = sum G (per slot)."""

    def __init__(self, grid):
        self.n = 0
        self.sE = 0.0
        self.sE2 = 0.0
        self.P1 = [[np.zeros_like(t) for t in row] for row in grid]
        self.P2 = [[np.zeros_like(t) for t in row] for row in grid]

    def add(self, spins, eloc, G):
        self.n += 1
        self.sE += eloc
        self.sE2 += eloc * eloc
        for k, row in enumerate(G):
            for m, g in enumerate(row):
                s = sidx(spins[k][m])
                self.P1[k][m][s] += g * eloc
                self.P2[k][m][s] += g

    def gradient(self):
        """dE/dA = <G E_loc> - <G><E_loc> (Sec. II A, Eq. (5); no factor 2)."""
        E = self.sE / self.n
        return [[p1 / self.n - (p2 / self.n) * E for p1, p2 in zip(r1, r2)]
                for r1, r2 in zip(self.P1, self.P2)], E


def sign_sgd(flat, grad_flat, delta, seed, step):
    """A <- A - r delta sgn(dE/dA), r ~ U[0,1) per element (Sec. II B, Eq. (10))."""
    r = philox.update_uniforms(seed, step, len(flat))
    return np.asarray(flat, dtype=np.float64) - r * delta * np.sign(grad_flat)
