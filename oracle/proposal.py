"""Learned proposal with exact Metropolis-Hastings acceptance -- FP64 oracle.

Test infrastructure only (see the package header).  The paper samples with single
nearest-neighbour swaps (Sec. II A) and names machine learning only as an outlook
(Sec. IV); this component follows the Metropolis-Hastings rule of Eq. (8) -- accept
with min[1, |Psi(S')|^2 q(S|S') / (|Psi(S)|^2 q(S'|S))], which the paper's K_a/K_b
factors instantiate for uniformly chosen pairs -- with a learned q.

Readings of points the paper leaves open:
* Network: three 3x3 convolutions with zero padding on the +-1 spin grid,
  1 -> 32 -> 32 -> 2 channels, ReLU after the first two.  Output channel 0 at (k, m)
  is the logit of the horizontal bond (k,m)-(k,m+1), channel 1 that of the vertical
  bond (k,m)-(k+1,m).
* Move in band k (rows k, k+1; the band is chosen independently of the state): the
  candidates are the antiparallel NN bonds inside the band, in the order: horizontal
  bonds of row k, horizontal bonds of row k+1, vertical bonds, each left to right.
  With probability 1/2 one pair is swapped, else two site-disjoint pairs; pairs are
  drawn one after the other from the softmax of their logits, the second among the
  candidates disjoint from the first.  q of a two-pair move sums both orders.  A
  two-pair draw with no disjoint candidate left proposes nothing.
* Uniforms: Philox (chain, sweep, 4*k + j, "LERN"), j = 0 pair count, 1 first pair,
  2 second pair, 3 acceptance.  A draw picks the first index whose cumulative
  probability exceeds u.
* Training target of a bond: log min(1, rho^2) clipped at -20, rho = Psi(S^b)/Psi(S)
  from the measurement; loss = mean squared error over antiparallel bonds; Adam.
"""
from __future__ import annotations

import numpy as np

from . import philox, vmc

TAG_LEARN = 0x4C45524E  # "LERN"
CHANNELS = 32


def init_params(seed):
    """He-initialised weights (w1 (32,1,3,3), b1, w2 (32,32,3,3), b2, w3 (2,32,3,3), b3)."""
    rng = np.random.default_rng(seed)
    shapes = [(CHANNELS, 1, 3, 3), (CHANNELS, CHANNELS, 3, 3), (2, CHANNELS, 3, 3)]
    p = []
    for s in shapes:
        p.append(rng.standard_normal(s) * np.sqrt(2.0 / (s[1] * 9)))
        p.append(np.zeros(s[0]))
    p[4] *= 0.1
    return p


def params_from_flat(flat):
    """The network's parameter list from one flat array (w1, b1, w2, b2, w3, b3)."""
    shapes = [(CHANNELS, 1, 3, 3), (CHANNELS,), (CHANNELS, CHANNELS, 3, 3), (CHANNELS,), (2, CHANNELS, 3, 3), (2,)]
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.array(flat[off:off + n], dtype=np.float64).reshape(s))
        off += n
    if off != len(flat):
        raise ValueError("wrong number of network parameters")
    return out


def conv3(x, w, b):
    """Zero-padded 3x3 convolution: x (B, Cin, Ly, Lx), w (Cout, Cin, 3, 3)."""
    B, Cin, Ly, Lx = x.shape
    xp = np.zeros((B, Cin, Ly + 2, Lx + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, w.shape[0], Ly, Lx))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,bcyx->boyx", w[:, :, dy, dx], xp[:, :, dy:dy + Ly, dx:dx + Lx])
    return out + b[None, :, None, None]


def forward(params, spins):
    """Logits (B, 2, Ly, Lx) and the cache for backward; spins (B, Ly, Lx) of +-1."""
    w1, b1, w2, b2, w3, b3 = params
    x = np.asarray(spins, dtype=np.float64)[:, None]
    z1 = conv3(x, w1, b1)
    h1 = np.maximum(z1, 0.0)
    z2 = conv3(h1, w2, b2)
    h2 = np.maximum(z2, 0.0)
    out = conv3(h2, w3, b3)
    return out, (x, z1, h1, z2, h2)


def conv3_backward(x, w, dout):
    """Gradients of a zero-padded 3x3 convolution: (dx, dw, db)."""
    B, Cin, Ly, Lx = x.shape
    xp = np.zeros((B, Cin, Ly + 2, Lx + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            dw[:, :, dy, dx] = np.einsum("boyx,bcyx->oc", dout, xp[:, :, dy:dy + Ly, dx:dx + Lx])
            dxp[:, :, dy:dy + Ly, dx:dx + Lx] += np.einsum("oc,boyx->bcyx", w[:, :, dy, dx], dout)
    return dxp[:, :, 1:-1, 1:-1], dw, dout.sum(axis=(0, 2, 3))


def backward(params, cache, dlogits):
    w1, b1, w2, b2, w3, b3 = params
    x, z1, h1, z2, h2 = cache
    dh2, dw3, db3 = conv3_backward(h2, w3, dlogits)
    dz2 = dh2 * (z2 > 0)
    dh1, dw2, db2 = conv3_backward(h1, w2, dz2)
    dz1 = dh1 * (z1 > 0)
    _, dw1, db1 = conv3_backward(x, w1, dz1)
    return [dw1, db1, dw2, db2, dw3, db3]


def bond_targets(spins, ratios_h, ratios_v):
    """Target (B, 2, Ly, Lx) and mask: log min(1, rho^2) clipped at -20 for antiparallel
    bonds; ratios_h[b, k, m] is rho of (k,m)-(k,m+1), ratios_v[b, k, m] of (k,m)-(k+1,m)."""
    s = np.asarray(spins)
    B, Ly, Lx = s.shape
    tgt = np.zeros((B, 2, Ly, Lx))
    mask = np.zeros((B, 2, Ly, Lx))
    anti_h = s[:, :, :-1] != s[:, :, 1:]
    anti_v = s[:, :-1, :] != s[:, 1:, :]
    with np.errstate(divide="ignore"):
        th = np.clip(np.log(np.minimum(1.0, np.asarray(ratios_h) ** 2)), -20.0, 0.0)
        tv = np.clip(np.log(np.minimum(1.0, np.asarray(ratios_v) ** 2)), -20.0, 0.0)
    tgt[:, 0, :, :-1] = np.where(anti_h, th, 0.0)
    mask[:, 0, :, :-1] = anti_h
    tgt[:, 1, :-1, :] = np.where(anti_v, tv, 0.0)
    mask[:, 1, :-1, :] = anti_v
    return tgt, mask


def loss_and_grad(params, spins, tgt, mask):
    out, cache = forward(params, spins)
    n = max(1.0, mask.sum())
    diff = (out - tgt) * mask
    loss = float((diff ** 2).sum() / n)
    return loss, backward(params, cache, 2.0 * diff / n)


def adam_step(params, grads, state, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; state = (m, v) lists."""
    m, v = state
    out = []
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i] = beta1 * m[i] + (1 - beta1) * g
        v[i] = beta2 * v[i] + (1 - beta2) * g * g
        mh = m[i] / (1 - beta1 ** t)
        vh = v[i] / (1 - beta2 ** t)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return out


# -------------------------------------------------------------------- moves and q

def candidates(spins, k):
    """Antiparallel NN bonds of band (k, k+1), as ((k1,m1),(k2,m2), channel, (k,m))."""
    s = np.asarray(spins)
    Ly, Lx = s.shape
    out = []
    for r in (k, k + 1):
        for m in range(Lx - 1):
            if s[r, m] != s[r, m + 1]:
                out.append(((r, m), (r, m + 1), 0, (r, m)))
    for m in range(Lx):
        if s[k, m] != s[k + 1, m]:
            out.append(((k, m), (k + 1, m), 1, (k, m)))
    return out


def _softmax(x):
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(x - x.max())
    return e / e.sum()


def _disjoint(c, b):
    return not ({c[0], c[1]} & {b[0], b[1]})


def move_logprob(logits, spins, k, move):
    """ln q(move | S) for ``move`` = tuple of 1 or 2 bonds (each ((k1,m1),(k2,m2)))."""
    cand = candidates(spins, k)
    lg = np.array([logits[c[2], c[3][0], c[3][1]] for c in cand])
    key = [(c[0], c[1]) for c in cand]
    p1 = _softmax(lg)
    if len(move) == 1:
        return float(np.log(0.5 * p1[key.index(move[0])]))
    total = 0.0
    for first, second in ((move[0], move[1]), (move[1], move[0])):
        i = key.index(first)
        rest = [j for j, c in enumerate(cand) if _disjoint(c, cand[i])]
        p2 = _softmax(lg[rest])
        total += p1[i] * p2[[key[j] for j in rest].index(second)]
    return float(np.log(0.5 * total))


def _draw(p, u):
    return int(min(np.searchsorted(np.cumsum(p), u, side="right"), len(p) - 1))


def propose(logits, spins, k, u0, u1, u2):
    """The move drawn with uniforms u0 (pair count), u1, u2; None if nothing is proposed."""
    cand = candidates(spins, k)
    if not cand:
        return None
    lg = np.array([logits[c[2], c[3][0], c[3][1]] for c in cand])
    i = _draw(_softmax(lg), u1)
    if u0 < 0.5:
        return ((cand[i][0], cand[i][1]),)
    rest = [j for j, c in enumerate(cand) if _disjoint(c, cand[i])]
    if not rest:
        return None
    j = rest[_draw(_softmax(lg[rest]), u2)]
    return ((cand[i][0], cand[i][1]), (cand[j][0], cand[j][1]))


def apply_move(spins, move):
    s = np.array(spins)
    for a, b in move:
        s[a], s[b] = s[b], s[a]
    return s


def band_psi_ratio(grid, spins, new, k, T, B):
    """Psi(S')/Psi(S) for S, S' differing only in rows k, k+1: four-line closures of the
    band between T_k and B_{k+1} (App. C)."""
    def closure(s):
        E = np.ones((1, 1, 1, 1))
        Lx = s.shape[1]
        scale = 0.0
        for m in range(Lx):
            a1 = grid[k][m][vmc.sidx(s[k, m])]
            a2 = grid[k + 1][m][vmc.sidx(s[k + 1, m])]
            E = vmc.env4_left(E, T[m], a1, a2, B[m])
            if m < Lx - 1:
                n = np.linalg.norm(E)
                E = E / n
                scale += np.log(n)
        return float(E.reshape(())), scale
    v1, s1 = closure(new)
    v0, s0 = closure(spins)
    return v1 / v0 * np.exp(s1 - s0)


def learned_band_step(grid, spins, k, T, B, params, seed, chain, sweep, trace=None):
    """One exact MH step with a learned move in band k; returns the new spins."""
    k0, k1 = philox.key_of(seed)
    u = [float(philox.uniform24(philox.philox4x32_10((chain, sweep, 4 * k + j, TAG_LEARN), (k0, k1))[0]))
         for j in range(4)]
    logits = forward(params, np.asarray(spins)[None])[0][0]
    move = propose(logits, spins, k, u[0], u[1], u[2])
    if move is None:
        if trace is not None:
            trace.append((k, None, 0.0, 0.0, False))
        return np.array(spins)
    new = apply_move(spins, move)
    lq_fwd = move_logprob(logits, spins, k, move)
    logits_new = forward(params, new[None])[0][0]
    lq_rev = move_logprob(logits_new, new, k, move)
    rho = band_psi_ratio(grid, spins, new, k, T, B)
    a = min(1.0, rho * rho * np.exp(lq_rev - lq_fwd))
    accept = u[3] < a
    if trace is not None:
        trace.append((k, move, rho, lq_rev - lq_fwd, accept))
    return new if accept else np.array(spins)


def learned_sweep(grid, spins, chi, W, n_fit, params, seed, chain, sweep, trace=None):
    """Bands k = 0 .. Ly-2 in order, each with one learned MH step; T_k is rebuilt after
    the band below it, B_{k+1} comes from the configuration at the start."""
    spins = np.array(spins, dtype=np.int8)
    Ly, Lx = spins.shape
    Bs, _ = vmc.bottom_envs(grid, spins, chi, W, n_fit)
    Ts = [vmc.trivial_mps(Lx)]
    for k in range(Ly - 1):
        spins = learned_band_step(grid, spins, k, Ts[k], Bs[k + 1], params, seed, chain, sweep, trace)
        V, _ = vmc.compress(vmc.mpo_times_mps(Ts[k], vmc.row_tensors(grid, spins, k)), chi, W, n_fit)
        Ts.append(V)
    return spins
