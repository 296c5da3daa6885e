"""Derivation of the float32 parity bounds of the GPU tests (run by hand, CPU only).

    python tests/float32_spread.py

The boundary-MPS fit (App. B) does a QR per site and half-sweep; at truncated Dc its
result depends on rounding order.  This script re-runs the oracle's arithmetic in
float32 -- every einsum in float32 and the fit's QR as plain float32 Householder, the
GPU's algorithm, with three summation orders of the reflector dot products (NumPy's
dot, sequential, reversed) -- and reports, against the float64 oracle, the worst
and median relative deviation of the sweep ratios (the cases of test_sweep_parity_*) and the
norm-wise deviation of G (the iid case of test_measure_parity).  The GPU tests bound
their float32 results by about twice the largest of these.  Nothing here is imported by
the tests; it only documents where their bounds come from.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))

from oracle import vmc  # noqa: E402
from paper_1908_09359_gb300 import inputs  # noqa: E402
import make_sampled_configs as golden  # noqa: E402

F32 = np.float32


def householder32(M, order):
    """Thin Q with diag(R) >= 0 in float32, reflector dot products summed in `order`."""
    A = np.array(M, dtype=F32)
    rows, cols = A.shape

    def dot(x, y):
        if order == "dot":
            return F32(np.dot(x, y))
        s = F32(0)
        for a, b in (zip(x, y) if order == "seq" else zip(x[::-1], y[::-1])):
            s = F32(s + a * b)
        return s

    beta, flip = [], []
    for j in range(cols):
        x = A[j:, j]
        alpha = F32(np.sqrt(dot(x, x)))
        x0 = A[j, j]
        if alpha == 0:
            beta.append(F32(0))
            flip.append(False)
            continue
        sg = F32(1) if x0 >= 0 else F32(-1)
        A[j, j] = F32(x0 + sg * alpha)
        beta.append(F32(1) / F32(alpha * (alpha + abs(x0))))
        flip.append(sg > 0)
        v = A[j:, j]
        for k in range(j + 1, cols):
            A[j:, k] = (A[j:, k] - F32(dot(v, A[j:, k]) * beta[j]) * v).astype(F32)
    Q = np.zeros((rows, cols), dtype=F32)
    Q[:cols, :cols] = np.eye(cols, dtype=F32)
    for j in range(cols - 1, -1, -1):
        if beta[j] == 0:
            continue
        v = A[j:, j]
        for k in range(j, cols):
            Q[j:, k] = (Q[j:, k] - F32(dot(v, Q[j:, k]) * beta[j]) * v).astype(F32)
    Q[:, flip] *= -1
    return Q, None


class Float32Oracle:
    """Context manager: the oracle's einsums and QR in float32."""

    def __init__(self, order):
        self.order = order

    def __enter__(self):
        self.saved = (vmc._einsum, vmc.qr_pos, vmc.np.einsum)
        e, npe = self.saved[0], self.saved[2]
        vmc._einsum = lambda spec, *ops: e(spec, *[np.asarray(o, F32) for o in ops]).astype(F32)
        vmc.np.einsum = lambda spec, *ops, **kw: npe(spec, *[np.asarray(o, F32) for o in ops], **kw).astype(F32)
        vmc.qr_pos = lambda M: householder32(M, self.order)
        return self

    def __exit__(self, *a):
        vmc._einsum, vmc.qr_pos, vmc.np.einsum = self.saved


def sweep_spread(w, start, seed, t, chains):
    g = vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])
    ref = {}
    for c in chains:
        tr = vmc.Trace()
        vmc.sweep(g, start[c], w["chi"], w["sketch"], 3, seed, c, t, trace=tr)
        ref[c] = tr.rows
    g32 = [[x.astype(F32) for x in row] for row in g]
    out = {}
    for order in ("dot", "seq", "rev"):
        dev = []
        with Float32Oracle(order):
            for c in chains:
                tr = vmc.Trace(follow={b: int(a) for b, _, _, a in ref[c]}, tie=1e-5)
                vmc.sweep(g32, start[c], w["chi"], w["sketch"].astype(F32), 3, seed, c, t, trace=tr)
                r64 = {b: rho for b, rho, _, _ in ref[c]}
                dev += [abs(rho - r64[b]) / max(abs(r64[b]), 1.0) for b, rho, _, _ in tr.rows]
        out[order] = {"max": float(np.max(dev)), "median": float(np.median(dev))}
    return out


def grad_spread(w, configs):
    g = vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])
    flat = lambda G: np.concatenate([x.ravel() for row in G for x in row])  # noqa: E731
    ref = [flat(vmc.measure(g, s, w["chi"], w["sketch"], 3, w["J1"], w["J2"])["G"]) for s in configs]
    g32 = [[x.astype(F32) for x in row] for row in g]
    out = {}
    for order in ("dot", "seq", "rev"):
        with Float32Oracle(order):
            errs = [np.linalg.norm(flat(vmc.measure(g32, s, w["chi"], w["sketch"].astype(F32), 3, w["J1"],
                                                    w["J2"])["G"]).astype(np.float64) - r) / np.linalg.norm(r)
                    for s, r in zip(configs, ref)]
        out[order] = max(errs)
    return out


def main():
    w = inputs.workload("peps_8x8", n_chains=6)
    w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
    print("sweep ratios, bond-decay 8x8:", sweep_spread(w, inputs.start_spins(6, 8, 8, 33, "random"), 77, 3,
                                                        range(6)), flush=True)
    w = inputs.workload("peps_8x8", n_chains=8)
    sampled = golden.load("peps_8x8")
    print("sweep ratios, iid 8x8 sampled:", sweep_spread(w, sampled, 77, 12, (0, 3, 5, 7)), flush=True)
    print("G, iid 8x8 sampled:", grad_spread(w, sampled), flush=True)


if __name__ == "__main__":
    main()
