"""Write tests/golden/float32_spread.json: the float32 spread of the oracle's own results,
from which the float32 parity bounds of the GPU tests are derived (CPU only, oracle only);
and the same for split-BF16 arithmetic, from which the bounds of the tensor-core form are
derived.

    python tests/golden/make_float32_spread.py

The boundary-MPS fit (App. B) does a QR per site and half-sweep; at truncated Dc its
result depends on rounding order.  This script re-runs the oracle's arithmetic in float32
-- every einsum in float32 and the fit's QR as plain float32 Householder (the GPU's
algorithm) -- in six rounding orders: three summation orders of the reflector dot products
(NumPy's dot, sequential, reversed) times two contraction orders of every einsum (the
oracle's pairwise order, and the pairwise order found for the operands listed in reverse).
The GPU differs from the oracle in both kinds of order.  Against the float64 oracle it
records, per order, the worst and median relative deviation of the sweep ratios (relative
to max(|rho|, 1)) and the norm-wise deviation of G, for the cases of tests/test_gpu_parity.py:
bond-decay 8x8 sweeps and the oracle-sampled iid 8x8 configurations.  The GPU tests bound
their float32 results by twice the largest value over the orders.

Split BF16 (tests/test_gpu_mixed.py, tests/test_gpu_parity_24x24.py): every pairwise
product of every einsum splits both operands into BF16 hi + lo and forms hi.hi + hi.lo +
lo.hi (the lo.lo product dropped, as the tensor-core form drops it) with float32
accumulation, the QR stays float32 Householder, in the same six rounding orders; recorded are
the worst sweep-ratio deviation, E_loc relative to its term scale, ln|Psi|, and G
norm-wise and element-wise, over the orders and the cases' chains (8x8: six chains, one
sweep and a measurement each; 24x24: the chains tests/test_gpu_parity_24x24.py checks in
the 512-chain launch -- the first column of the sweep of chains 0 and 341 and the
measurement of the start configurations of chains 85 and 426).  A ratio
whose contraction nearly cancels can move by ~1e-3 with the QR's summation order alone,
which is why one order is not enough.  ``--split-only`` recomputes only these figures,
``--split24-only`` only the 24x24 ones.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

from oracle import vmc  # noqa: E402
from paper_1908_09359_gb300 import inputs  # noqa: E402
import make_sampled_configs as golden  # noqa: E402

F32 = np.float32
ORDERS = [(dots, path) for path in ("oracle", "reversed") for dots in ("dot", "seq", "rev")]
# chains of the 512-chain 24x24 launch whose first-column sweep and start-configuration
# measurement tests/test_gpu_parity_24x24.py compares with the float64 oracle
SWEEP_CHAINS_24 = (0, 341)
MEASURE_CHAINS_24 = (85, 426)


def householder32(M, order):
    """Thin Q with diag(R) >= 0 in float32, reflector dot products summed in `order`."""
    A = np.array(M, dtype=F32)
    rows, cols = A.shape

    def dot(x, y):
        if order == "dot":
            return F32(np.dot(x, y))
        # sequential float32 sums of the float32 products (np.cumsum accumulates in order)
        p = np.multiply(x, y, dtype=F32)
        return np.cumsum(p if order == "seq" else p[::-1], dtype=F32)[-1] if len(p) else F32(0)

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


def reversed_einsum(spec, *ops):
    """The same contraction with the operands listed in reverse: another pairwise order."""
    ins, out = spec.split("->")
    terms = ins.split(",")
    rspec = ",".join(terms[::-1]) + "->" + out
    rops = ops[::-1]
    path = np.einsum_path(rspec, *rops, optimize=("greedy", 1e15))[0]
    return np.einsum(rspec, *rops, optimize=path)


class Float32Oracle:
    """Context manager: the oracle's einsums and QR in float32, in one rounding order."""

    def __init__(self, order):
        self.dots, self.path = order

    def __enter__(self):
        self.saved = (vmc._einsum, vmc.qr_pos, vmc.np.einsum)
        e, npe = self.saved[0], self.saved[2]
        base = e if self.path == "oracle" else reversed_einsum
        vmc._einsum = lambda spec, *ops: base(spec, *[np.asarray(o, F32) for o in ops]).astype(F32)
        vmc.np.einsum = lambda spec, *ops, **kw: npe(spec, *[np.asarray(o, F32) for o in ops], **kw).astype(F32)
        vmc.qr_pos = lambda M: householder32(M, self.dots)
        return self

    def __exit__(self, *a):
        vmc._einsum, vmc.qr_pos, vmc.np.einsum = self.saved


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), kept as float32."""
    u = np.ascontiguousarray(x, dtype=F32).view(np.uint32)
    r = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return r.view(F32)


def split_round(x):
    """x as the tensor cores see it in split BF16: hi + lo, both BF16."""
    x = np.asarray(x, dtype=F32)
    hi = bf16(x)
    return hi + bf16(x - hi)


def split_product(spec, a, b):
    """One pairwise product as the tensor cores form it in split BF16: both operands split
    into BF16 hi + lo, the three products hi.hi + hi.lo + lo.hi (lo.lo dropped) each exact
    in float32 and accumulated in float32."""
    a, b = np.asarray(a, F32), np.asarray(b, F32)
    ah, bh = bf16(a), bf16(b)
    al, bl = bf16(a - ah), bf16(b - bh)
    return (np.einsum(spec, ah, bh + bl) + np.einsum(spec, al, bh)).astype(F32)


def split_einsum(spec, *ops):
    """The einsum as pairwise products in the oracle's greedy order, each product formed
    as split_product forms it."""
    ins, out = spec.split("->")
    terms = ins.split(",")
    ops = [np.asarray(o, F32) for o in ops]
    if len(ops) == 1:
        return np.einsum(spec, split_round(ops[0])).astype(F32)
    path = np.einsum_path(spec, *ops, optimize=("greedy", 1e15))[0][1:]
    for i, j in path:
        a, b = terms[i], terms[j]
        rest = [t for n, t in enumerate(terms) if n not in (i, j)]
        keep = set(out).union(*[set(t) for t in rest]) if rest else set(out)
        res = "".join(dict.fromkeys(c for c in a + b if c in keep))
        if not rest:
            res = out
        prod = split_product(f"{a},{b}->{res}", ops[i], ops[j])
        ops = [o for n, o in enumerate(ops) if n not in (i, j)] + [prod]
        terms = rest + [res]
    return np.einsum(f"{terms[0]}->{out}", ops[0]).astype(F32)


class SplitOracle:
    """Context manager: the oracle's einsums in emulated split BF16, the QR in float32,
    in one of the six rounding orders (QR dot-product order x contraction order)."""

    def __init__(self, order=("dot", "oracle")):
        self.dots, self.path = order

    def __enter__(self):
        self.saved = (vmc._einsum, vmc.qr_pos, vmc.np.einsum)
        npe = self.saved[2]
        if self.path == "oracle":
            vmc._einsum = split_einsum
        else:
            def rev(spec, *ops):
                ins, out = spec.split("->")
                return split_einsum(",".join(ins.split(",")[::-1]) + "->" + out, *ops[::-1])
            vmc._einsum = rev
        vmc.np.einsum = lambda spec, *ops, **kw: npe(spec, *[np.asarray(o, F32) for o in ops], **kw).astype(F32)
        vmc.qr_pos = lambda M: householder32(M, self.dots)
        return self

    def __exit__(self, *a):
        vmc._einsum, vmc.qr_pos, vmc.np.einsum = self.saved


def split_spread(w, start, seed, t, chains, first_column_only=False, order=("dot", "oracle"),
                 measure_chains=None):
    """Sweep-ratio and measurement deviations of emulated split BF16 from float64, in one
    rounding order: the sweep (or its first column) of every chain in ``chains`` and the
    measurement of ``start[c]`` for every c in ``measure_chains`` (default: ``chains``)."""
    g = vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])
    g32 = [[x.astype(F32) for x in row] for row in g]
    W, W32 = w["sketch"], w["sketch"].astype(F32)
    flat = lambda G: np.concatenate([x.ravel() for row in G for x in row])  # noqa: E731

    def first_column(grid, spins, sk, trace):
        gT = vmc.transpose_lattice(grid)
        st = np.ascontiguousarray(np.asarray(spins).T).astype(np.int8)
        Bs, _ = vmc.bottom_envs(gT, st, w["chi"], sk, 3)
        vmc._sample_row(gT, st, 0, vmc.trivial_mps(w["Ly"]), Bs[0], seed, c, t, 0, trace)

    ratio_dev, out = [], {}
    eloc_dev, lp_dev, g_nrm, g_el = [], [], [], []
    for c in chains:
        ref = vmc.Trace()
        if first_column_only:
            first_column(g, start[c], W, ref)
        else:
            vmc.sweep(g, start[c], w["chi"], W, 3, seed, c, t, trace=ref)
        with SplitOracle(order):
            tr = vmc.Trace(follow={b: int(a) for b, _, _, a in ref.rows}, tie=1e-5)
            if first_column_only:
                first_column(g32, start[c], W32, tr)
            else:
                vmc.sweep(g32, start[c], w["chi"], W32, 3, seed, c, t, trace=tr)
        r64 = {b: rho for b, rho, _, _ in ref.rows}
        ratio_dev += [abs(rho - r64[b]) / max(abs(r64[b]), 1.0) for b, rho, _, _ in tr.rows]
        print("split sweep", w["Ly"], order, c, max(ratio_dev), flush=True)
    for c in (chains if measure_chains is None else measure_chains):
        m64 = vmc.measure(g, start[c], w["chi"], W, 3, w["J1"], w["J2"])
        with SplitOracle(order):
            m32 = vmc.measure(g32, start[c], w["chi"], W32, 3, w["J1"], w["J2"])
        eloc_dev.append(abs(m32["eloc"] - m64["eloc"]) / m64["eloc_scale"])
        lp_dev.append(abs(m32["logpsi"] - m64["logpsi"]))
        G64, G32 = flat(m64["G"]), flat(m32["G"]).astype(np.float64)
        g_nrm.append(np.linalg.norm(G32 - G64) / np.linalg.norm(G64))
        g_el.append(np.max(np.abs(G32 - G64)) / np.max(np.abs(G64)))
        print("split measure", w["Ly"], order, c, eloc_dev[-1], lp_dev[-1], g_nrm[-1], g_el[-1], flush=True)
    out["sweep_ratio_max"] = float(np.max(ratio_dev))
    out["sweep_ratio_median"] = float(np.median(ratio_dev))
    out["eloc_rel_scale_max"] = float(np.max(eloc_dev))
    out["logpsi_abs_max"] = float(np.max(lp_dev))
    out["grad_norm_max"] = float(np.max(g_nrm))
    out["grad_elementwise_max"] = float(np.max(g_el))
    return out


def sweep_spread(w, start, seed, t, chains):
    g = vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])
    ref = {}
    for c in chains:
        tr = vmc.Trace()
        vmc.sweep(g, start[c], w["chi"], w["sketch"], 3, seed, c, t, trace=tr)
        ref[c] = tr.rows
    g32 = [[x.astype(F32) for x in row] for row in g]
    out = {}
    for order in ORDERS:
        dev = []
        with Float32Oracle(order):
            for c in chains:
                tr = vmc.Trace(follow={b: int(a) for b, _, _, a in ref[c]}, tie=1e-5)
                vmc.sweep(g32, start[c], w["chi"], w["sketch"].astype(F32), 3, seed, c, t, trace=tr)
                r64 = {b: rho for b, rho, _, _ in ref[c]}
                dev += [abs(rho - r64[b]) / max(abs(r64[b]), 1.0) for b, rho, _, _ in tr.rows]
        out["%s/%s" % order] = {"max": float(np.max(dev)), "median": float(np.median(dev))}
        print(order, out["%s/%s" % order], flush=True)
    return out


def grad_spread(w, configs):
    g = vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"])
    flat = lambda G: np.concatenate([x.ravel() for row in G for x in row])  # noqa: E731
    ref = [flat(vmc.measure(g, s, w["chi"], w["sketch"], 3, w["J1"], w["J2"])["G"]) for s in configs]
    g32 = [[x.astype(F32) for x in row] for row in g]
    out = {}
    for order in ORDERS:
        with Float32Oracle(order):
            errs = [np.linalg.norm(flat(vmc.measure(g32, s, w["chi"], w["sketch"].astype(F32), 3, w["J1"],
                                                    w["J2"])["G"]).astype(np.float64) - r) / np.linalg.norm(r)
                    for s, r in zip(configs, ref)]
        out["%s/%s" % order] = float(max(errs))
        print(order, out["%s/%s" % order], flush=True)
    return out


def _split_case(args):
    name, order = args
    if name == "8x8":
        w = inputs.workload("peps_8x8", n_chains=6)
        w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
        return split_spread(w, inputs.start_spins(6, 8, 8, 31, "random"), 11, 3, range(6), order=order)
    # the chains and start configurations that tests/test_gpu_parity_24x24.py checks
    w = inputs.workload("peps_24x24", n_chains=512)
    w["tensors"] = inputs.peps_tensors(24, 24, 8, w["seed"], False, bond_decay=1.0)
    return split_spread(w, inputs.start_spins(512, 24, 24, w["seed"], "random"), w["seed"], 7, SWEEP_CHAINS_24,
                        first_column_only=True, order=order, measure_chains=MEASURE_CHAINS_24)


def split_over_orders(name, pool):
    """Worst (and worst median) over the six rounding orders of each split-BF16 figure."""
    per = pool.map(_split_case, [(name, o) for o in ORDERS])
    out = {k: float(max(r[k] for r in per)) for k in per[0]}
    out["per_order"] = {"%s/%s" % o: r for o, r in zip(ORDERS, per)}
    return out


def summary(per_order):
    vals = list(per_order.values())
    if isinstance(vals[0], dict):
        return {"max": max(v["max"] for v in vals), "median": max(v["median"] for v in vals),
                "per_order": per_order}
    return {"max": max(vals), "per_order": per_order}


def main():
    if "--split-only" in sys.argv[1:] or "--split24-only" in sys.argv[1:]:
        # keep the float32 figures (and with --split24-only the 8x8 split ones), recompute the rest
        with open(os.path.join(HERE, "float32_spread.json")) as f:
            res = json.load(f)
        _split_into(res, only24="--split24-only" in sys.argv[1:])
        _write(res)
        return
    res = {"how": HOW}
    w = inputs.workload("peps_8x8", n_chains=6)
    w["tensors"] = inputs.peps_tensors(8, 8, 4, w["seed"], True, bond_decay=1.0)
    res["sweep_ratios_bond_decay_8x8"] = summary(
        sweep_spread(w, inputs.start_spins(6, 8, 8, 33, "random"), 77, 3, range(6)))
    w = inputs.workload("peps_8x8", n_chains=8)
    sampled = golden.load("peps_8x8")
    res["sweep_ratios_iid_8x8_sampled"] = summary(sweep_spread(w, sampled, 77, 12, (0, 3, 5, 7)))
    res["grad_iid_8x8_sampled"] = summary(grad_spread(w, sampled))
    _split_into(res)
    _write(res)


def _split_into(res, only24=False):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(len(ORDERS)) as pool:
        if not only24:
            res["split_bf16_bond_decay_8x8"] = split_over_orders("8x8", pool)
        res["split_bf16_bond_decay_24x24"] = split_over_orders("24x24", pool)
    res["how"] = HOW


HOW = ("tests/golden/make_float32_spread.py: the oracle in float32 (plain Householder QR) and in emulated split "
       "BF16 (hi.hi + hi.lo + lo.hi per pairwise product), each in 3 dot-product orders x 2 contraction orders, "
       "against the float64 oracle")


def _write(res):
    with open(os.path.join(HERE, "float32_spread.json"), "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
