"""Python binding of the pepsvmc C ABI: argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module copies
numpy arrays in and out and passes torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import EINVAL, ESTATE, FP32, MIXED_BF16, MIXED_BF16X3, MIXED_TF32, PepsvmcError  # noqa: F401


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _i8(a):
    return a.ctypes.data_as(C.POINTER(C.c_int8)) if a is not None else None


PRECISIONS = {"fp32": FP32, "bf16": MIXED_BF16, "tf32": MIXED_TF32, "bf16x3": MIXED_BF16X3}


class PepsVMC:
    """One pepsvmc context (one device, n_chains Markov chains).

    ``tensors``: float64 packed PEPS (see include/pepsvmc.h), ``sketch``: float64
    (max(Ly,Lx), chi, D, chi) starting guess of the truncation fit.
    """

    def __init__(self, Ly, Lx, D, chi, n_chains, tensors, sketch, J1=1.0, J2=0.0, seed=0, n_fit=3,
                 precision=FP32, stream=None, chi_measure=0, wait_budget_cycles=0, chain_offset=0,
                 symmetrize=False):
        self.lib = _lib.load()
        cfg = _lib.Config()
        cfg.Ly, cfg.Lx, cfg.D, cfg.chi, cfg.n_chains, cfg.n_fit = Ly, Lx, D, chi, n_chains, n_fit
        cfg.J1, cfg.J2, cfg.seed, cfg.precision = float(J1), float(J2), int(seed), int(precision)
        cfg.chi_measure = int(chi_measure)
        cfg.wait_budget_cycles = int(wait_budget_cycles)
        cfg.chain_offset = int(chain_offset)
        cfg.symmetrize = 1 if symmetrize else 0
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.shape = (n_chains, Ly, Lx)
        self.n_chains, self.Ly, self.Lx = n_chains, Ly, Lx
        t = np.ascontiguousarray(tensors, dtype=np.float64)
        s = np.ascontiguousarray(sketch, dtype=np.float64)
        X = max(chi, chi_measure)
        if s.shape != (max(Ly, Lx), X, D, X):
            raise ValueError(f"sketch must have shape {(max(Ly, Lx), X, D, X)}")
        self.ctx = C.c_void_p()
        rc = self.lib.pepsvmc_init(C.byref(cfg), _dp(t), _dp(s), C.c_void_p(stream), C.byref(self.ctx))
        if rc != 0:
            msg = self.lib.pepsvmc_last_error(self.ctx).decode() if self.ctx else ""
            if self.ctx:
                self.lib.pepsvmc_destroy(self.ctx)
                self.ctx = None
            raise PepsvmcError(rc, msg)
        if t.size != self.n_params:
            self.close()
            raise ValueError(f"tensors must have {self.n_params} entries, got {t.size}")

    # ----------------------------------------------------------------- plumbing
    def _check(self, rc):
        if rc != 0:
            raise PepsvmcError(rc, self.lib.pepsvmc_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pepsvmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_params(self):
        return int(self.lib.pepsvmc_n_params(self.ctx))

    @property
    def n_grad_entries(self):
        return int(self.lib.pepsvmc_n_grad_entries(self.ctx))

    @property
    def launches(self):
        return int(self.lib.pepsvmc_launch_count(self.ctx))

    @property
    def n_bonds(self):
        return 2 * self.Lx * self.Ly - self.Lx - self.Ly

    # ----------------------------------------------------------------- state
    def set_spins(self, spins):
        s = np.ascontiguousarray(spins, dtype=np.int8).reshape(self.shape)
        self._check(self.lib.pepsvmc_set_spins(self.ctx, _i8(s)))

    def get_spins(self):
        s = np.empty(self.shape, dtype=np.int8)
        self._check(self.lib.pepsvmc_get_spins(self.ctx, _i8(s)))
        return s

    def set_tensors(self, t):
        t = np.ascontiguousarray(t, dtype=np.float64)
        self._check(self.lib.pepsvmc_set_tensors(self.ctx, _dp(t)))

    def get_tensors(self):
        t = np.empty(self.n_params, dtype=np.float64)
        self._check(self.lib.pepsvmc_get_tensors(self.ctx, _dp(t)))
        return t

    def set_sweep_counter(self, n):
        self._check(self.lib.pepsvmc_set_sweep_counter(self.ctx, int(n)))

    @property
    def sweep_counter(self):
        return int(self.lib.pepsvmc_get_sweep_counter(self.ctx))

    # ----------------------------------------------------------------- hot path
    def sample_sweep(self, n_sweeps=1):
        r = C.c_double()
        self._check(self.lib.pepsvmc_sample_sweep(self.ctx, int(n_sweeps), C.byref(r)))
        return r.value

    def random_sweep(self, n_sweeps=1):
        """Sweeps of the random-NNASP scheme (N attempts each); returns the acceptance rate."""
        r = C.c_double()
        self._check(self.lib.pepsvmc_random_sweep(self.ctx, int(n_sweeps), C.byref(r)))
        return r.value

    def get_random_trace(self):
        shp = (self.n_chains, self.Ly * self.Lx)
        bond = np.empty(shp, dtype=np.int32)
        ratio = np.empty(shp)
        dec = np.empty(shp, dtype=np.int8)
        self._check(self.lib.pepsvmc_get_random_trace(self.ctx, bond.ctypes.data_as(C.POINTER(C.c_int32)),
                                                      _dp(ratio), _i8(dec)))
        return bond, ratio, dec

    def enable_trace(self, on=True):
        self._check(self.lib.pepsvmc_enable_trace(self.ctx, 1 if on else 0))

    def get_trace(self):
        ratio = np.empty((self.n_chains, self.n_bonds), dtype=np.float64)
        dec = np.empty((self.n_chains, self.n_bonds), dtype=np.int8)
        self._check(self.lib.pepsvmc_get_trace(self.ctx, _dp(ratio), _i8(dec)))
        return ratio, dec

    def measure(self):
        e = np.empty(self.n_chains)
        lp = np.empty(self.n_chains)
        sg = np.empty(self.n_chains, dtype=np.int8)
        self._check(self.lib.pepsvmc_measure(self.ctx, _dp(e), _dp(lp), _i8(sg)))
        return e, lp, sg

    def phi(self):
        """(E^Phi, w) per S, S-bar pair of the last measurement (symmetrize=True)."""
        e = np.empty(self.n_chains // 2)
        w = np.empty(self.n_chains // 2)
        self._check(self.lib.pepsvmc_get_phi(self.ctx, _dp(e), _dp(w)))
        return e, w

    def chain_grad(self, chain):
        g = np.empty(self.n_grad_entries)
        self._check(self.lib.pepsvmc_get_chain_grad(self.ctx, int(chain), _dp(g)))
        return g

    def amplitude(self, row):
        lp = np.empty(self.n_chains)
        sg = np.empty(self.n_chains, dtype=np.int8)
        self._check(self.lib.pepsvmc_amplitude(self.ctx, int(row), _dp(lp), _i8(sg)))
        return lp, sg

    def energy_and_grad(self, n_sweeps, want_samples=True, want_grad=True):
        Em, Ev = C.c_double(), C.c_double()
        n = int(n_sweeps) * self.n_chains
        el = np.empty(n) if want_samples else None
        lp = np.empty(n) if want_samples else None
        sg = np.empty(n, dtype=np.int8) if want_samples else None
        gr = np.empty(self.n_params) if want_grad else None
        self._check(self.lib.pepsvmc_energy_and_grad(self.ctx, int(n_sweeps), C.byref(Em), C.byref(Ev),
                                                     _dp(el), _dp(lp), _i8(sg), _dp(gr)))
        return dict(E_mean=Em.value, E_var=Ev.value, eloc=el, logpsi=lp, sign=sg, grad=gr)

    def set_profiling(self, on=True):
        self._check(self.lib.pepsvmc_set_profiling(self.ctx, 1 if on else 0))

    def get_profile(self):
        out = np.zeros(6)
        self._check(self.lib.pepsvmc_get_profile(self.ctx, _dp(out)))
        return dict(gemm_launches=int(out[0]), gemm_flops=out[1], gemm_ms=out[2],
                    qr_launches=int(out[3]), qr_ms=out[4], gemm_bytes=out[5])

    def env3_left(self, E, T, A, spins, B, out, dims):
        """Three-line environment step on device tensors (torch CUDA tensors or raw
        pointers); ``dims`` = (n_chains, cT, cB, cT2, cB2, Dl, Dr, Du, Dd)."""
        ptr = lambda t: C.c_void_p(t if isinstance(t, int) else (t.data_ptr() if t is not None else 0))  # noqa: E731
        self._check(self.lib.pepsvmc_env3_left(self.ctx, ptr(E), ptr(T), ptr(A), ptr(spins), ptr(B), ptr(out),
                                               *[int(v) for v in dims]))

    def env4_left(self, E, T, A1, spins1, A2, spins2, B, out, dims, bmajor=False):
        """Four-line environment step on device tensors; ``dims`` = (n_chains, cT, cB, cT2,
        cB2, D1l, D1r, Du1, Dd1, D2l, D2r, Dd2); bmajor: E and out stored [b][a][l1][l2]."""
        ptr = lambda t: C.c_void_p(t if isinstance(t, int) else (t.data_ptr() if t is not None else 0))  # noqa: E731
        self._check(self.lib.pepsvmc_env4_left(self.ctx, ptr(E), ptr(T), ptr(A1), ptr(spins1), ptr(A2), ptr(spins2),
                                               ptr(B), ptr(out), *[int(v) for v in dims], 1 if bmajor else 0))

    def get_profile_shapes(self):
        import json
        buf = C.create_string_buffer(1 << 20)
        self._check(self.lib.pepsvmc_get_profile_shapes(self.ctx, buf, len(buf)))
        return json.loads(buf.value.decode())

    # ------------------------------------------------------------- learned proposal
    def set_proposal_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        if p.size != _lib.NET_PARAMS:
            raise ValueError(f"proposal network needs {_lib.NET_PARAMS} parameters")
        self._check(self.lib.pepsvmc_set_proposal_params(self.ctx, _dp(p)))

    def get_proposal_params(self):
        p = np.empty(_lib.NET_PARAMS)
        self._check(self.lib.pepsvmc_get_proposal_params(self.ctx, _dp(p)))
        return p

    def proposal_logits(self):
        out = np.empty((self.n_chains, 2, self.Ly, self.Lx))
        self._check(self.lib.pepsvmc_proposal_logits(self.ctx, _dp(out)))
        return out

    def proposal_collect(self, n_sweeps):
        self._check(self.lib.pepsvmc_proposal_collect(self.ctx, int(n_sweeps)))
        return int(self.lib.pepsvmc_proposal_dataset_size(self.ctx))

    def proposal_dataset_size(self):
        return int(self.lib.pepsvmc_proposal_dataset_size(self.ctx))

    def proposal_load(self, spins, rho):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        r = np.ascontiguousarray(rho, dtype=np.float64)
        self._check(self.lib.pepsvmc_proposal_load(self.ctx, _i8(s), _dp(r), len(s)))

    def proposal_train(self, epochs, batch, lr):
        loss = C.c_double()
        self._check(self.lib.pepsvmc_proposal_train(self.ctx, int(epochs), int(batch), float(lr), C.byref(loss)))
        return loss.value

    def train_proposal(self, configs, epochs, lr):
        """Measure the given +-1 configurations (n, Ly, Lx), train on them, return the
        last epoch's mean loss."""
        c = np.ascontiguousarray(configs, dtype=np.int8).reshape(-1, self.Ly, self.Lx)
        loss = C.c_double()
        self._check(self.lib.pepsvmc_train_proposal(self.ctx, _i8(c), int(len(c)), int(epochs), float(lr),
                                                     C.byref(loss)))
        return loss.value

    def set_proposal(self, mode):
        self._check(self.lib.pepsvmc_set_proposal(self.ctx, int(mode)))

    def learned_sweep(self, n=1):
        r = C.c_double()
        self._check(self.lib.pepsvmc_learned_sweep(self.ctx, int(n), C.byref(r)))
        return r.value

    def get_learned_trace(self):
        shp = (self.n_chains, self.Ly - 1)
        rho, dlq, dec = np.empty(shp), np.empty(shp), np.empty(shp, dtype=np.int8)
        self._check(self.lib.pepsvmc_get_learned_trace(self.ctx, _dp(rho), _dp(dlq), _i8(dec)))
        return rho, dlq, dec

    def set_graphs(self, on=True):
        self._check(self.lib.pepsvmc_set_graphs(self.ctx, 1 if on else 0))

    def set_contraction_kernel(self, kind, tile=0):
        """kind: "auto", "f32" (tile 0..5), "tc" (N tile 32, 64, 128, 256) or "tc2" (split
        BF16 with two shared-memory stages, N tile 32 or 64)."""
        k = {"auto": 0, "f32": 1, "tc": 2, "tc2": 3}[kind]
        self._check(self.lib.pepsvmc_set_contraction_kernel(self.ctx, k, int(tile)))

    def set_autotune(self, on=True):
        self._check(self.lib.pepsvmc_set_autotune(self.ctx, 1 if on else 0))

    def get_tuning(self):
        import json
        buf = C.create_string_buffer(1 << 22)
        self._check(self.lib.pepsvmc_get_tuning(self.ctx, buf, len(buf)))
        return json.loads(buf.value.decode())

    def update(self, delta, step):
        self._check(self.lib.pepsvmc_update(self.ctx, float(delta), int(step)))

    def set_fused(self, on=True):
        self._check(self.lib.pepsvmc_set_fused(self.ctx, 1 if on else 0))

    def set_wait_budget(self, cycles):
        self._check(self.lib.pepsvmc_set_wait_budget(self.ctx, int(cycles)))

    # ------------------------------------------------- gradient sums (multi-rank jobs)
    def get_sums(self):
        """(scalars[3] = sum E, sum E^2, n; sumGE; sumG) of the last energy_and_grad."""
        sc = np.empty(3)
        ge = np.empty(self.n_params)
        g = np.empty(self.n_params)
        self._check(self.lib.pepsvmc_get_sums(self.ctx, _dp(sc), _dp(ge), _dp(g)))
        return sc, ge, g

    def set_sums(self, scalars, sumGE, sumG):
        """Replace the sums (e.g. by their all-reduced totals) and recompute the gradient."""
        sc = np.ascontiguousarray(scalars, dtype=np.float64)
        ge = np.ascontiguousarray(sumGE, dtype=np.float64)
        g = np.ascontiguousarray(sumG, dtype=np.float64)
        if sc.size != 3 or ge.size != self.n_params or g.size != self.n_params:
            raise ValueError("set_sums: scalars must have 3 entries, sumGE and sumG n_params each")
        self._check(self.lib.pepsvmc_set_sums(self.ctx, _dp(sc), _dp(ge), _dp(g)))

    def sums_device(self):
        """Device addresses (scalars, sumGE, sumG) of the context's float64 sums."""
        a, b, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
        self._check(self.lib.pepsvmc_sums_device(self.ctx, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def finalize_sums(self):
        """Recompute the gradient from the device sums (after an in-place reduction)."""
        self._check(self.lib.pepsvmc_finalize_sums(self.ctx))


def env3_left_noalloc(E, T, A, spins, B, out, dims, stream=None):
    """The three-line environment step without a context and without any device
    allocation (for callers that must not allocate once running); the intermediates
    use the library's fixed scratch array, so calls must not overlap on the GPU.
    Arguments as PepsVMC.env3_left; ``stream`` defaults to torch's current stream."""
    lib = _lib.load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    ptr = lambda t: C.c_void_p(t if isinstance(t, int) else (t.data_ptr() if t is not None else 0))  # noqa: E731
    rc = lib.pepsvmc_env3_left_noalloc(ptr(E), ptr(T), ptr(A), ptr(spins), ptr(B), ptr(out),
                                       *[int(v) for v in dims], C.c_void_p(stream))
    if rc != 0:
        raise PepsvmcError(rc, "pepsvmc_env3_left_noalloc failed (sizes beyond the fixed scratch, "
                               "null pointers or a CUDA error)")


def qr_pos(Y, Q, col_major=False, stream=None):
    """Batched thin QR with diag(R) > 0 (pepsvmc_qr_pos) of the float32 CUDA tensor Y
    (batch, rows, cols) into Q (same shape; may be Y itself).  Y and Q hold each matrix
    row-major, or column-major with col_major (then the tensors' last two dimensions are
    read as (cols, rows))."""
    lib = _lib.load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    batch = Y.shape[0]
    rows, cols = (Y.shape[2], Y.shape[1]) if col_major else (Y.shape[1], Y.shape[2])
    rc = lib.pepsvmc_qr_pos(C.c_void_p(Y.data_ptr()), C.c_void_p(Q.data_ptr()), int(batch), int(rows), int(cols),
                            int(bool(col_major)), C.c_void_p(stream))
    if rc != 0:
        raise PepsvmcError(rc, "pepsvmc_qr_pos failed (invalid sizes, null pointers or a CUDA error)")


def simple_update(Ly, Lx, D, B, lam_h, lam_v, J1=1.0, J2=0.0, tau=0.01, max_steps=100, tol=1e-11, stream=None):
    """Simple-update imaginary-time evolution (pepsvmc_simple_update) from the packed site
    tensors B and link vectors lam_h (Ly, Lx-1, D), lam_v (Ly-1, Lx, D).  Returns
    (B, lam_h, lam_v, peps, steps, change): the evolved state, the Monte Carlo tensors
    with lambda^(1/2) absorbed, the steps run and the last mean relative lambda change."""
    lib = _lib.load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    b = np.ascontiguousarray(B, dtype=np.float64).copy()
    lh = np.ascontiguousarray(lam_h, dtype=np.float64).reshape(Ly, max(Lx - 1, 0), D).copy()
    lv = np.ascontiguousarray(lam_v, dtype=np.float64).reshape(max(Ly - 1, 0), Lx, D).copy()
    out = np.empty_like(b)
    steps = C.c_int32()
    change = C.c_double()
    rc = lib.pepsvmc_simple_update(int(Ly), int(Lx), int(D), float(J1), float(J2), float(tau), int(max_steps),
                                   float(tol), _dp(b), _dp(lh), _dp(lv), _dp(out), C.byref(steps), C.byref(change),
                                   C.c_void_p(stream))
    if rc != 0:
        raise PepsvmcError(rc, "pepsvmc_simple_update failed")
    return b, lh, lv, out, steps.value, change.value
