"""Simple update (App. A) on the GPU against the oracle (oracle/simple_update.py).

Both sides run in float64 with the same Trotter order, truncation rule and sign rule of
the singular vectors; they differ in the SVD algorithm (LAPACK on the oracle side, Jacobi
eigen-decomposition of the short-side Gram matrix on the GPU), which changes a singular
value sigma_i by ~1e-16 sigma_max^2 / sigma_i and its vectors by that over the gap.  On
these random states the kept singular values stay above ~1e-3 sigma_max, so the lambdas
are compared to 1e-8 and every site tensor to 1e-7 of its norm after one Trotter step,
and to 1e-6 after twenty.  The evolved tensors, with lambda^(1/2) absorbed, then drive the
Monte Carlo sampler, whose mean E_loc at exact Dc matches the enumerated energy of that
PEPS within five tau-corrected standard errors.
"""
import numpy as np
import pytest

from oracle import exact, simple_update as su, vmc
from paper_1908_09359_gb300 import autocorr, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    from paper_1908_09359_gb300 import api as a
    return a


def start(Ly, Lx, D, seed):
    st = su.init_state(Ly, Lx, D, seed)
    rng = np.random.default_rng(seed + 1)
    for row in st.lh + st.lv:
        for i in range(len(row)):
            v = rng.uniform(0.2, 1.0, size=D)
            row[i] = v / np.linalg.norm(v)
    return st


def arrays(st):
    lh = np.array(st.lh, dtype=np.float64).reshape(st.Ly, st.Lx - 1, -1)
    lv = np.array(st.lv, dtype=np.float64).reshape(st.Ly - 1, st.Lx, -1)
    return vmc.pack(st.B), lh, lv


def compare(st, B, lh, lv, tol_lam, tol_t):
    ref_B, ref_lh, ref_lv = arrays(st)
    assert np.max(np.abs(lh - ref_lh)) <= tol_lam and np.max(np.abs(lv - ref_lv)) <= tol_lam
    got = vmc.unpack(B, st.Ly, st.Lx, ref_lh.shape[-1])
    for k in range(st.Ly):
        for m in range(st.Lx):
            ref = st.B[k][m]
            assert np.linalg.norm(got[k][m] - ref) <= tol_t * np.linalg.norm(ref), (k, m)


@pytest.mark.parametrize("Ly,Lx,D,J2", [(4, 4, 2, 0.0), (4, 4, 3, 0.5), (3, 5, 4, 0.5), (6, 6, 8, 0.5)])
def test_one_trotter_step_matches_oracle(api, Ly, Lx, D, J2):
    st = start(Ly, Lx, D, 7)
    B, lh, lv = arrays(st)
    B2, lh2, lv2, peps, steps, _ = api.simple_update(Ly, Lx, D, B, lh, lv, J1=1.0, J2=J2, tau=0.1, max_steps=1,
                                                     tol=-1.0)
    assert steps == 1
    su.trotter_step(st, 1.0, J2, 0.1, D)
    compare(st, B2, lh2, lv2, 1e-8, 1e-7)
    ref = vmc.pack(su.to_peps(st))
    assert np.linalg.norm(peps - ref) <= 1e-7 * np.linalg.norm(ref)


def test_twenty_steps_match_and_converge(api):
    Ly, Lx, D = 4, 4, 2
    st = start(Ly, Lx, D, 3)
    B, lh, lv = arrays(st)
    B2, lh2, lv2, peps, steps, change = api.simple_update(Ly, Lx, D, B, lh, lv, J1=1.0, J2=0.5, tau=0.05,
                                                          max_steps=20, tol=-1.0)
    assert steps == 20
    changes = []
    for _ in range(20):
        old = st.copy()
        su.trotter_step(st, 1.0, 0.5, 0.05, D)
        changes.append(su.lambda_change(old, st))
    compare(st, B2, lh2, lv2, 1e-6, 1e-6)
    assert abs(change - changes[-1]) <= 1e-6
    # stopping rule: a tolerance above the first step's change stops after one step
    *_, s1, _ = api.simple_update(Ly, Lx, D, B, lh, lv, J1=1.0, J2=0.5, tau=0.05, max_steps=20, tol=1.0)
    assert s1 == 1


def test_simple_update_tensors_drive_the_sampler(api):
    """App. A's hand-over: the evolved PEPS (lambda^(1/2) absorbed) is the sampler's input;
    at exact Dc its mean E_loc equals the enumerated energy of that PEPS, which lies below
    the random start's energy and above the exact ground-state energy E0 = -9.18921 of the
    4x4 open Heisenberg lattice (variational), within 10 % of E0 at D = 2."""
    Ly, Lx, D, E0 = 4, 4, 2, -9.189207065192946
    st = su.init_state(Ly, Lx, D, 5)
    B, lh, lv = arrays(st)
    E_start = exact.energy_exact(su.to_peps(st), 1.0, 0.0)[0]
    _, _, _, peps, steps, _ = api.simple_update(Ly, Lx, D, B, lh, lv, J1=1.0, J2=0.0, tau=0.05, max_steps=150,
                                                tol=1e-9)
    assert steps > 1
    E_su = exact.energy_exact(vmc.unpack(peps, Ly, Lx, D), 1.0, 0.0)[0]
    assert E0 - 1e-9 <= E_su < E_start
    assert E_su <= 0.9 * E0, (E_su, E0)
    C = 1024
    sk = inputs.sketch(4, 4, 2, 11)
    ctx = api.PepsVMC(Ly, Lx, D, 4, C, peps, sk, J1=1.0, J2=0.0, seed=3, n_fit=1)
    ctx.set_spins(inputs.start_spins(C, 4, 4, 7, "random"))
    ctx.sample_sweep(20)
    el = ctx.energy_and_grad(40, want_grad=False)["eloc"].reshape(40, C)
    mean, err = autocorr.mean_and_error(el)
    assert abs(mean - E_su) <= 5 * err, (mean, E_su, err)
    ctx.close()
