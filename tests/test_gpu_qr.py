"""pepsvmc_qr_pos, the batched thin QR with diag(R) > 0 that moves the orthogonality
centre in the variational fit (App. B), against the oracle's qr_pos.

Well-conditioned input must match the oracle's Q element by element within a bound
that scales with the condition number; for every input, including ill-conditioned and
rank-deficient ones, Q must be orthonormal, Q^T Y upper triangular with a non-negative
diagonal, and Y = Q (Q^T Y), all checked in float64.
"""
import numpy as np
import pytest

from oracle import vmc

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)
# orthogonality and backward error of a float32 Householder QR of up to 300 x 40: a few
# ulps times sqrt(rows) at most (the method is backward stable to O(u))
ORTH_TOL = 64 * EPS32
# forward error of Q: the backward error amplified by the condition number
FWD_TOL_PER_KAPPA = 64 * EPS32


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import build
    build.build()
    return t


def conditioned(rng, rows, cols, kappa):
    """rows x cols with singular values log-spaced from 1 to 1/kappa."""
    U, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, cols)))
    return (U * np.logspace(0, -np.log10(kappa), cols)) @ V.T


def run(torch, Y, col_major=False, in_place=False):
    """Y: float32 (batch, rows, cols); returns Q (batch, rows, cols) in float64."""
    from paper_1908_09359_gb300 import api
    store = np.ascontiguousarray(Y.transpose(0, 2, 1) if col_major else Y)
    dY = torch.from_numpy(store).cuda()
    dQ = dY if in_place else torch.full_like(dY, float("nan"))
    api.qr_pos(dY, dQ, col_major=col_major)
    torch.cuda.synchronize()
    Q = dQ.cpu().numpy().astype(np.float64)
    return Q.transpose(0, 2, 1) if col_major else Q


def check_valid(Y, Q):
    """Orthonormal Q, R = Q^T Y upper triangular with R(j,j) >= 0, Y = Q R."""
    for b in range(Y.shape[0]):
        y, q = Y[b].astype(np.float64), Q[b]
        scale = np.linalg.norm(y, 2)
        assert np.max(np.abs(q.T @ q - np.eye(q.shape[1]))) <= ORTH_TOL
        r = q.T @ y
        assert np.max(np.abs(np.tril(r, -1))) <= ORTH_TOL * scale
        assert np.min(np.diag(r)) >= -ORTH_TOL * scale
        assert np.max(np.abs(y - q @ r)) <= ORTH_TOL * scale


# the register form (rows <= 256, cols <= 32) in its three block sizes, ragged shapes,
# and the shared-memory form beyond it
@pytest.mark.parametrize("rows,cols", [(256, 32), (128, 32), (64, 32), (8, 8), (72, 24), (200, 17), (300, 40),
                                       (64, 64)])
@pytest.mark.parametrize("col_major", [False, True])
def test_matches_the_oracle(torch, rows, cols, col_major):
    rng = np.random.default_rng(rows * 100 + cols + 7 * col_major)
    kappas = (1.0, 10.0, 100.0)
    Y = np.stack([conditioned(rng, rows, cols, k) for k in kappas]).astype(np.float32)
    Q = run(torch, Y, col_major)
    check_valid(Y, Q)
    for b, kappa in enumerate(kappas):
        ref, _ = vmc.qr_pos(Y[b].astype(np.float64))
        assert np.max(np.abs(Q[b] - ref)) <= FWD_TOL_PER_KAPPA * kappa * np.sqrt(rows)


def test_in_place_batch(torch):
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((64, 256, 32)).astype(np.float32)
    Q = run(torch, Y, in_place=True)
    check_valid(Y, Q)
    for b in (0, 31, 63):
        ref, _ = vmc.qr_pos(Y[b].astype(np.float64))
        assert np.max(np.abs(Q[b] - ref)) <= FWD_TOL_PER_KAPPA * 10 * 16


def test_ill_conditioned_and_rank_deficient(torch):
    rng = np.random.default_rng(11)
    Y = np.stack([conditioned(rng, 256, 32, 1e6), conditioned(rng, 256, 32, 1e5),
                  rng.standard_normal((256, 32)), rng.standard_normal((256, 32))]).astype(np.float32)
    Y[2][:, 5] = 0.0                      # a zero column
    Y[3][:, 9] = Y[3][:, 2]               # a repeated column
    Q = run(torch, Y)
    check_valid(Y, Q)
    # the zero column gets R(5,5) = 0
    r = Q[2].T @ Y[2].astype(np.float64)
    assert abs(r[5, 5]) <= ORTH_TOL * np.linalg.norm(Y[2], 2)


def test_rejects_invalid_sizes(torch):
    from paper_1908_09359_gb300 import api
    from paper_1908_09359_gb300._lib import PepsvmcError
    Y = torch.zeros((2, 4, 8), device="cuda")
    with pytest.raises(PepsvmcError):
        api.qr_pos(Y, Y)  # rows < cols
