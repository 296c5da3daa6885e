"""The tau_int estimator against series whose autocorrelation is known in closed form.

AR(1), x_t = phi x_{t-1} + e_t, has rho(t) = phi^t and so tau_int = (1 + phi) / (2 (1 - phi));
iid noise has tau_int = 1/2; the tau-corrected error bar of the mean must match the
spread of the mean over independent replicas.
"""
import numpy as np
import pytest

from paper_1908_09359_gb300 import autocorr


def ar1(phi, T, n, rng):
    x = np.empty((T, n))
    x[0] = rng.standard_normal(n) / np.sqrt(1 - phi * phi)   # stationary start
    e = rng.standard_normal((T, n))
    for t in range(1, T):
        x[t] = phi * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("phi", [0.5, 0.8, 0.95])
def test_ar1_tau_matches_closed_form(phi):
    rng = np.random.default_rng(int(phi * 100))
    x = ar1(phi, 4000, 64, rng)
    tau, w = autocorr.tau_int(x)
    exact = (1 + phi) / (2 * (1 - phi))
    # Sokal: var(tau) ~ 2 (2W + 1) / n tau^2; the cut tail phi^(W+1) / (1 - phi) is below
    # 1 % of tau at W >= 5 tau
    rel = 3 * np.sqrt(2 * (2 * w + 1) / x.size) + 0.01
    assert tau == pytest.approx(exact, rel=rel)
    assert w >= 5 * tau * 0.99


def test_iid_and_constant_series():
    rng = np.random.default_rng(0)
    tau, _ = autocorr.tau_int(rng.standard_normal((2000, 32)))
    assert tau == pytest.approx(0.5, abs=0.03)
    assert autocorr.tau_int(np.ones((50, 4)))[0] == 0.5


def test_autocovariance_matches_direct_sum():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((37, 5))
    y = x - x.mean()
    direct = [np.mean([np.mean(y[: 37 - t, c] * y[t:, c]) for c in range(5)]) for t in range(37)]
    assert np.allclose(autocorr.autocovariance(x), direct, rtol=1e-12, atol=1e-14)


def test_error_bar_matches_replica_spread():
    rng = np.random.default_rng(7)
    phi = 0.9
    means, errs = [], []
    for _ in range(200):
        x = ar1(phi, 400, 8, rng)
        m, e = autocorr.mean_and_error(x)
        means.append(m)
        errs.append(e)
    spread = np.std(means)
    assert np.median(errs) == pytest.approx(spread, rel=0.15)


def test_staggered_magnetisation():
    neel = np.where(np.add.outer(np.arange(4), np.arange(6)) % 2 == 0, 1, -1)
    assert autocorr.staggered_mz2(neel) == pytest.approx(0.25)
    stripes = np.tile(np.array([1, 1, -1, -1, 1, -1]), (4, 1))
    s = np.stack([neel, stripes])
    m = autocorr.staggered_mz2(s)
    expect = (0.5 * np.sum(stripes * np.where(np.add.outer(np.arange(4), np.arange(6)) % 2 == 0, 1, -1)) / 24) ** 2
    assert m[0] == pytest.approx(0.25) and m[1] == pytest.approx(expect)
