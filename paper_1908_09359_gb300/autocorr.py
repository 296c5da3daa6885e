"""Integrated autocorrelation time and effective sample counts of Markov-chain series.

The sampler runs many independent chains, each producing one sample per sweep (Sec. II:
one sweep of the sequential scheme, then E_loc and G on the final configuration).  The
samples of one chain are correlated; the number of independent samples a run is worth
is n_samples / (2 tau_int) with

    tau_int = 1/2 + sum_{t >= 1} rho(t),

rho the normalised autocorrelation function of the observable.  The sum is cut at the
first window W with W >= c tau_int(W) (Sokal's automatic windowing, c = 5), which keeps
the estimator's variance bounded while the neglected tail stays small for a single
dominant relaxation mode.

For several chains the autocovariance of each chain about the common mean is averaged
over chains before normalising, so short chains still give a usable estimate when
tau_int is well below the chain length.  Host-side NumPy; nothing here touches the
device.
"""
import numpy as np


def autocovariance(x):
    """Autocovariance c(t), t = 0 .. T-1, of series x of shape (T,) or (T, n_chains),
    each chain about the mean over all chains, averaged over chains (FFT, zero padded
    so there is no wrap-around)."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    T = x.shape[0]
    if T < 2:
        raise ValueError("need at least two samples per chain")
    y = x - x.mean()
    n = 1 << int(np.ceil(np.log2(2 * T)))
    f = np.fft.rfft(y, n=n, axis=0)
    acf = np.fft.irfft(f * np.conj(f), n=n, axis=0)[:T]
    # lag-t products available per chain: T - t
    acf /= (T - np.arange(T))[:, None]
    return acf.mean(axis=1)


def tau_int(x, c=5.0):
    """(tau_int, window) of series x (T,) or (T, n_chains) by automatic windowing.

    A constant series (zero variance) has tau_int = 1/2 by convention: every sample is
    as good as independent for estimating its (exact) mean."""
    cov = autocovariance(x)
    if cov[0] <= 0.0:
        return 0.5, 0
    rho = cov / cov[0]
    tau = 0.5
    for w in range(1, len(rho)):
        tau += rho[w]
        if w >= c * tau:
            return float(tau), w
    return float(tau), len(rho) - 1


def effective_samples(x, c=5.0):
    """Number of independent samples a run of x (T, n_chains) is worth."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    t, _ = tau_int(x, c)
    return n / (2.0 * t)


def mean_and_error(x, c=5.0):
    """Mean of x (T,) or (T, n_chains) and its standard error corrected by tau_int."""
    x = np.asarray(x, dtype=np.float64)
    t, _ = tau_int(x, c)
    var = autocovariance(x)[0]
    return float(x.mean()), float(np.sqrt(max(var, 0.0) * 2.0 * t / x.size))


def staggered_mz2(spins):
    """Squared staggered magnetisation per configuration, (sum_i (-1)^(x+y) S^z_i / N)^2
    with S^z = sigma / 2, for spins of shape (..., Ly, Lx) in {-1, +1}."""
    s = np.asarray(spins, dtype=np.float64)
    Ly, Lx = s.shape[-2:]
    sign = (-1.0) ** np.add.outer(np.arange(Ly), np.arange(Lx))
    m = 0.5 * np.sum(s * sign, axis=(-2, -1)) / (Ly * Lx)
    return m * m
