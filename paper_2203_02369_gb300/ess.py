"""Effective sample size of MCMC traces (host, float64).

Geyer's initial monotone sequence estimator (Geyer 1992, "Practical Markov
chain Monte Carlo", Statistical Science 7): sum the autocorrelations in
adjacent pairs Gamma_m = rho_{2m} + rho_{2m+1}, stop at the first
non-positive pair, and force the pair sums to be non-increasing.
"""
from __future__ import annotations

import numpy as np


def autocorr(x):
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    x = x - x.mean()
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f), 2 * n)[:n]
    if ac[0] <= 0:
        return np.ones(1)
    return ac / ac[0]


def ess(x):
    """ESS of one scalar trace (n / integrated autocorrelation time)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if n < 4 or np.all(x == x[0]):
        return float(n) if n else 0.0
    rho = autocorr(x)
    pairs = []
    m = 0
    while 2 * m + 1 < n:
        g = rho[2 * m] + rho[2 * m + 1]
        if g <= 0:
            break
        if pairs and g > pairs[-1]:
            g = pairs[-1]
        pairs.append(g)
        m += 1
    tau = -1.0 + 2.0 * float(np.sum(pairs)) if pairs else 1.0
    tau = max(tau, 1.0 / n)
    return float(min(n / tau, n * np.log10(max(n, 10))))


def ess_columns(X):
    """ESS of every column of a (n_samples, n_vars) array."""
    X = np.asarray(X, dtype=np.float64)
    return np.array([ess(X[:, j]) for j in range(X.shape[1])])
