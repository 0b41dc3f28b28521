"""Integrated autocorrelation time of a Monte Carlo series (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/dqmc.py).

The paper reports an autocorrelation time of S_CDW (Benchmarks section) without naming
its estimator.  Reading used here: the integrated autocorrelation time
tau_int = 1/2 + sum_{t=1}^{W} rho(t), with the self-consistent window of Madras and
Sokal (the smallest W with W >= c * tau_int(W), c = 6), so that a series of n sweeps
holds n / (2 tau_int) independent samples.
"""
import numpy as np


def autocorrelation(x):
    """rho(t) for t = 0..n-1 with C(t) = (1/n) sum_s (x_s - xbar)(x_{s+t} - xbar)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    d = x - x.mean()
    c0 = float(d @ d) / n
    if c0 == 0.0:
        out = np.zeros(n)
        out[0] = 1.0
        return out
    rho = np.empty(n)
    for t in range(n):
        rho[t] = float(d[: n - t] @ d[t:]) / n / c0
    return rho


def tau_int(x, c=6.0):
    """(tau_int, window) with the automatic window W = min{W : W >= c tau_int(W)}."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        return 0.5, 0
    rho = autocorrelation(x)
    tau = 0.5
    for W in range(1, n):
        tau += rho[W]
        if W >= c * tau:
            return float(tau), W
    return float(tau), n - 1


def effective_samples(x, c=6.0):
    t, _ = tau_int(x, c)
    return len(x) / (2.0 * max(t, 0.5))
