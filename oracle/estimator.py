"""Energy estimator over the branching history (FP64).

Sec. II.A: after each reconfiguration the walker weights restart at 1 and the
mean weight wbar_n is kept; the global population factor is
    Gbar_n^p = prod_{j=1..p} wbar_{n-j}          (fewer factors while n < p)
and the energy is E = sum_n Gbar_n^p ebar_n / sum_n Gbar_n^p over the
equilibrated branchings n >= n_equil.  The products are formed in log space
and normalised by their maximum before exponentiation (same value, no overflow).

Error bar (the paper only asks for "appropriate estimators"): block jackknife
of the ratio estimator over consecutive blocks of B branchings, for
B = 1, 2, 4, ... while at least 8 blocks remain; the largest of these errors
is reported (a conservative stand-in for the blocking plateau).
"""
from __future__ import annotations

import numpy as np


def log_gbar(wbar, p):
    wbar = np.asarray(wbar, dtype=np.float64)
    lw = np.log(wbar)
    out = np.zeros(len(wbar))
    for n in range(len(wbar)):
        lo = max(0, n - p)
        out[n] = np.sum(lw[lo:n])
    return out


def energy(wbar, ebar, p, n_equil=0):
    ebar = np.asarray(ebar, dtype=np.float64)
    lg = log_gbar(wbar, p)[n_equil:]
    e = ebar[n_equil:]
    if len(e) == 0:
        return float("nan")
    g = np.exp(lg - lg.max())
    return float(np.sum(g * e) / np.sum(g))


def energy_error(wbar, ebar, p, n_equil=0, min_blocks=8):
    ebar = np.asarray(ebar, dtype=np.float64)
    lg = log_gbar(wbar, p)[n_equil:]
    e = ebar[n_equil:]
    n = len(e)
    if n < 2 * min_blocks:
        return float("nan")
    g = np.exp(lg - lg.max())
    num_all, den_all = np.sum(g * e), np.sum(g)
    best = 0.0
    B = 1
    while n // B >= min_blocks:
        nb = n // B
        num = np.array([np.sum(g[k * B:(k + 1) * B] * e[k * B:(k + 1) * B]) for k in range(nb)])
        den = np.array([np.sum(g[k * B:(k + 1) * B]) for k in range(nb)])
        tn, td = np.sum(num), np.sum(den)
        jk = (tn - num) / (td - den)
        var = (nb - 1) / nb * np.sum((jk - jk.mean()) ** 2)
        best = max(best, float(np.sqrt(var)))
        B *= 2
    del num_all, den_all
    return best


def extrapolate_a(a, E, err, order=1):
    """Lattice-space extrapolation (Sec. II: the LRDMC energy has an O(a^2)
    bias; runs at several a are extrapolated to a -> 0).  Weighted least
    squares for E(a) = sum_{j<=order} c_j a^(2j) with weights 1/err^2, written
    as the ordinary least-squares problem of the rows divided by err and solved
    by numpy's lstsq; the covariance is (X_w^T X_w)^-1.
    Returns (coef, cov, chi2)."""
    a = np.asarray(a, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    err = np.asarray(err, dtype=np.float64)
    X = np.stack([a ** (2 * j) for j in range(order + 1)], axis=1) / err[:, None]
    y = E / err
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    cov = np.linalg.inv(X.T @ X)
    chi2 = float(np.sum((y - X @ coef) ** 2))
    return coef, cov, chi2
