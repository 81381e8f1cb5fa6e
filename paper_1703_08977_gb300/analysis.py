"""Post-processing of the space-averaged outputs (host side, on a few numbers).

growth_fit: the paper's estimator of the energy from the growth of z(t).  By
Eq. 4, lambda_1 = lambda_0 - lim (1/t) ln E[exp(-int V_P)]; with z(t) the
space average of the weights, (1/t) ln z(t) is fitted as A + B / t over the
sampled times (the form the printed "ls fit" columns of the result tables
follow) and lambda_1 = lambda_0 - A, with lambda_0 the trial energy E_T.

dt_extrapolate: linear extrapolation of energies at several time steps to
dt -> 0 (the Euler-Maruyama time-step bias is first order in dt).
"""
from __future__ import annotations

import numpy as np


def growth_fit(t, y, sigma=None):
    """Least-squares fit y(t) = A + B / t; sigma (optional) weights the points by
    1 / sigma^2.  Returns (A, B, covariance 2x2 of (A, B) from the weights/residuals)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    X = np.stack([np.ones_like(t), 1.0 / t], axis=1)
    w = np.ones_like(t) if sigma is None else 1.0 / np.asarray(sigma, dtype=np.float64) ** 2
    XtW = X.T * w
    M = XtW @ X
    A, B = np.linalg.solve(M, XtW @ y)
    r = y - X @ np.array([A, B])
    dof = max(len(t) - 2, 1)
    cov = np.linalg.inv(M) * (float(r @ (w * r)) / dof if sigma is None else 1.0)
    return float(A), float(B), cov


def lambda_from_growth(lambda0, t, ln_z, sigma=None):
    """lambda_1 = lambda_0 - A from ln z(t) / t = A + B / t (Eq. 4)."""
    t = np.asarray(t, dtype=np.float64)
    A, B, cov = growth_fit(t, np.asarray(ln_z) / t, sigma)
    return lambda0 - A, float(np.sqrt(cov[0, 0]))


def growth_from_series(e_trial, dt, ln_z, times=(8, 16, 24, 32, 40, 48)):
    """lambda_1 from a gfk_energy ln z series (index k = after k moves of dt) sampled
    at the given times (the paper samples t = 8 ... 48)."""
    ln_z = np.asarray(ln_z)
    idx = [int(round(t / dt)) for t in times]
    if idx[-1] >= len(ln_z):
        raise ValueError("series shorter than the last sampling time")
    return lambda_from_growth(e_trial, np.asarray(times, dtype=np.float64), ln_z[idx])


def dt_extrapolate(dts, energies, errors=None):
    """Weighted linear fit E(dt) = E0 + k dt; returns (E0, its standard error, k)."""
    dts = np.asarray(dts, dtype=np.float64)
    e = np.asarray(energies, dtype=np.float64)
    X = np.stack([np.ones_like(dts), dts], axis=1)
    w = np.ones_like(dts) if errors is None else 1.0 / np.asarray(errors, dtype=np.float64) ** 2
    M = (X.T * w) @ X
    coef = np.linalg.solve(M, (X.T * w) @ e)
    cov = np.linalg.inv(M)
    if errors is None:
        r = e - X @ coef
        cov = cov * float(r @ r) / max(len(e) - 2, 1)
    return float(coef[0]), float(np.sqrt(cov[0, 0])), float(coef[1])


def read_table(path):
    """A golden copy of one of the paper's growth tables: (lambda0, lambda1, rows)."""
    lam = {}
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] in ("lambda0", "lambda1"):
            lam[f[0]] = float(f[1])
        else:
            rows.append([float(v) for v in f])
    return lam["lambda0"], lam["lambda1"], np.array(rows)
