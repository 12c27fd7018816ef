"""Reporting helpers for the accuracy figures of Sec. 4.2 (host side, not
part of the estimator): the exact optimum of the mean-variance problem of
Eq. 3 with independent assets, and the relative squared error of an
iterate's objective value against it.

With Sigma = diag(sd^2) the problem min lambda w'Sigma w - mu'w over
{w >= 0, 1'w <= 1} separates under one multiplier nu >= 0 of the budget:
the KKT conditions give w_j = max(0, (mu_j - nu) / (2 lambda sd_j^2)), with
nu = 0 when that allocation already fits the budget, else the nu at which
it sums to one (a decreasing piecewise-linear function of nu, solved exactly
between its breakpoints).
"""
from __future__ import annotations

import numpy as np


def diag_optimum(mu: np.ndarray, sd: np.ndarray, lam: float = 0.5) -> tuple[np.ndarray, float]:
    """(w*, f*) of min lam w'diag(sd^2)w - mu'w over {w >= 0, 1'w <= 1}."""
    mu = np.asarray(mu, dtype=np.float64)
    c = 1.0 / (2.0 * lam * np.asarray(sd, dtype=np.float64) ** 2)   # w_j = c_j (mu_j - nu)+

    def alloc(nu):
        return c * np.maximum(mu - nu, 0.0)

    w = alloc(0.0)
    if w.sum() > 1.0:
        # sum_j c_j (mu_j - nu)+ = 1: walk the breakpoints mu_j in decreasing order
        order = np.argsort(-mu)
        m, cc = mu[order], c[order]
        csum, cmsum = np.cumsum(cc), np.cumsum(cc * m)
        nu = 0.0
        for i in range(m.size):
            # with the first i + 1 assets active: nu = (sum c_j mu_j - 1) / sum c_j
            cand = (cmsum[i] - 1.0) / csum[i]
            lo = m[i + 1] if i + 1 < m.size else -np.inf
            if lo <= cand <= m[i]:
                nu = cand
                break
        w = alloc(max(nu, 0.0))
    f = float(lam * np.sum(sd ** 2 * w ** 2) - mu @ w)
    return w, f


def rse(f_t, f_star):
    """Relative squared error in percent, ((f_t - f*) / f_t)^2 x 100, the
    paper's form (divided by the iterate's value)."""
    f_t = np.asarray(f_t, dtype=np.float64)
    return ((f_t - f_star) / f_t) ** 2 * 100.0
