"""The exact optimum of the mean-variance problem with independent assets
(used for the RSE figures) against scipy's SLSQP, and the RSE formula
against the oracle's."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2404_11631_gb300 import inputs
from paper_2404_11631_gb300.reporting import diag_optimum, rse


@pytest.mark.parametrize("d,seed,lam", [(5, 0, 0.5), (12, 1, 0.5), (30, 2, 1.0), (8, 3, 20.0)])
def test_diag_optimum_against_slsqp(d, seed, lam):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1, 1, d)
    sd = rng.uniform(0.2, 1.5, d)
    w, f = diag_optimum(mu, sd, lam)
    assert np.all(w >= 0) and w.sum() <= 1 + 1e-12
    fun = lambda y: lam * np.sum(sd ** 2 * y ** 2) - mu @ y
    res = minimize(fun, np.full(d, 0.5 / d), jac=lambda y: 2 * lam * sd ** 2 * y - mu, method="SLSQP",
                   bounds=[(0, None)] * d, constraints=[{"type": "ineq", "fun": lambda y: 1 - y.sum()}],
                   options={"ftol": 1e-15, "maxiter": 1000})
    assert f <= res.fun + 1e-10 and f >= res.fun - 1e-6 * max(1.0, abs(res.fun))


def test_diag_optimum_at_the_paper_scale():
    # Sec. 4.1's assets: the budget binds and the optimum is a valid allocation
    mu, sd = inputs.paper_assets(5000, 0)
    w, f = diag_optimum(mu, sd)
    assert abs(w.sum() - 1.0) < 1e-12 and np.all(w >= 0)
    # optimality: no feasible direction improves (KKT with the budget's multiplier)
    g = 2 * 0.5 * sd ** 2 * w - mu
    nu = -g[w > 0].mean()
    assert np.allclose(g[w > 0], -nu, rtol=0, atol=1e-9) and np.all(g[w == 0] >= -nu - 1e-9)


def test_rse_is_the_oracles():
    f_t = np.array([-0.9, -0.95, -0.99])
    assert np.allclose(rse(f_t, -1.0), [oracle.rse(x, -1.0) for x in f_t])
