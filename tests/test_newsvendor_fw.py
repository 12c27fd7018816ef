"""Algorithm 2 (Frank-Wolfe for the newsvendor of Sec. 3.2) on the host:
the linear subproblem against brute-force vertex enumeration, and the whole
loop, driven by the oracle's Monte Carlo gradient, against the optimum of
the closed-form expected cost (normal demand) found by scipy."""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.stats import norm

import oracle
from paper_2404_11631_gb300.newsvendor_fw import lmo, newsvendor_fw


def _vertices(A, C):
    # vertices of {s : A s <= C, s >= 0}: n active constraints out of R + n
    R, n = A.shape
    G = np.vstack([A, -np.eye(n)])
    hvec = np.concatenate([C, np.zeros(n)])
    out = []
    for rows in itertools.combinations(range(R + n), n):
        Gs = G[list(rows)]
        if abs(np.linalg.det(Gs)) < 1e-12:
            continue
        v = np.linalg.solve(Gs, hvec[list(rows)])
        if np.all(G @ v <= hvec + 1e-9):
            out.append(v)
    return out


@pytest.mark.parametrize("R,n,seed", [(1, 6, 0), (1, 6, 1), (2, 4, 2), (2, 5, 3), (3, 5, 4)])
def test_lmo_against_vertex_enumeration(R, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.5, 1.5, (R, n))
    C = rng.uniform(1.0, 3.0, R)
    for _ in range(5):
        g = rng.standard_normal(n)
        s = lmo(g, A, C)
        assert np.all(A @ s <= C + 1e-9) and np.all(s >= -1e-12)
        best = min(float(g @ v) for v in _vertices(A, C))
        assert float(g @ s) <= best + 1e-9


def _cost(x, mu, sigma, k, h, v):
    z = (x - mu) / sigma
    over = (x - mu) * norm.cdf(z) + sigma * norm.pdf(z)         # E[(x - d)+]
    under = (mu - x) * norm.sf(z) + sigma * norm.pdf(z)         # E[(d - x)+]
    return float(np.sum(k * x + h * over + v * under))


def test_algorithm_2_reaches_the_optimum():
    rng = np.random.default_rng(7)
    n, S = 20, 4000
    mu, sigma = rng.uniform(20, 50, n), rng.uniform(10, 20, n)
    k, h, v = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n), rng.uniform(1.0, 4.0, n)
    A = rng.uniform(0.5, 1.5, (1, n))
    C = np.array([0.5 * float(A[0] @ mu)])   # the budget binds: half the mean demand's worth

    def grad(x, epoch):
        g, _ = oracle.newsvendor_grad(oracle.make_newsvendor(mu, sigma, k, h, v, S, seed=3, epoch=epoch), x)
        return g[0]

    out = newsvendor_fw(grad, A, C, np.zeros(n), epochs=20, M=10)
    assert np.all(out["gap_trace"] >= -1e-9)
    x = out["x"]
    assert float(A[0] @ x) <= C[0] + 1e-9 and np.all(x >= 0)
    cons = [{"type": "ineq", "fun": lambda y: C[0] - A[0] @ y}]
    res = minimize(lambda y: _cost(y, mu, sigma, k, h, v), np.full(n, 0.1), method="SLSQP",
                   jac=lambda y: k - v + (h + v) * norm.cdf((y - mu) / sigma),
                   bounds=[(0, None)] * n, constraints=cons, options={"ftol": 1e-12, "maxiter": 500})
    f_star, f = res.fun, _cost(x, mu, sigma, k, h, v)
    assert f >= f_star - 1e-6 and (f - f_star) <= 2e-2 * abs(f_star)


def test_lmo_edge_cases():
    A, C = np.array([[1.0, 2.0, 4.0]]), np.array([8.0])
    assert np.array_equal(lmo(np.array([0.0, 1.0, 2.0]), A, C), np.zeros(3))     # nothing pays: s = 0
    # the best cost per unit of resource: -1/1 vs -3/2 vs -4/4 -> product 1, at C / a_1
    assert np.array_equal(lmo(np.array([-1.0, -3.0, -4.0]), A, C), np.array([0.0, 4.0, 0.0]))
    # equal ratios: the first index
    assert np.array_equal(lmo(np.array([-1.0, -2.0, -4.0]), A, C), np.array([8.0, 0.0, 0.0]))
