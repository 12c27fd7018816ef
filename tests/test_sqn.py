"""Algorithm 3 (SQN) and Algorithm 4 (BFGS inverse-Hessian update) on the
host: the two-loop product equals Algorithm 4's dense H_t times g; the
iteration, driven by the oracle's mini-batch gradient and sub-sampled
Hessian product, lowers the objective F of Sec. 3.3 and uses correction
pairs once past 2L iterations."""
import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs
from paper_2404_11631_gb300.sqn import dense_h, sqn, two_loop


@pytest.mark.parametrize("m", [1, 2, 5, 25])
def test_two_loop_is_algorithm_4(m):
    rng = np.random.default_rng(m)
    n = 12
    A = rng.standard_normal((n, n))
    A = A @ A.T + 0.5 * np.eye(n)   # SPD curvature: s'y > 0 for every pair
    pairs = []
    for _ in range(m):
        s = rng.standard_normal(n)
        pairs.append((s, A @ s))
    g = rng.standard_normal(n)
    assert np.allclose(two_loop(g, pairs), dense_h(pairs) @ g, rtol=1e-10, atol=1e-12)
    # with one pair the update satisfies the secant equation H y = s
    if m == 1:
        s, y = pairs[0]
        assert np.allclose(dense_h(pairs) @ y, s, rtol=1e-12)


def _oracle_callables(op):
    def grad(w, idx):
        return oracle.logistic_eval(op, w[None], idx=idx, want=("F", "grad"))["grad"][0]

    def hvp(w, v, idx):
        return oracle.logistic_eval(op, w[None], V=v[None], idx=idx, want=("F", "hvp"))["hvp"][0]
    return grad, hvp


def test_sqn_lowers_the_objective():
    n, N, L = 100, 3000, 10
    op = oracle.make_logistic(n, N, inputs.logistic_weights(n, 4), seed=4)
    grad, hvp = _oracle_callables(op)
    w0 = np.zeros(n)
    F = lambda w: float(oracle.logistic_eval(op, w[None], want=("F",))["F"][0])
    res = sqn(grad, hvp, w0, N, iters=6 * L, L=L, M=25, beta=2.0, b=50, b_H=600,
              rng=np.random.default_rng(1), trace_every=L)
    assert res.pairs_used >= 3 and res.skipped_pairs == 0
    f = [F(w) for w in res.w_trace]
    assert F(res.w) < 0.8 * F(w0)            # F(0) = log 2
    assert f[-1] < f[1]                      # still descending after the SGD phase


def test_sqn_keeps_the_last_M_pairs_and_skips_flat_curvature():
    n = 6
    calls = {"h": 0}

    def grad(w, idx):
        return w - 1.0   # F = |w - 1|^2 / 2

    def hvp(w, v, idx):
        calls["h"] += 1
        return v if calls["h"] % 3 else 0.0 * v   # every third pair has s'y = 0

    res = sqn(grad, hvp, np.zeros(n), 100, iters=200, L=5, M=4, beta=1.0, rng=np.random.default_rng(0))
    assert res.pairs_used <= 4 and res.skipped_pairs >= 1
    assert np.allclose(res.w, 1.0, atol=5e-2)
