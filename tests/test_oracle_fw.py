"""Pins for the oracle's Frank-Wolfe loop (Algorithm 1) and the RSE of
Table 2's notes.

The LMO over W = {w >= 0, 1'w <= 1} is checked by brute force over the
vertices of W, the step schedule gamma_t = 2/(t+2) by its first steps, the
loop by feasibility, by bitwise resume, and by convergence to the optimum of
Eq. 3 found by scipy's SLSQP on the exact (Sigma, mu).
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2404_11631_gb300 import inputs


def test_lmo_and_step_brute_force():
    rng = np.random.default_rng(0)
    for trial in range(200):
        d = int(rng.integers(1, 9))
        g = rng.normal(size=d)
        if trial % 5 == 0:
            g = np.abs(g)            # all-positive gradient: zero vertex
        if trial % 7 == 0 and d > 1:
            g[1] = g.min()           # tie: first index wins
        w = rng.dirichlet(np.ones(d + 1))[:d]
        t = int(rng.integers(0, 50))
        js, gap, wn = oracle.fw_step(g, w, t)
        verts = [np.zeros(d)] + [np.eye(d)[j] for j in range(d)]
        vals = [v @ g for v in verts]
        best = min(vals)
        s = verts[vals.index(best)]
        assert (js == -1 and best == 0.0 and np.all(g >= 0)) or (js >= 0 and np.array_equal(s, np.eye(d)[js]))
        assert np.isclose(gap, g @ w - best, rtol=1e-14, atol=1e-15)
        assert gap >= 0
        gamma = 2.0 / (t + 2)
        assert np.allclose(wn, w + gamma * (s - w), rtol=1e-15, atol=1e-16)
        assert np.all(wn >= 0) and wn.sum() <= 1 + 1e-12


def test_first_step_takes_the_vertex():
    g = np.array([0.3, -0.2, -0.5, 0.1])
    js, gap, wn = oracle.fw_step(g, np.full(4, 0.1), 0)
    assert js == 2 and np.array_equal(wn, np.eye(4)[2])


def _problem(d, N, law=oracle.LAW_GAUSS, seed=0):
    inst = inputs.instance(d, seed=0)
    return oracle.make_problem(d, N, inst.mu, inst.chol, law=law, seed=seed), inst


def test_iterates_stay_feasible_and_resume_is_bitwise():
    d, N, M = 6, 2000, 3
    prob, inst = _problem(d, N)
    w0 = inputs.fw_start(d)
    full = oracle.fw(prob, 32, w0, T=10, M=M, want_w_trace=True)
    assert np.all(full["w_trace"] >= 0) and np.all(full["w_trace"].sum(1) <= 1 + 1e-12)
    assert np.all(full["gap_trace"] >= 0)
    first = oracle.fw(prob, 32, w0, T=4, M=M)
    rest = oracle.fw(prob, 32, first["w"], T=6, M=M, t0=4)
    assert np.array_equal(rest["w"], full["w"])
    assert np.array_equal(np.concatenate([first["f_trace"], rest["f_trace"]]), full["f_trace"])


def test_resampling_every_M_iterations():
    d, N = 4, 500
    prob, inst = _problem(d, N)
    w = inputs.fw_start(d)
    tr = oracle.fw(prob, 64, w, T=6, M=3, want_w_trace=True)
    # iterations 0..2 use resample index 0, iterations 3..5 index 1
    for it in range(6):
        f = oracle.saa(prob, 64, tr["w_trace"][it], epoch=it // 3)["f"][0]
        assert f == tr["f_trace"][it]


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_STUDENT_T])
def test_converges_to_the_qp_optimum(law):
    d, N = 8, 20_000
    prob, inst = _problem(d, N, law=law)
    scale = 2.0 if law == oracle.LAW_STUDENT_T else 1.0   # Cov of the t law (nu = 4)
    S, mu = scale * inst.sigma, inst.mu

    def f(w):
        return 0.5 * w @ S @ w - mu @ w

    res = minimize(f, np.full(d, 0.5 / d), jac=lambda w: S @ w - mu, method="SLSQP",
                   bounds=[(0, None)] * d, constraints=[{"type": "ineq", "fun": lambda w: 1 - w.sum()}],
                   options={"ftol": 1e-14, "maxiter": 500})
    fstar = res.fun
    out = oracle.fw(prob, 64, inputs.fw_start(d), T=300, M=25)
    assert f(out["w"]) - fstar < 2e-2 * abs(fstar) + 1e-3
    assert f(out["w"]) >= fstar - 1e-9


def test_rse_definition():
    assert oracle.rse(2.0, 1.0) == 25.0
    assert oracle.rse(-4.0, -3.0) == 6.25
    assert oracle.rse(1.5, 1.5) == 0.0
