"""Pins for the oracle's SAA estimator (Sec. 3.1, Eq. 4 with Eq. 5) and its
gradient in w.

f_hat(w) = lambda (1/(N-1)) sum_i (w'(R_i - R_bar))^2 - w'R_bar estimates the
mean-variance objective of Eq. 3, f(w) = (1/2) w'Sigma w - w'mu (lambda = 1/2;
Eq. 4 as printed has lambda = 1).  The pins: numpy's sample variance and
covariance (library routines), exact rational arithmetic on a discrete law
enumerated with multiplicities, the closed-form expectation under the
Gaussian, lognormal and t laws with z-score bounds, the 1/sqrt(N) rate of the
sample mean, and central differences of the quadratic f_hat.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs


@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_d1_matches_numpy_var_and_mean(lam):
    R = np.random.default_rng(0).normal(0.3, 2.0, size=(5000, 1))
    w = 0.7
    out = oracle.saa_explicit(R, [[w]], lam=lam, grad=True)
    assert np.isclose(out["var"][0], w * w * np.var(R[:, 0], ddof=1), rtol=1e-13)
    assert np.isclose(out["pbar"][0], w * R[:, 0].mean(), rtol=1e-13)
    assert np.isclose(out["f"][0], lam * w * w * np.var(R[:, 0], ddof=1) - w * R[:, 0].mean(), rtol=1e-13)
    g = 2 * lam * w * np.var(R[:, 0], ddof=1) - R[:, 0].mean()
    assert np.isclose(out["grad"][0, 0], g, rtol=1e-12)


@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_matches_numpy_sample_covariance(lam):
    rng = np.random.default_rng(1)
    N, d, K = 300, 7, 4
    R = rng.normal(size=(N, d)) @ rng.normal(size=(d, d)) + rng.normal(size=d)
    W = rng.uniform(size=(K, d))
    out = oracle.saa_explicit(R, W, lam=lam, grad=True)
    S = np.cov(R.T, ddof=1)
    Rbar = R.mean(0)
    for k in range(K):
        w = W[k]
        assert np.isclose(out["var"][k], w @ S @ w, rtol=1e-12)
        assert np.isclose(out["pbar"][k], w @ Rbar, rtol=1e-12)
        assert np.isclose(out["f"][k], lam * (w @ S @ w) - w @ Rbar, rtol=1e-12)
        assert np.allclose(out["grad"][k], 2 * lam * S @ w - Rbar, rtol=1e-11, atol=1e-12)


def test_discrete_law_brute_force_exact():
    # A discrete law with rational probabilities c_j / sum(c): the samples list
    # every support point c_j times, so (N-1)/N * V_hat is the law's exact
    # variance of w'R and R_bar its exact mean (rational arithmetic).
    support = [(Fraction(1, 2), Fraction(-3, 4), Fraction(2)), (Fraction(-1), Fraction(1, 8), Fraction(0)),
               (Fraction(3, 2), Fraction(5, 4), Fraction(-1, 2)), (Fraction(0), Fraction(0), Fraction(7, 4))]
    counts = [3, 1, 5, 2]
    w = (Fraction(1, 4), Fraction(1, 2), Fraction(1, 8))
    N = sum(counts)
    p = [Fraction(c, N) for c in counts]
    proj = [sum(wi * ri for wi, ri in zip(w, r)) for r in support]
    mean = sum(pi * x for pi, x in zip(p, proj))
    var = sum(pi * (x - mean) ** 2 for pi, x in zip(p, proj))
    Ebar = [sum(pi * r[j] for pi, r in zip(p, support)) for j in range(3)]
    cov_w = [sum(pi * (r[j] - Ebar[j]) * (x - mean) for pi, r, x in zip(p, support, proj)) for j in range(3)]
    R = np.array([[float(v) for v in r] for r, c in zip(support, counts) for _ in range(c)])
    for lam in (Fraction(1, 2), Fraction(1)):
        out = oracle.saa_explicit(R, [[float(v) for v in w]], lam=float(lam), grad=True)
        f_exact = lam * var * Fraction(N, N - 1) - mean
        assert abs(out["f"][0] - float(f_exact)) < 1e-14
        assert abs(out["var"][0] * (N - 1) / N - float(var)) < 1e-14
        g_exact = [2 * lam * Fraction(N, N - 1) * cv - e for cv, e in zip(cov_w, Ebar)]
        assert np.allclose(out["grad"][0], [float(v) for v in g_exact], atol=1e-14, rtol=0)


def _gauss_problem(d, N, seed, law=oracle.LAW_GAUSS, lam=0.5, inst_seed=0, nu=4):
    inst = inputs.instance(d, seed=inst_seed)
    return oracle.make_problem(d, N, inst.mu, inst.chol, law=law, lam=lam, seed=seed, nu=nu), inst


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_closed_form_expectation_gaussian(prec, lam):
    # E f_hat = lambda x'Sigma x - mu'x exactly (1/(N-1) is unbiased);
    # Var f_hat = x'Sigma x / N + lambda^2 2 (x'Sigma x)^2 / (N-1) for Gaussian R.
    d, N = 10, 10_000
    x = inputs.decisions(1, d, seed=0)[0]
    zs = []
    for seed in range(12):
        prob, inst = _gauss_problem(d, N, seed, lam=lam)
        out = oracle.saa(prob, prec, x, grad=True)
        sp2 = x @ inst.sigma @ x
        f = lam * sp2 - inst.mu @ x
        se = np.sqrt(sp2 / N + lam ** 2 * 2 * sp2 ** 2 / (N - 1))
        zs.append((out["f"][0] - f) / se)
        # gradient: E = 2 lambda Sigma x - mu
        g = 2 * lam * inst.sigma @ x - inst.mu
        Sx = inst.sigma @ x
        se_g = np.sqrt(4 * lam ** 2 * (np.diag(inst.sigma) * sp2 + Sx ** 2) / (N - 1) + np.diag(inst.sigma) / N)
        assert np.all(np.abs(out["grad"][0] - g) < 5 * se_g)
    zs = np.array(zs)
    assert np.all(np.abs(zs) < 5)
    assert abs(zs.mean()) < 5 / np.sqrt(len(zs))


def test_closed_form_expectation_lognormal_and_mixture():
    # standardised lognormal innovations keep mean mu and covariance Sigma
    d, N = 8, 20_000
    x = inputs.decisions(1, d, seed=2)[0]
    for law in (oracle.LAW_LOGN_STD, oracle.LAW_MIX):
        fs = []
        for seed in range(16):
            prob, inst = _gauss_problem(d, N, seed, law=law)
            fs.append(oracle.saa(prob, 32, x)["f"][0])
        f = 0.5 * x @ inst.sigma @ x - inst.mu @ x
        fs = np.array(fs)
        assert abs(fs.mean() - f) < 5 * fs.std(ddof=1) / np.sqrt(len(fs))


def test_closed_form_student_t_mean_term():
    # t law: Cov = nu/(nu-2) Sigma; V_hat has infinite variance at nu = 4,
    # so the z-score bound is applied to the mean term only.
    d, N, nu = 6, 20_000, 4
    x = inputs.decisions(1, d, seed=3)[0]
    vs = []
    for seed in range(12):
        prob, inst = _gauss_problem(d, N, seed, law=oracle.LAW_STUDENT_T, nu=nu)
        out = oracle.saa(prob, 64, x)
        sp2 = nu / (nu - 2) * (x @ inst.sigma @ x)
        assert abs(out["pbar"][0] - inst.mu @ x) < 5 * np.sqrt(sp2 / N)
        vs.append(out["var"][0] / sp2)
    assert 0.8 < np.median(vs) < 1.2


def test_sample_mean_error_decays_as_inverse_sqrt_N():
    d = 4
    x = inputs.decisions(1, d, seed=4)[0]
    Ns = [1 << 10, 1 << 12, 1 << 14, 1 << 16]
    rms = []
    for N in Ns:
        errs = []
        for seed in range(24):
            prob, inst = _gauss_problem(d, N, 100 + seed)
            errs.append(oracle.saa(prob, 32, x)["pbar"][0] - inst.mu @ x)
        rms.append(np.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(Ns), np.log(rms), 1)[0]
    assert -0.65 < slope < -0.35


@pytest.mark.parametrize("prec", [32, 64])
def test_gradient_matches_central_differences(prec):
    # f_hat is quadratic in w on fixed samples, so central differences are
    # exact up to rounding for any step h.
    d, N, h = 6, 3000, 1e-3
    prob, inst = _gauss_problem(d, N, 9, law=oracle.LAW_MIX)
    x = inputs.decisions(1, d, seed=5)[0]
    g = oracle.saa(prob, prec, x, grad=True)["grad"][0]
    E = np.eye(d)
    W = np.concatenate([x + h * E, x - h * E])
    f = oracle.saa(prob, prec, W)["f"]
    cd = (f[:d] - f[d:]) / (2 * h)
    assert np.allclose(g, cd, rtol=1e-8, atol=1e-9)


def test_thread_count_does_not_change_results():
    import os
    import subprocess
    import sys
    code = ("import oracle, numpy as np; from paper_2404_11631_gb300 import inputs;"
            "inst = inputs.instance(5, 0); P = oracle.make_problem(5, 5000, inst.mu, inst.chol, seed=3);"
            "o = oracle.saa(P, 32, inputs.decisions(3, 5, 0), grad=True);"
            "print(np.concatenate([o['f'], o['grad'].ravel()]).tobytes().hex())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for th in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=th, PYTHONPATH=root)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True).stdout)
    assert outs[0] == outs[1]


def test_each_decision_depends_only_on_the_scenarios_and_its_own_w():
    # Eq. 4 for decision w_k involves only the scenarios and w_k, so any
    # subset or order of the K decisions gives the same rows, bit for bit:
    # the property that lets the GPU path run many decisions in chunks.
    d, N = 9, 4000
    prob, inst = _gauss_problem(d, N, 11, law=oracle.LAW_MIX)
    X = inputs.decisions(7, d, seed=4)
    full = oracle.saa(prob, 32, X, grad=True)
    for rows in ([0, 1, 2], [6], [5, 3, 4]):
        part = oracle.saa(prob, 32, X[rows], grad=True)
        for key in ("f", "pbar", "var", "grad"):
            assert np.array_equal(part[key], full[key][rows]), (key, rows)
