"""Pins for the oracle's diagonal-covariance samples (Sigma = diag(sd^2), the
independent assets of Sec. 4.1), which need no d x d factor.

The diagonal branch must reproduce the dense branch given C = diag(sd) bit
for bit (the dense sum adds exact zeros for the off-diagonal terms), for
every law and both sample precisions, in value and gradient; at a dimension
where no dense factor is formed, the sample variance must be unbiased for
w'Sigma w = sum_j sd_j^2 w_j^2 under the Gaussian law (its mean over many
resamples within a few standard errors)."""
import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", [32, 64])
def test_diagonal_branch_is_the_dense_one(law, prec):
    d, N, K = 37, 3000, 3
    mu, sd = inputs.paper_assets(d, 1)
    dense = oracle.make_problem(d, N, mu, np.diag(sd), law=law, seed=5)
    diag = oracle.make_problem(d, N, mu, None, law=law, seed=5, sd=sd)
    W = inputs.decisions(K, d, seed=2)
    a = oracle.saa(dense, prec, W, grad=True)
    b = oracle.saa(diag, prec, W, grad=True)
    for key in ("f", "pbar", "var", "grad"):
        assert np.array_equal(a[key], b[key]), key
    fa = oracle.fw(dense, prec, inputs.fw_start(d), T=6, M=2)
    fb = oracle.fw(diag, prec, inputs.fw_start(d), T=6, M=2)
    assert np.array_equal(fa["w"], fb["w"]) and np.array_equal(fa["f_trace"], fb["f_trace"])


def test_large_dimension_variance_is_unbiased():
    d, N, E = 20_000, 64, 60
    mu, sd = inputs.paper_assets(d, 3)
    w = inputs.decisions(1, d, seed=3)[0] / d
    truth = float(np.sum(sd ** 2 * w ** 2))
    v = np.array([oracle.saa(oracle.make_problem(d, N, mu, None, seed=11, epoch=e, sd=sd), 64, w)["var"][0]
                  for e in range(E)])
    # the sample variance of N normals: Var[V] = 2 truth^2 / (N - 1)
    se = truth * np.sqrt(2.0 / (N - 1) / E)
    assert abs(v.mean() - truth) < 5 * se
    with pytest.raises(ValueError):
        oracle.generate(oracle.make_problem(d, N, mu, None, sd=sd), 64, 0, 4, want_xi=True)


def test_gradient_expectation_is_the_closed_form():
    # E[grad f_hat] = 2 lambda Sigma w - mu with Sigma = diag(sd^2): the sample
    # covariance is unbiased and R_bar has mean mu; checked per component
    # against the spread of independent resamples (Gaussian law)
    d, N, E, lam = 200, 400, 120, 0.5
    rng = np.random.default_rng(5)
    mu = rng.uniform(-1.0, 1.0, d)
    sd = rng.uniform(0.5, 1.5, d)
    w = rng.uniform(0.0, 1.0, d) / d
    g = np.array([oracle.saa(oracle.make_problem(d, N, mu, None, lam=lam, seed=7, epoch=e, sd=sd), 64, w,
                             grad=True)["grad"][0] for e in range(E)])
    truth = 2.0 * lam * sd ** 2 * w - mu
    se = g.std(axis=0, ddof=1) / np.sqrt(E)
    assert np.all(np.abs(g.mean(axis=0) - truth) <= 5.0 * se)
    # and the spread is the one the sample mean alone would give (the variance
    # term's noise is of order lambda sd_j sigma_p / sqrt(N), far smaller here)
    assert np.allclose(g.std(axis=0, ddof=1), sd / np.sqrt(N), rtol=0.35)
