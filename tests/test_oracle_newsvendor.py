"""Pins for the oracle's newsvendor Monte Carlo gradient (Sec. 3.2: the
approximated gradient k_j - v_j + (h_j + v_j) (1/S) sum_s 1{d_j^(s) <= x_j},
normal demands).

The counts are checked by recounting the oracle's exported demand samples
with numpy, and the samples by recomputing Box-Muller with numpy from raw
Philox words of the demand stream.  The estimator is checked against the
closed-form gradient k_j - v_j + (h_j + v_j) Phi((x_j - mu_j) / sigma_j) of
the same section (binomial z-scores over many products), and against its
limits x << mu and x >> mu."""
import numpy as np
from scipy import stats

import oracle


def _nv(n, S, seed=3, instance=5, epoch=1):
    rng = np.random.default_rng([n, S, 11])
    mu = rng.uniform(20.0, 50.0, n)          # Sec. 4.1's demand setup
    sigma = rng.uniform(10.0, 20.0, n)
    k = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.1, 1.0, n)
    v = rng.uniform(1.0, 4.0, n)
    return oracle.make_newsvendor(mu, sigma, k, h, v, S, seed=seed, instance=instance, epoch=epoch), (mu, sigma, k,
                                                                                                        h, v)


def _words(seed, block, i, epoch, tag, instance):
    ctr = np.stack([block, i, np.full_like(i, epoch), np.full_like(i, (tag << 24) | instance)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    return oracle.philox(ctr.astype(np.uint32), key).astype(np.uint64)


def test_demand_samples_are_box_muller_of_the_demand_stream():
    P, par = _nv(4, 1001)
    j = 2
    z = oracle.newsvendor_demands(P, j)
    b = np.arange((1001 + 3) // 4, dtype=np.uint32)
    x = _words(3, b, np.full_like(b, j), 1, 3, 5)
    u = (2 * (x >> np.uint64(9)) + 1).astype(np.float64) * 2.0 ** -24
    r01 = np.sqrt(-2 * np.log(u[:, 0]))
    r23 = np.sqrt(-2 * np.log(u[:, 2]))
    ref = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r01 * np.sin(2 * np.pi * u[:, 1]),
                    r23 * np.cos(2 * np.pi * u[:, 3]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1).ravel()[:1001]
    assert np.abs(z - ref).max() <= 8 * 2.0 ** -24 * max(1.0, np.abs(ref).max())
    # a different tag from the estimator's normals: not the scenario stream
    x0 = _words(3, b, np.full_like(b, j), 1, 0, 5)
    assert not np.array_equal(x, x0)


def test_counts_recount_the_exported_samples():
    n, S = 37, 513
    P, (mu, sigma, k, h, v) = _nv(n, S)
    rng = np.random.default_rng(2)
    X = np.stack([mu + sigma * rng.normal(size=n), mu - 0.3 * sigma, mu + 1.7 * sigma])
    g, cnt = oracle.newsvendor_grad(P, X)
    for j in range(n):
        z = oracle.newsvendor_demands(P, j)
        for kk in range(3):
            tau = np.float32((X[kk, j] - mu[j]) / sigma[j])
            assert cnt[kk, j] == int(np.sum(z <= tau)), (kk, j)
            assert g[kk, j] == (k[j] - v[j]) + (h[j] + v[j]) * (cnt[kk, j] / S)


def test_matches_the_closed_form_gradient_in_distribution():
    # the count is binomial(S, Phi(tau)): z-scores over products are N(0, 1)
    n, S = 4000, 2000
    P, (mu, sigma, k, h, v) = _nv(n, S, seed=7)
    rng = np.random.default_rng(3)
    X = mu + sigma * rng.uniform(-2.0, 2.0, n)
    g, cnt = oracle.newsvendor_grad(P, X)
    p = stats.norm.cdf(((X - mu) / sigma).astype(np.float32).astype(np.float64))
    zs = (cnt[0] - S * p) / np.sqrt(S * p * (1 - p))
    assert abs(zs.mean()) < 5 / np.sqrt(n) and abs(zs.std() - 1.0) < 0.05
    assert stats.kstest(zs, "norm").pvalue > 1e-4
    exact = k - v + (h + v) * stats.norm.cdf((X - mu) / sigma)
    sd = (h + v) * np.sqrt(p * (1 - p) / S)
    assert np.all(np.abs(g[0] - exact) <= 6 * sd + 1e-12)


def test_limits_and_reproducibility():
    n, S = 50, 400
    P, (mu, sigma, k, h, v) = _nv(n, S)
    g, cnt = oracle.newsvendor_grad(P, np.stack([mu - 40 * sigma, mu + 40 * sigma]))
    assert np.all(cnt[0] == 0) and np.all(cnt[1] == S)
    assert np.array_equal(g[0], k - v) and np.array_equal(g[1], (k - v) + (h + v))
    g2, _ = oracle.newsvendor_grad(P, np.stack([mu - 40 * sigma, mu + 40 * sigma]))
    assert np.array_equal(g, g2)
    # another epoch resamples the demands
    P2, _ = _nv(n, S, epoch=2)
    assert not np.array_equal(oracle.newsvendor_demands(P, 0), oracle.newsvendor_demands(P2, 0))
