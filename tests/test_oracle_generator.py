"""Pins for the oracle's scenario generator.

Sec. 3.1 draws i.i.d. samples R_i ~ N(mu, Sigma) and resamples them every M
iterations of Algorithm 1.  The generator forms R_i = mu + s_i C zhat_i from
counter-based Philox draws.  These tests tie every step to something outside
the oracle: numpy's log/cos/sin/exp for the Box-Muller and law transforms,
scipy's normal and chi-square CDFs for the distributions, and the sample
covariance for the Cholesky factor's orientation.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2404_11631_gb300 import inputs


def _prob(d=8, N=1 << 12, law=oracle.LAW_GAUSS, nu=4, seed=5, instance=3, epoch=2):
    inst = inputs.instance(d, seed=1)
    return oracle.make_problem(d, N, inst.mu, inst.chol, law=law, nu=nu, seed=seed, instance=instance,
                               epoch=epoch), inst


def _words(seed, block, i, epoch, tag, instance):
    ctr = np.stack([block, i, np.full_like(i, epoch), np.full_like(i, (tag << 24) | instance)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    return oracle.philox(ctr.astype(np.uint32), key).astype(np.uint64)


def test_box_muller_wiring_f32():
    (P, _), inst = _prob(d=7)
    n = 512
    z, s, _ = oracle.generate((P, _), 32, 0, n)
    i = np.arange(n, dtype=np.uint32)
    for b in range(2):  # d = 7 -> blocks 0, 1 (last draw of block 1 discarded)
        x = _words(5, np.full(n, b, np.uint32), i, 2, 0, 3)
        u = (2 * (x >> np.uint64(9)) + 1).astype(np.float64) * 2.0 ** -24
        r01 = np.sqrt(-2 * np.log(u[:, 0]))
        r23 = np.sqrt(-2 * np.log(u[:, 2]))
        ref = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r01 * np.sin(2 * np.pi * u[:, 1]),
                        r23 * np.cos(2 * np.pi * u[:, 3]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1)
        cols = [4 * b + q for q in range(4) if 4 * b + q < 7]
        got = z[:, cols]
        ref = ref[:, :len(cols)]
        assert np.abs(got - ref).max() <= 8 * 2.0 ** -24 * np.maximum(np.abs(ref), 1.0).max()
    assert np.all(s == 1.0)


def test_box_muller_wiring_f64():
    (P, k), inst = _prob(d=5)
    n = 256
    z, s, _ = oracle.generate((P, k), 64, 0, n)
    i = np.arange(n, dtype=np.uint32)
    for b in range(3):
        x = _words(5, np.full(n, b, np.uint32), i, 2, 0, 3)
        v1 = (x[:, 0] << np.uint64(32)) | x[:, 1]
        v2 = (x[:, 2] << np.uint64(32)) | x[:, 3]
        u1 = (2 * (v1 >> np.uint64(12)) + 1).astype(np.float64) * 2.0 ** -53
        u2 = (2 * (v2 >> np.uint64(12)) + 1).astype(np.float64) * 2.0 ** -53
        r = np.sqrt(-2 * np.log(u1))
        ref = np.stack([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)], axis=1)
        cols = [2 * b + q for q in range(2) if 2 * b + q < 5]
        assert np.abs(z[:, cols] - ref[:, :len(cols)]).max() < 1e-14


@pytest.mark.parametrize("prec", [32, 64])
def test_normals_are_standard_normal(prec):
    (P, k), _ = _prob(d=8, N=1 << 16)
    z, _, _ = oracle.generate((P, k), prec, 0, 1 << 16)
    flat = z.ravel()
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    assert abs(flat.mean()) < 5 / np.sqrt(flat.size)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / flat.size)
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(8)).max() < 5 / np.sqrt(z.shape[0])


def test_slices_epochs_and_instances():
    (P, k), _ = _prob(d=6, N=1000)
    z, s, _ = oracle.generate((P, k), 32, 0, 1000)
    z2, s2, _ = oracle.generate((P, k), 32, 137, 200)
    assert np.array_equal(z[137:337], z2)
    ze, _, _ = oracle.generate((P, k), 32, 0, 1000, epoch=3)
    assert not np.any(ze == z)
    (P2, k2), _ = _prob(d=6, N=1000, instance=4)
    zi, _, _ = oracle.generate((P2, k2), 32, 0, 1000)
    assert not np.any(zi == z)


@pytest.mark.parametrize("prec,tol", [(32, 4e-7), (64, 1e-15)])
def test_lognormal_innovations(prec, tol):
    (Pg, kg), _ = _prob(d=8, N=1 << 15, law=oracle.LAW_GAUSS)
    (Pl, kl), _ = _prob(d=8, N=1 << 15, law=oracle.LAW_LOGN_STD)
    zg, _, _ = oracle.generate((Pg, kg), prec, 0, 1 << 15)
    zl, _, _ = oracle.generate((Pl, kl), prec, 0, 1 << 15)
    e = np.e
    ref = (np.exp(zg) - np.sqrt(e)) / np.sqrt(e * e - e)
    assert np.abs(zl - ref).max() <= tol * np.abs(ref).max() * 4
    flat = zl.ravel()
    # mean 0, variance 1, skewness (e+2) sqrt(e-1) of the sigma = 1 lognormal
    assert abs(flat.mean()) < 6 / np.sqrt(flat.size)
    assert abs(flat.var() - 1) < 0.1
    assert 3.0 < stats.skew(flat) < 9.0


@pytest.mark.parametrize("prec", [32, 64])
def test_student_t_scale_is_chi_square(prec):
    nu = 4
    (P, k), _ = _prob(d=4, N=1 << 15, law=oracle.LAW_STUDENT_T, nu=nu)
    _, s, _ = oracle.generate((P, k), prec, 0, 1 << 15)
    W = nu / s ** 2
    assert stats.kstest(W, stats.chi2(nu).cdf).pvalue > 1e-3
    # wiring: W = -2 (log u0 + log u1) from the tag-1 draw of block 0
    n = 64
    i = np.arange(n, dtype=np.uint32)
    x = _words(5, np.zeros(n, np.uint32), i, 2, 1, 3)
    if prec == 32:
        u = (2 * (x >> np.uint64(9)) + 1).astype(np.float64) * 2.0 ** -24
        Wref = -2 * (np.log(u[:, 0]) + np.log(u[:, 1]))
        assert np.allclose(W[:n], Wref, rtol=2e-6)
    else:
        v0 = (x[:, 0] << np.uint64(32)) | x[:, 1]
        v1 = (x[:, 2] << np.uint64(32)) | x[:, 3]
        u0 = (2 * (v0 >> np.uint64(12)) + 1).astype(np.float64) * 2.0 ** -53
        u1 = (2 * (v1 >> np.uint64(12)) + 1).astype(np.float64) * 2.0 ** -53
        assert np.allclose(W[:n], -2 * (np.log(u0) + np.log(u1)), rtol=1e-14)


def test_mixture_halves():
    N = 1001
    (Pm, km), _ = _prob(d=5, N=N, law=oracle.LAW_MIX)
    (Pg, kg), _ = _prob(d=5, N=N, law=oracle.LAW_GAUSS)
    (Pl, kl), _ = _prob(d=5, N=N, law=oracle.LAW_LOGN_STD)
    zm, _, _ = oracle.generate((Pm, km), 32, 0, N)
    zg, _, _ = oracle.generate((Pg, kg), 32, 0, N)
    zl, _, _ = oracle.generate((Pl, kl), 32, 0, N)
    h = N // 2
    assert np.array_equal(zm[:h], zg[:h])
    assert np.array_equal(zm[h:], zl[h:])


@pytest.mark.parametrize("prec", [32, 64])
def test_samples_at_scenario_precision(prec):
    (P, k), inst = _prob(d=9, N=4096, law=oracle.LAW_STUDENT_T)
    z, s, xi = oracle.generate((P, k), prec, 0, 4096, want_xi=True)
    ref = inst.mu[None, :] + s[:, None] * (z @ inst.chol.T)
    tol = 1e-13 if prec == 64 else 2e-6
    assert np.abs(xi - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_sample_covariance_recovers_sigma():
    # orientation of the Cholesky factor: Cov[C z] = C C' = Sigma, not C'C
    d, N = 6, 1 << 17
    (P, k), inst = _prob(d=d, N=N)
    z, s, xi = oracle.generate((P, k), 64, 0, N, want_xi=True)
    S = np.cov(xi.T, ddof=1)
    sd = np.sqrt(np.outer(np.diag(inst.sigma), np.diag(inst.sigma)) + inst.sigma ** 2) / np.sqrt(N)
    assert np.all(np.abs(S - inst.sigma) < 5 * sd)
    assert np.all(np.abs(xi.mean(0) - inst.mu) < 5 * np.sqrt(np.diag(inst.sigma) / N))
    wrong = inst.chol.T @ inst.chol
    assert np.abs(S - wrong).max() > 10 * sd.max()
