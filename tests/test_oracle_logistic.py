"""Pins for the oracle's binary-classification task (Sec. 3.3; data set of
Sec. 4.1's setup).

Features are recomputed with numpy from raw Philox words (the bit layout),
labels from the integer labelling rule and the noise words (exactly), the
label noise rate against its binomial law.  The objective is pinned at
omega = 0, where c = 1/2 exactly gives F = log 2 and closed forms for the
gradient and the Hessian product; the gradient against central differences
of F and the Hessian product against central differences of the gradient;
the Hessian's symmetry and positive semi-definiteness; the overflow-free
evaluation at large |x'omega|; and the index semantics of the sample S
(repeats weigh as often as they appear)."""
import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs


def _data(n, N, seed=1, instance=0, flip=oracle.LABEL_NOISE_10PCT, wseed=0):
    w = inputs.logistic_weights(n, wseed)
    return oracle.make_logistic(n, N, w, seed=seed, instance=instance, flip=flip), w


def _words(seed, b, i, tag, instance):
    ctr = np.stack([b, i, np.zeros_like(i), np.full_like(i, (tag << 24) | instance)], axis=1).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    return oracle.philox(ctr, key)


def test_features_are_the_philox_bits():
    n, N = 300, 257
    P, w = _data(n, N, seed=12345678901, instance=3)
    x, z = oracle.logistic_data(P)
    nb = (n + 127) // 128
    i = np.repeat(np.arange(N, dtype=np.uint32), nb)
    b = np.tile(np.arange(nb, dtype=np.uint32), N)
    words = _words(12345678901, b, i, 4, 3).reshape(N, nb, 4)
    bits = (words[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1      # [N, nb, 4, 32]
    ref = bits.reshape(N, nb * 128)[:, :n].astype(np.uint8)
    assert np.array_equal(x, ref)
    # Bernoulli(1/2): z-score of the mean over N n features
    assert abs(x.mean() - 0.5) < 5 * 0.5 / np.sqrt(x.size)


def test_labels_follow_the_rule_and_the_noise_words():
    n, N = 64, 20_000
    P, w = _data(n, N, seed=7)
    x, z = oracle.logistic_data(P)
    clean = (2 * (x.astype(np.int64) @ w) > w.sum()).astype(np.uint8)
    noise = _words(7, np.zeros(N, np.uint32), np.arange(N, dtype=np.uint32), 5, 0)[:, 0]
    flips = (noise < oracle.LABEL_NOISE_10PCT).astype(np.uint8)
    assert np.array_equal(z, clean ^ flips)
    rate = flips.mean()
    assert abs(rate - 0.1) < 5 * np.sqrt(0.1 * 0.9 / N)
    # no noise: the labels are the rule itself
    P0, _ = _data(n, N, seed=7, flip=0)
    assert np.array_equal(oracle.logistic_data(P0)[1], clean)


def test_closed_forms_at_zero():
    n, N = 40, 3000
    P, w = _data(n, N, seed=2)
    x, z = oracle.logistic_data(P)
    v = np.random.default_rng(0).normal(size=n)
    out = oracle.logistic_eval(P, np.zeros(n), V=v)
    assert abs(out["F"][0] - np.log(2.0)) < 1e-15
    xf = x.astype(np.float64)
    assert np.allclose(out["grad"][0], (0.5 - z) @ xf / N, rtol=1e-13, atol=1e-16)
    assert np.allclose(out["hvp"][0], 0.25 * ((xf @ v) @ xf) / N, rtol=1e-12, atol=1e-15)


def test_gradient_and_hessian_product_against_differences():
    n, N = 20, 2000
    P, w = _data(n, N, seed=5)
    rng = np.random.default_rng(4)
    om = 0.3 * rng.normal(size=n)
    v = rng.normal(size=n)
    out = oracle.logistic_eval(P, om, V=v)
    h = 1e-5
    fd = np.empty(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        fd[j] = (oracle.logistic_eval(P, om + e)["F"][0] - oracle.logistic_eval(P, om - e)["F"][0]) / (2 * h)
    assert np.linalg.norm(out["grad"][0] - fd) <= 1e-7 * np.linalg.norm(fd)
    gp = oracle.logistic_eval(P, om + h * v)["grad"][0]
    gm = oracle.logistic_eval(P, om - h * v)["grad"][0]
    assert np.linalg.norm(out["hvp"][0] - (gp - gm) / (2 * h)) <= 1e-7 * np.linalg.norm(out["hvp"][0])


def test_hessian_is_symmetric_and_psd():
    n, N = 30, 1500
    P, w = _data(n, N, seed=6)
    rng = np.random.default_rng(1)
    om = 0.2 * rng.normal(size=n)
    u, v = rng.normal(size=n), rng.normal(size=n)
    hu = oracle.logistic_eval(P, np.stack([om, om]), V=np.stack([u, v]))["hvp"]
    assert abs(v @ hu[0] - u @ hu[1]) <= 1e-12 * (abs(v @ hu[0]) + 1e-300)
    assert u @ hu[0] >= 0.0 and v @ hu[1] >= 0.0


def test_large_margins_do_not_overflow():
    n, N = 16, 500
    P, w = _data(n, N, seed=3)
    x, z = oracle.logistic_data(P)
    om = 400.0 * np.sign(w - 0.5)            # |t| in the hundreds: exp(t) overflows a naive evaluation
    out = oracle.logistic_eval(P, om)
    t = x.astype(np.float64) @ om
    ref = np.mean(np.logaddexp(0.0, t) - z * t)   # numpy's overflow-free log(1 + e^t)
    assert np.abs(t).max() >= 400.0
    assert np.isfinite(out["F"][0]) and np.all(np.isfinite(out["grad"]))
    assert abs(out["F"][0] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_sample_indices_weigh_by_multiplicity():
    n, N = 24, 800
    P, w = _data(n, N, seed=8)
    om = np.random.default_rng(2).normal(size=n) * 0.1
    a = oracle.logistic_eval(P, om, idx=[17])
    b = oracle.logistic_eval(P, om, idx=[401])
    ab = oracle.logistic_eval(P, om, idx=[17, 401, 17])
    assert np.isclose(ab["F"][0], (2 * a["F"][0] + b["F"][0]) / 3, rtol=1e-14)
    assert np.allclose(ab["grad"][0], (2 * a["grad"][0] + b["grad"][0]) / 3, rtol=1e-13, atol=1e-16)
    full = oracle.logistic_eval(P, om)
    every = oracle.logistic_eval(P, om, idx=np.arange(N))
    assert np.isclose(full["F"][0], every["F"][0], rtol=1e-14)
    with pytest.raises(ValueError):
        oracle.logistic_eval(P, om, idx=[N])
