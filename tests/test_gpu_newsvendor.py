"""saa_newsvendor_grad (Sec. 3.2's Monte Carlo gradient of the newsvendor
cost) against the oracle: the counts are exact integers, so counts and
gradient estimates must be bit-identical.  Shapes cover one product and one
sample, sample counts that are not multiples of 4, several decisions, few
products with many samples and the n = 10^6, S = 1000 workload (exact on
sampled product ranges, and in distribution against the closed-form
gradient)."""
import numpy as np
import pytest
import torch
from scipy import stats

import oracle

pytestmark = pytest.mark.gpu


def _problem(n, S, seed=3, instance=5, epoch=1):
    from paper_2404_11631_gb300 import saa
    rng = np.random.default_rng([n, S, 11])
    arrs = dict(mu=rng.uniform(20.0, 50.0, n), sigma=rng.uniform(10.0, 20.0, n), k=rng.uniform(0.5, 2.0, n),
                h=rng.uniform(0.1, 1.0, n), v=rng.uniform(1.0, 4.0, n))
    gp = saa.Newsvendor(**{a: torch.tensor(x, device="cuda") for a, x in arrs.items()}, S=S, seed=seed,
                        instance=instance, epoch=epoch)
    op = oracle.make_newsvendor(arrs["mu"], arrs["sigma"], arrs["k"], arrs["h"], arrs["v"], S, seed=seed,
                                instance=instance, epoch=epoch)
    return gp, op, arrs


def _decisions(arrs, K, seed=0):
    rng = np.random.default_rng(seed)
    n = arrs["mu"].shape[0]
    return arrs["mu"] + arrs["sigma"] * rng.uniform(-3.0, 3.0, (K, n))


@pytest.mark.parametrize("n,S,K", [(1, 1, 1), (37, 513, 3), (1000, 97, 8), (5000, 2048, 2), (100, 100_003, 1)])
def test_newsvendor_bit_exact(n, S, K):
    from paper_2404_11631_gb300 import saa
    gp, op, arrs = _problem(n, S)
    X = _decisions(arrs, K)
    g, cnt = saa.saa_newsvendor_grad(gp, torch.tensor(X, device="cuda"), return_counts=True)
    saa.saa_ctx_sync()
    rg, rc = oracle.newsvendor_grad(op, X)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), rc)
    assert np.array_equal(g.cpu().numpy(), rg)


def test_newsvendor_full_size_sampled_ranges_and_law():
    # n = 10^6 products (Sec. 4.1's largest inventory), S = 1000 samples each
    from paper_2404_11631_gb300 import saa
    n, S = 1_000_000, 1000
    gp, op, arrs = _problem(n, S, seed=0)
    X = _decisions(arrs, 1, seed=1)
    g, cnt = saa.saa_newsvendor_grad(gp, torch.tensor(X, device="cuda"), return_counts=True)
    saa.saa_ctx_sync()
    g, cnt = g.cpu().numpy(), cnt.cpu().numpy().astype(np.int64)
    for j0, j1 in ((0, 300), (499_950, 500_050), (999_800, 1_000_000)):
        rg, rc = oracle.newsvendor_grad(op, X, products=(j0, j1))
        assert np.array_equal(cnt[:, j0:j1], rc) and np.array_equal(g[:, j0:j1], rg)
    tau = ((X[0] - arrs["mu"]) / arrs["sigma"]).astype(np.float32).astype(np.float64)
    p = stats.norm.cdf(tau)
    ok = (p > 1e-3) & (p < 1 - 1e-3)
    zs = (cnt[0, ok] - S * p[ok]) / np.sqrt(S * p[ok] * (1 - p[ok]))
    assert abs(zs.mean()) < 5 / np.sqrt(ok.sum()) and abs(zs.std() - 1.0) < 0.01


def test_newsvendor_deterministic_and_checked():
    from paper_2404_11631_gb300 import saa
    gp, op, arrs = _problem(20_000, 300)
    X = torch.tensor(_decisions(arrs, 4), device="cuda")
    a = saa.saa_newsvendor_grad(gp, X)
    b = saa.saa_newsvendor_grad(gp, X)
    saa.saa_ctx_sync()
    assert torch.equal(a, b)
    bad = saa.Newsvendor(mu=gp.mu, sigma=gp.sigma.clone(), k=gp.k, h=gp.h, v=gp.v, S=300)
    bad.sigma[7] = 0.0
    saa.saa_newsvendor_grad(bad, X)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()
    with pytest.raises(saa.SAAError):
        saa.saa_newsvendor_grad(gp, torch.zeros(9, gp.n, dtype=torch.float64, device="cuda"))
