"""Pins of the oracle's scenario-range partial sums (the sums over i of
Eq. 4 / Eq. 5, Sec. 3.1, split by scenario) and of the estimate finalized
from their totals:

* brute force: P1..P4 of a small range equal numpy sums written out from the
  oracle's own FP64 samples R_i (saa_generate's xi), centred at mu;
* additivity: the partials of a split of [0, N) add up to those of [0, N);
* the finalize of the whole sample's partials equals the oracle's direct
  two-pass estimator (itself pinned to closed forms, brute force and numpy);
* planted mistakes (P4 read in the wrong index order, a dropped P1) are
  caught.
"""
import numpy as np
import pytest

import oracle
from paper_2404_11631_gb300 import inputs


def _problem(d, N, law=oracle.LAW_MIX, seed=4, lam=0.5):
    ins = inputs.instance(d, 0)
    return oracle.make_problem(d, N, ins.mu, ins.chol, law=law, seed=seed, lam=lam), ins


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
def test_partials_brute_force_from_samples(law):
    d, N, K = 7, 500, 3
    P, ins = _problem(d, N, law=law)
    X = inputs.decisions(K, d, 1)
    i0, n = 123, 250
    part = oracle.partials(P, 64, i0, n, X, grad=True)
    _, _, xi = oracle.generate(P, 64, i0, n, want_xi=True)
    D = xi - ins.mu[None, :]
    p = D @ X.T                                   # [n, K]
    ref = np.concatenate([p.sum(0), (p * p).sum(0), D.sum(0), (D.T @ p).T.ravel()])
    assert np.allclose(part, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("prec", [32, 64])
def test_partials_add_across_ranges(prec):
    d, N, K = 9, 3001, 4
    P, ins = _problem(d, N)
    X = inputs.decisions(K, d, 2)
    whole = oracle.partials(P, prec, 0, N, X, grad=True)
    cuts = [0, 700, 1500, 1501, N]                # includes a one-scenario range across the mixed law's split
    parts = [oracle.partials(P, prec, a, b - a, X, grad=True) for a, b in zip(cuts[:-1], cuts[1:])]
    assert np.allclose(np.sum(parts, axis=0), whole, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("lam", [0.5, 1.0])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_STUDENT_T])
def test_finalize_of_totals_equals_direct_estimator(lam, law):
    d, N, K = 12, 4000, 5
    P, ins = _problem(d, N, law=law, lam=lam)
    X = inputs.decisions(K, d, 3)
    tot = oracle.partials(P, 32, 0, 2000, X, grad=True) + oracle.partials(P, 32, 2000, N - 2000, X, grad=True)
    got = oracle.finalize_partials(N, X, ins.mu, lam, tot, grad=True)
    ref = oracle.saa(P, 32, X, grad=True)
    for k in ("f", "pbar", "var"):
        assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-12), k
    assert np.allclose(got["grad"], ref["grad"], rtol=1e-9, atol=1e-11)


def test_planted_mistakes_are_caught():
    d, N, K = 6, 2000, 3
    P, ins = _problem(d, N)
    X = inputs.decisions(K, d, 5)
    tot = oracle.partials(P, 32, 0, N, X, grad=True)
    ref = oracle.saa(P, 32, X, grad=True)
    bad = tot.copy()                              # P4 read with the wrong index order
    bad[2 * K + d:] = tot[2 * K + d:].reshape(K, d)[::-1, ::-1].ravel()
    got = oracle.finalize_partials(N, X, ins.mu, 0.5, bad, grad=True)
    assert not np.allclose(got["grad"], ref["grad"], rtol=1e-6)
    bad = tot.copy()                              # P1 dropped: the centring term vanishes
    bad[:K] = 0.0
    got = oracle.finalize_partials(N, X, ins.mu, 0.5, bad, grad=True)
    assert not np.allclose(got["grad"], ref["grad"], rtol=1e-6) or not np.allclose(got["pbar"], ref["pbar"])
