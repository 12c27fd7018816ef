"""saa_cholesky (the factor C, C C' = Sigma, of the normal law in Sec. 3.1)
against the oracle's row-by-row factor: sizes on and off the 32-wide block
boundary, in place, the upper triangle not read, indefinite input flagged
on the device; and the prologue's check of a problem's Cholesky diagonal."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, est_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", [1, 5, 31, 32, 33, 64, 100, 257, 1024])
def test_cholesky_matches_oracle(d):
    from paper_2404_11631_gb300 import saa
    S = inputs.instance(d, seed=d).sigma
    C = saa.saa_cholesky(torch.tensor(S, device="cuda"))
    saa.saa_ctx_sync()
    c = C.cpu().numpy()
    ref = oracle.cholesky(S)
    assert np.max(np.abs(c - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(np.triu(c, 1), np.zeros((d, d)))


def test_cholesky_in_place_and_upper_triangle_ignored():
    from paper_2404_11631_gb300 import saa
    d = 70
    S = inputs.instance(d, seed=1).sigma
    T = torch.tensor(np.tril(S) + np.triu(np.full((d, d), 7.0), 1), device="cuda")
    out = saa.saa_cholesky(T, out=T)
    saa.saa_ctx_sync()
    assert out.data_ptr() == T.data_ptr()
    assert np.max(np.abs(T.cpu().numpy() - oracle.cholesky(S))) <= 1e-12 * np.max(np.abs(S))


def test_cholesky_is_deterministic():
    from paper_2404_11631_gb300 import saa
    S = torch.tensor(inputs.instance(300, seed=2).sigma, device="cuda")
    a, b = saa.saa_cholesky(S), saa.saa_cholesky(S)
    saa.saa_ctx_sync()
    assert torch.equal(a, b)


def test_indefinite_sigma_is_flagged_and_context_survives():
    from paper_2404_11631_gb300 import saa
    S = torch.tensor(np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]]), device="cuda")
    saa.saa_cholesky(S)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()   # cleared
    C = saa.saa_cholesky(torch.eye(4, dtype=torch.float64, device="cuda") * 4.0)
    saa.saa_ctx_sync()
    assert torch.equal(C, torch.eye(4, dtype=torch.float64, device="cuda") * 2.0)


def test_problem_from_device_factor_matches_oracle():
    # the estimator on the device-computed factor agrees with the oracle on its own factor
    from paper_2404_11631_gb300 import saa
    d, N, K = 48, 20_000, 3
    inst = inputs.instance(d, seed=5)
    C = saa.saa_cholesky(torch.tensor(inst.sigma, device="cuda"))
    mu = torch.tensor(inst.mu, device="cuda")
    gp = saa.Problem(mu=mu, chol=C, N=N, law=oracle.LAW_MIX, seed=4)
    op = oracle.make_problem(d, N, inst.mu, oracle.cholesky(inst.sigma), law=oracle.LAW_MIX, seed=4)
    X = inputs.decisions(K, d, seed=5)
    out = saa.saa_eval(gp, torch.tensor(X, device="cuda"), "fp64")
    saa.saa_ctx_sync()
    ref = oracle.saa(op, 64, X)
    assert est_err(out["f"].cpu().numpy(), ref["f"], ref["var"], X, inst.mu, 0.5) <= 1e-10


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan")])
def test_prologue_flags_a_bad_cholesky_diagonal(bad):
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(40, 1000)
    ch = gp.chol.clone()
    ch[17, 17] = bad
    gp2 = saa.Problem(mu=gp.mu, chol=ch, N=1000)
    saa.saa_eval(gp2, torch.zeros(2, 40, dtype=torch.float64, device="cuda"), "fp32")
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()
