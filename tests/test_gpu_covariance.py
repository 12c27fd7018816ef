"""Covariance-first form (saa_moments + saa_eval_moments): the sums
M = sum_i a_i a_i' and mt = sum_i a_i of the whitened samples, formed once on
the tensor cores, then Eq. 4, Eq. 5 and the gradient for any K decisions in
FP64.  Checked against the oracle's plain definition on the same samples
(every law, d up to 128, K up to 256; d = 130 to 1024, where M is formed in
128 x 128 blocks, on two laws), M and mt directly against sums of the
oracle's draws (one slice and three), and against the direct tensor-core
path at the full d = 128, N = 2^20, K = 256 workload."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, est_err, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(d, N, K, law, prec, seed=3, lam=0.5):
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(d, N, law=law, seed=seed, lam=lam)
    X = inputs.decisions(K, d, seed=seed)
    mom = saa.saa_moments(gp, prec)
    out = saa.saa_eval_moments(gp, torch.tensor(X, device="cuda"), mom)
    saa.saa_ctx_sync()
    ref = oracle.saa(op, 32, X, grad=True)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref, X, inst, mom


@pytest.mark.parametrize("d,N,K", [(1, 4099, 1), (7, 5000, 3), (64, 20_000, 32), (100, 9_999, 33), (128, 40_000, 256)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_covariance_first_matches_oracle(d, N, K, law, prec):
    out, ref, X, inst, _ = _run(d, N, K, law, prec)
    e_f = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    e_p = est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5)
    e_g = grad_err(out["grad"], ref["grad"])
    print(f"{prec} d={d} N={N} K={K} law={law}: f {e_f:.2e} pbar {e_p:.2e} grad {e_g:.2e}")
    assert e_f <= TOL[prec] and e_p <= TOL[prec] and e_g <= TOL_GRAD[prec]


@pytest.mark.parametrize("d,N,K", [(130, 5_000, 9), (256, 4_099, 17), (300, 3_000, 33), (1024, 2_500, 64)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_covariance_first_blocked_matches_oracle(d, N, K, law, prec):
    out, ref, X, inst, _ = _run(d, N, K, law, prec)
    e_f = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    e_p = est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5)
    e_g = grad_err(out["grad"], ref["grad"])
    print(f"{prec} d={d} N={N} K={K} law={law}: f {e_f:.2e} pbar {e_p:.2e} grad {e_g:.2e}")
    assert e_f <= TOL[prec] and e_p <= TOL[prec] and e_g <= TOL_GRAD[prec]


@pytest.mark.parametrize("d", [37, 300])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_moments_against_sums_of_oracle_draws(d, prec):
    from paper_2404_11631_gb300 import saa
    N = 3001
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, seed=2)
    mom = saa.saa_moments(gp, prec)
    saa.saa_ctx_sync()
    z, s, _ = oracle.generate(op, 32, 0, N)
    a = (z * s[:, None]).astype(np.float32).astype(np.float64)
    M_ref, m_ref = a.T @ a, a.sum(axis=0)
    M = mom["M"].cpu().numpy()
    # hi/lo operands: 2^-22 (FP16) or 2^-17 (BF16) per product; m~ from FP32 partials of 128 draws
    tol = {"f16x3": 2e-6, "bf16x3": 5e-5}[prec]
    assert np.max(np.abs(M - M_ref)) <= tol * np.max(np.abs(np.diag(M_ref)))
    assert np.max(np.abs(mom["mt"].cpu().numpy() - m_ref)) <= 1e-7 * np.abs(a).sum(axis=0).max()


def test_covariance_first_matches_direct_path_full_size():
    from paper_2404_11631_gb300 import saa
    d, N, K = 128, 1 << 20, 256
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=0)
    X = torch.tensor(inputs.decisions(K, d, seed=0), device="cuda")
    mom = saa.saa_moments(gp, "f16x3")
    a = saa.saa_eval_moments(gp, X, mom)
    b = saa.saa_eval(gp, X, "f16x3")
    c = saa.saa_grad(gp, X[:64].contiguous(), "fp32")
    saa.saa_ctx_sync()
    scale = (0.5 * b["var"] + (X @ gp.mu).abs()).cpu().numpy()
    assert np.max(np.abs((a["f"] - b["f"]).cpu().numpy()) / scale) <= 2e-6
    assert grad_err(a["grad"][:64].cpu().numpy(), c["grad"].cpu().numpy()) <= 2e-6


def test_covariance_first_blocked_matches_direct_path_large():
    # d = 1024 (36 blocks of M over 4 scenario ranges), N = 2^18, against
    # the direct tensor-core value-and-gradient path on the same scenarios
    from paper_2404_11631_gb300 import saa
    d, N, K = 1024, 1 << 18, 8
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=1)
    X = torch.tensor(inputs.decisions(K, d, seed=1), device="cuda")
    mom = saa.saa_moments(gp, "f16x3")
    a = saa.saa_eval_moments(gp, X, mom)
    b = saa.saa_grad(gp, X, "f16x3")
    saa.saa_ctx_sync()
    scale = (0.5 * a["var"] + (X @ gp.mu).abs()).cpu().numpy()
    assert np.max(np.abs((a["f"] - b["f"]).cpu().numpy()) / scale) <= 2e-6
    assert grad_err(a["grad"].cpu().numpy(), b["grad"].cpu().numpy()) <= 2e-6


def test_covariance_first_limits():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(1025, 1000)
    with pytest.raises(saa.SAAError):
        saa.saa_moments(gp, "f16x3")
    gp, op, inst = make(16, 1000)
    with pytest.raises(saa.SAAError):
        saa.saa_moments(gp, "fp32")
