"""Parity of the CUDA estimator (Eq. 4, Eq. 5 and the gradient of Eq. 4 in w)
with the CPU oracle on identical seeded samples.  Sizes span several tiles
with ragged ends; the full-size d=128, N=2^20, K=256 workload is checked on
sampled decisions."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, ORACLE_PREC, est_err, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(prec, d, N, K, law=oracle.LAW_GAUSS, lam=0.5, grad=False, seed=3, xseed=0, nu=4):
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(d, N, law=law, lam=lam, seed=seed, nu=nu)
    X = inputs.decisions(K, d, seed=xseed)
    Xt = torch.tensor(X, device="cuda")
    if grad:
        out = saa.saa_grad(gp, Xt, prec)
    else:
        out = saa.saa_eval(gp, Xt, prec)
    ref = oracle.saa(op, ORACLE_PREC[prec], X, grad=grad)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref, X, inst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plain_d10_fp64_workload(prec):
    # d = 10, N = 10,000 Gaussian scenarios, K = 1 decision, seed 0
    out, ref, X, inst = _run(prec, 10, 10_000, 1, seed=0)
    e = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    assert e <= TOL[prec]
    assert est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    assert np.max(np.abs(out["var"] - ref["var"]) / ref["var"]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,N,K", [(1, 2, 1), (5, 1000, 3), (33, 4099, 65), (128, 20_000, 130), (300, 3001, 7),
                                   (1024, 2000, 2)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
def test_value_parity(prec, d, N, K, law):
    out, ref, X, inst = _run(prec, d, N, K, law=law)
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    assert est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    assert np.max(np.abs(out["var"] - ref["var"]) / ref["var"]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,N,K", [(1, 3, 1), (10, 10_000, 1), (33, 4099, 65), (200, 5000, 3), (1024, 1500, 2)])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_grad_parity(prec, d, N, K, lam):
    out, ref, X, inst = _run(prec, d, N, K, law=oracle.LAW_MIX, lam=lam, grad=True)
    assert grad_err(out["grad"], ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, lam) <= TOL[prec]


def test_gradient_matches_central_differences_on_gpu():
    # f_hat is quadratic in w on fixed samples: central differences of the
    # GPU's own f_hat reproduce its gradient up to rounding (FP64 path).
    from paper_2404_11631_gb300 import saa
    d, N, h = 12, 5000, 1e-3
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, seed=11)
    x = inputs.decisions(1, d, seed=4)[0]
    g = saa.saa_grad(gp, torch.tensor(x[None], device="cuda"), "fp64")["grad"].cpu().numpy()[0]
    E = np.eye(d)
    W = torch.tensor(np.concatenate([x + h * E, x - h * E]), device="cuda")
    f = saa.saa_eval(gp, W, "fp64")["f"].cpu().numpy()
    assert np.allclose(g, (f[:d] - f[d:]) / (2 * h), rtol=1e-7, atol=1e-9)


def test_results_are_bitwise_deterministic():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(64, 50_000, law=oracle.LAW_MIX, seed=9)
    X = torch.tensor(inputs.decisions(70, 64, seed=1), device="cuda")
    a = [saa.saa_grad(gp, X, "fp32") for _ in range(3)]
    for r in a[1:]:
        assert torch.equal(r["grad"], a[0]["grad"]) and torch.equal(r["f"], a[0]["f"])


def test_full_size_d128_N1M_K256_sampled_decisions():
    # the launch configuration of the d=128, N=2^20, K=256 benchmark workload
    from paper_2404_11631_gb300 import saa
    d, N, K = 128, 1 << 20, 256
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=0)
    X = inputs.decisions(K, d, seed=0)
    out = saa.saa_eval(gp, torch.tensor(X, device="cuda"), "fp32")
    pick = [0, 97, 255]
    ref = oracle.saa(op, 32, X[pick])
    f = out["f"].cpu().numpy()[pick]
    assert est_err(f, ref["f"], ref["var"], X[pick], inst.mu, 0.5) <= TOL["fp32"]
