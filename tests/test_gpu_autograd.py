"""The autograd.Function over the adjoint kernel: gradients of sums of
f_hat(w_k) (Eq. 4) against central differences of the GPU's own values on
random coordinates, and against the oracle's gradient.  f_hat is quadratic in
w on fixed samples, so central differences are exact up to rounding for any
step; h = 0.5 keeps the FP32 rounding of f_hat (~1e-7 V) far below the
tolerance."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_GRAD, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autograd_matches_oracle_and_central_differences(prec):
    from paper_2404_11631_gb300.autograd import SAAFunction
    from paper_2404_11631_gb300 import saa
    d, N, K = 40, 20_000, 6
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=5)
    X = torch.tensor(inputs.decisions(K, d, seed=2), device="cuda", requires_grad=True)
    weights = torch.linspace(0.5, 1.5, K, dtype=torch.float64, device="cuda")
    f = SAAFunction.apply(X, gp, prec)
    (f * weights).sum().backward()
    g = X.grad.cpu().numpy()
    ref = oracle.saa(op, 64 if prec == "fp64" else 32, X.detach().cpu().numpy(), grad=True)
    w = weights.cpu().numpy()
    assert grad_err(g / w[:, None], ref["grad"]) <= TOL_GRAD[prec]
    # central differences of the GPU value on 16 random coordinates
    rng = np.random.default_rng(0)
    h = 0.5
    for _ in range(16):
        k, j = int(rng.integers(K)), int(rng.integers(d))
        Xp = X.detach().clone()
        Xm = X.detach().clone()
        Xp[k, j] += h
        Xm[k, j] -= h
        fp = saa.saa_eval(gp, Xp, prec)["f"][k].item()
        fm = saa.saa_eval(gp, Xm, prec)["f"][k].item()
        cd = (fp - fm) / (2 * h)
        assert abs(cd - g[k, j] / w[k]) <= 1e-5 * max(1.0, abs(cd))


def test_autograd_value_only_path_needs_no_gradient():
    from paper_2404_11631_gb300.autograd import saa_objective
    gp, op, inst = make(16, 5000, seed=1)
    x = torch.tensor(inputs.decisions(1, 16, seed=1)[0], device="cuda")
    f = saa_objective(x, gp, "fp32")
    assert f.shape == () and not f.requires_grad


def test_autograd_full_size_adjoint_d1024_N1M_K64():
    # adjoint-gradient workload: d = 1024, N = 2^20 Gaussian, K = 64, FP32;
    # central differences on 16 random coordinates
    from paper_2404_11631_gb300.autograd import SAAFunction
    from paper_2404_11631_gb300 import saa
    d, N, K = 1024, 1 << 20, 64
    gp, op, inst = make(d, N, seed=0)
    X = torch.tensor(inputs.decisions(K, d, seed=0), device="cuda", requires_grad=True)
    SAAFunction.apply(X, gp, "fp32").sum().backward()
    g = X.grad.cpu().numpy()
    rng = np.random.default_rng(1)
    h = 0.5
    for _ in range(16):
        k, j = int(rng.integers(K)), int(rng.integers(d))
        Xp = X.detach()[k:k + 1].clone()
        Xm = Xp.clone()
        Xp[0, j] += h
        Xm[0, j] -= h
        cd = (saa.saa_eval(gp, Xp, "fp32")["f"].item() - saa.saa_eval(gp, Xm, "fp32")["f"].item()) / (2 * h)
        assert abs(cd - g[k, j]) <= 1e-5 * max(1.0, abs(cd))
