"""Oracle parity at the shapes of the large workloads, where every CTA runs
many tiles and the long contractions (d = 1024) are exercised:

* Algorithm 1 on d = 1024 Student-t (nu = 4) scenarios regenerated every
  iteration (M = 1), K = 1: teacher-forced steps against the oracle's
  estimate and gradient at the GPU's own iterate, on the FP32 path (the
  1024-thread narrow tile) and the F16X3 tensor path.
* The gradient of Eq. 4 at d = 1024, K = 64 on the tensor paths with
  N = 2^18 (2048 tiles, so each CTA folds G over many tiles): three sampled
  decisions element by element against the oracle.
* The autograd.Function at the tensor precisions: against the oracle's
  gradient and against central differences (h = 1e-3) of the oracle's FP64
  estimate on the same samples, which are exact up to rounding because
  f_hat is quadratic in w.
The reference values all come from the oracle; N is reduced from the
benchmark's 2^22 / 2^20 only as far as the oracle needs to finish in
seconds."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, est_err, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_fw_teacher_forced_d1024_t4(prec):
    from paper_2404_11631_gb300 import saa
    d, N, M = 1024, 1 << 16, 1
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, nu=4, seed=0)
    w = torch.tensor(inputs.fw_start(d), device="cuda")
    for t in range(4):
        out = saa.saa_solve(gp, w, T=1, M=M, t0=t, prec=prec)
        saa.saa_ctx_sync()
        wt = w.cpu().numpy()
        ref = oracle.saa(op, 32, wt, grad=True, epoch=t // M)
        f_gpu = out["f_trace"].cpu().numpy()[0]
        scale = max(abs(ref["f"][0]), 0.5 * ref["var"][0] + abs(wt @ inst.mu))
        assert abs(f_gpu - ref["f"][0]) <= TOL[prec] * scale
        g = ref["grad"][0]
        js, gap, wn = oracle.fw_step(g, wt, t)
        w_next = out["w"].cpu().numpy()
        gamma = 2.0 / (t + 2)
        s_gpu = (w_next - (1 - gamma) * wt) / gamma
        # the GPU's vertex is one of W's vertices, optimal for the oracle's
        # gradient up to the tolerance, and its gap is the oracle's
        nz = np.flatnonzero(np.abs(s_gpu) > 1e-6)
        assert nz.size <= 1 and (nz.size == 0 or abs(s_gpu[nz[0]] - 1.0) <= 1e-6)
        assert s_gpu @ g <= g.min(initial=0.0) + TOL_GRAD[prec] * np.linalg.norm(g)
        assert abs(out["gap_trace"].cpu().numpy()[0] - gap) <= 1e-5 * max(1.0, abs(gap))
        w = out["w"]


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "bf16x3"])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_grad_parity_d1024_t_law(prec, lam):
    from paper_2404_11631_gb300 import saa
    d, N, K = 1024, 3000, 2
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, nu=4, lam=lam, seed=13)
    X = inputs.decisions(K, d, seed=13)
    out = saa.saa_grad(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    ref = oracle.saa(op, 32, X, grad=True)
    assert grad_err(out["grad"].cpu().numpy(), ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(out["f"].cpu().numpy(), ref["f"], ref["var"], X, inst.mu, lam) <= TOL[prec]


@pytest.fixture(scope="module")
def grad_d1024_N256k():
    """The d = 1024, K = 64 gradient workload at N = 2^18, and the oracle's
    estimate and gradient for three of its decisions."""
    d, N, K = 1024, 1 << 18, 64
    gp, op, inst = make(d, N, seed=0)
    X = inputs.decisions(K, d, seed=0)
    pick = [0, 29, 63]
    ref = oracle.saa(op, 32, X[pick], grad=True)
    return gp, X, pick, ref, inst


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_grad_d1024_N256k_K64_sampled_decisions(prec, grad_d1024_N256k):
    from paper_2404_11631_gb300 import saa
    gp, X, pick, ref, inst = grad_d1024_N256k
    out = saa.saa_grad(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    g = out["grad"].cpu().numpy()[pick]
    f = out["f"].cpu().numpy()[pick]
    e_g = grad_err(g, ref["grad"])
    e_f = est_err(f, ref["f"], ref["var"], X[pick], inst.mu, 0.5)
    print(f"{prec} d=1024 N=2^18 K=64: grad {e_g:.2e} f {e_f:.2e}")
    assert e_g <= TOL_GRAD[prec] and e_f <= TOL[prec]
    # element by element: every component within the tolerance of the row's norm
    assert np.max(np.abs(g - ref["grad"]) / np.linalg.norm(ref["grad"], axis=1)[:, None]) <= TOL_GRAD[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_autograd_tensor_precisions_d1024(prec):
    from paper_2404_11631_gb300.autograd import SAAFunction
    d, N, K = 1024, 1 << 14, 4
    gp, op, inst = make(d, N, seed=2)
    Xn = inputs.decisions(K, d, seed=2)
    X = torch.tensor(Xn, device="cuda", requires_grad=True)
    weights = torch.tensor([1.0, 0.5, 2.0, 1.5], dtype=torch.float64, device="cuda")
    (SAAFunction.apply(X, gp, prec) * weights).sum().backward()
    g = X.grad.cpu().numpy() / weights.cpu().numpy()[:, None]
    ref = oracle.saa(op, 32, Xn, grad=True)
    assert grad_err(g, ref["grad"]) <= TOL_GRAD[prec]
    # central differences (h = 1e-3) of the oracle's FP64 estimate on the same samples
    rng = np.random.default_rng(3)
    h = 1e-3
    coords = [(int(rng.integers(K)), int(rng.integers(d))) for _ in range(12)]
    rows = []
    for k, j in coords:
        for sgn in (1.0, -1.0):
            x = Xn[k].copy()
            x[j] += sgn * h
            rows.append(x)
    fr = oracle.saa(op, 32, np.array(rows))["f"]
    for n, (k, j) in enumerate(coords):
        cd = (fr[2 * n] - fr[2 * n + 1]) / (2 * h)
        assert abs(cd - g[k, j]) <= TOL_GRAD[prec] * np.linalg.norm(ref["grad"][k]), (k, j, cd, g[k, j])
