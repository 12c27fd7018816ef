"""Parity of the tcgen05 gradient path (SAA_F16X3, SAA_BF16X3 with the
gradient: forward split-precision contraction, then the adjoint G_k =
sum_i a_i Q_ik on the tensor cores) with the oracle on the same FP32-mode
samples: Eq. 4 with Eq. 5 and its gradient in w (Sec. 3.1), and Algorithm 1
steps driven by it.  Shapes cover one and several 64-dimension forward
blocks and 128-dimension adjoint blocks with ragged last ones, decision
counts that are not multiples of 32, ragged scenario tails and every law.
The d = 1024, N = 2^20, K = 64 workload is checked through properties that
hold at any size: f_hat is quadratic in w on fixed samples, so central
differences of the value reproduce the gradient."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, est_err, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(1, 4099, 1), (7, 5000, 3), (64, 20_000, 32), (100, 9_999, 33), (130, 7_000, 64), (300, 5_001, 17),
          (1024, 3_000, 64), (1000, 2_500, 5)]


def _grad(d, N, K, law=oracle.LAW_GAUSS, seed=3, nu=4, lam=0.5, prec="f16x3"):
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(d, N, law=law, seed=seed, nu=nu, lam=lam)
    X = inputs.decisions(K, d, seed=seed)
    out = saa.saa_grad(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    ref = oracle.saa(op, 32, X, grad=True)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref, X, inst


@pytest.mark.parametrize("d,N,K", SHAPES)
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_grad_parity(d, N, K, law, prec):
    out, ref, X, inst = _grad(d, N, K, law=law, prec=prec)
    e_g = grad_err(out["grad"], ref["grad"])
    e_f = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    print(f"{prec} d={d} N={N} K={K} law={law}: grad {e_g:.2e} f {e_f:.2e}")
    assert e_g <= TOL_GRAD[prec] and e_f <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_tc_grad_lambda(prec, lam):
    out, ref, X, inst = _grad(96, 6_000, 9, law=oracle.LAW_MIX, lam=lam, seed=8, prec=prec)
    assert grad_err(out["grad"], ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, lam) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
@pytest.mark.parametrize("N", [40 * 128 + 5, 76 * 128 - 51, 101 * 128 + 1])
def test_tc_grad_partial_blocks_of_G(prec, N):
    # The adjoint accumulates a block of G over four tiles before each
    # compensated fold.  With 8-CTA clusters at d = 1024 these scenario
    # counts leave each cluster 2 or 3, 5 or 6, and 6 or 7 tiles at 15
    # resident clusters (2 to 8 for 13 to 20 clusters), so the last block is
    # partial, and for 2 or 3 tiles the first block is also the last.
    out, ref, X, inst = _grad(1024, N, 5, law=oracle.LAW_MIX, seed=N % 97, prec=prec)
    assert grad_err(out["grad"], ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_grad_small_N_edge(prec):
    # N = 2 (one partial tile), a tile-exact N = 128 and one row past it
    for N in (2, 128, 129):
        out, ref, X, inst = _grad(20, N, 3, seed=N, prec=prec)
        assert grad_err(out["grad"], ref["grad"]) <= TOL_GRAD[prec] * 10
        assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec] * 10


def test_tc_grad_deterministic():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(200, 40_000, law=oracle.LAW_MIX, seed=9)
    X = torch.tensor(inputs.decisions(40, 200, seed=1), device="cuda")
    a = [saa.saa_grad(gp, X, "f16x3") for _ in range(3)]
    saa.saa_ctx_sync()
    for r in a[1:]:
        assert torch.equal(r["grad"], a[0]["grad"]) and torch.equal(r["f"], a[0]["f"])


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_teacher_forced_fw_steps(prec):
    # Algorithm 1 on the tensor path: each step's f, vertex and gap against
    # the oracle's gradient at the GPU's own iterate
    from paper_2404_11631_gb300 import saa
    d, N, M = 40, 4000, 3
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, seed=21)
    w = torch.tensor(inputs.fw_start(d), device="cuda")
    for t in range(6):
        out = saa.saa_solve(gp, w, T=1, M=M, t0=t, prec=prec)
        saa.saa_ctx_sync()
        wt = w.cpu().numpy()
        ref = oracle.saa(op, 32, wt, grad=True, epoch=t // M)
        f_gpu = out["f_trace"].cpu().numpy()[0]
        assert abs(f_gpu - ref["f"][0]) <= TOL[prec] * max(abs(ref["f"][0]), 0.5 * ref["var"][0] + abs(wt @ inst.mu))
        g = ref["grad"][0]
        js, gap, wn = oracle.fw_step(g, wt, t)
        w_next = out["w"].cpu().numpy()
        s_gpu = (w_next - (1 - 2.0 / (t + 2)) * wt) / (2.0 / (t + 2))
        assert s_gpu @ g <= g.min(initial=0.0) + TOL_GRAD[prec] * np.linalg.norm(g)
        assert abs(out["gap_trace"].cpu().numpy()[0] - gap) <= 1e-4 * max(1.0, abs(gap))
        w = out["w"]


def test_tc_grad_full_size_d1024_N1M_K64():
    # full adjoint workload: agreement with the FP32 path (itself pinned to
    # the oracle) and with central differences of the FP32 value on 12
    # random coordinates (f_hat is quadratic in w on fixed samples)
    from paper_2404_11631_gb300 import saa
    d, N, K = 1024, 1 << 20, 64
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=0)
    X = torch.tensor(inputs.decisions(K, d, seed=0), device="cuda")
    a = saa.saa_grad(gp, X, "f16x3")
    b = saa.saa_grad(gp, X, "fp32")
    saa.saa_ctx_sync()
    ga, gb = a["grad"].cpu().numpy(), b["grad"].cpu().numpy()
    assert grad_err(ga, gb) <= 2e-6
    rng = np.random.default_rng(1)
    h = 0.5
    for _ in range(12):
        k, j = int(rng.integers(K)), int(rng.integers(d))
        Xp = X[k:k + 1].clone()
        Xm = Xp.clone()
        Xp[0, j] += h
        Xm[0, j] -= h
        cd = (saa.saa_eval(gp, Xp, "fp32")["f"].item() - saa.saa_eval(gp, Xm, "fp32")["f"].item()) / (2 * h)
        assert abs(cd - ga[k, j]) <= 1e-5 * max(1.0, abs(cd))


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_grad_more_than_64_decisions_in_chunks(prec):
    # K = 150: launches of 64, 64 and 22 decisions in one workspace; against
    # the oracle, and each chunk bit for bit the call on its own decisions
    from paper_2404_11631_gb300 import saa
    d, N, K = 300, 5_001, 150
    out, ref, X, inst = _grad(d, N, K, law=oracle.LAW_MIX, seed=5, prec=prec)
    assert grad_err(out["grad"], ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=5)
    Xt = torch.tensor(X, device="cuda")
    for k0 in (0, 64, 128):
        part = saa.saa_grad(gp, Xt[k0:k0 + 64], prec)
        saa.saa_ctx_sync()
        assert np.array_equal(part["grad"].cpu().numpy(), out["grad"][k0:k0 + 64])
        assert np.array_equal(part["f"].cpu().numpy(), out["f"][k0:k0 + 64])


def test_tc_grad_unsupported_shapes_are_rejected():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(1025, 1000)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_grad(gp, torch.zeros(2, 1025, dtype=torch.float64, device="cuda"), "bf16x3")
    assert e.value.status in (saa.SAA_EINVAL, saa.SAA_EUNSUPPORTED)
