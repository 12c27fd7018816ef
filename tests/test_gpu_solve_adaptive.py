"""Algorithm 1 with a sample size per epoch on the GPU (saa_solve_adaptive)
against the oracle's fw_adaptive: the FP64 path follows the oracle's run,
a constant schedule reproduces saa_solve bit for bit, a schedule split at
an epoch boundary resumes bit for bit, and a growing schedule converges to
the optimum of Eq. 3 found by scipy on the exact (Sigma, mu)."""
import numpy as np
import pytest
import torch
from scipy.optimize import minimize

import oracle
from helpers import make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_probs(d, Ns, inst, law, seed):
    return [oracle.make_problem(d, int(N), inst.mu, inst.chol, law=law, seed=seed) for N in Ns]


def test_adaptive_matches_oracle_fp64():
    from paper_2404_11631_gb300 import saa
    d, M = 10, 4
    Ns = [2000, 4000, 4000, 8000, 16000]
    gp, op, inst = make(d, Ns[0], law=oracle.LAW_STUDENT_T, seed=3)
    w0 = inputs.fw_start(d)
    out = saa.saa_solve_adaptive(gp, torch.tensor(w0, device="cuda"), Ns, M=M, prec="fp64")
    ref = oracle.fw_adaptive(_oracle_probs(d, Ns, inst, oracle.LAW_STUDENT_T, 3), 64, w0, M)
    assert np.allclose(out["f_trace"].cpu().numpy(), ref["f_trace"], rtol=1e-10, atol=1e-12)
    assert np.allclose(out["gap_trace"].cpu().numpy(), ref["gap_trace"], rtol=1e-8, atol=1e-12)
    assert np.allclose(out["w"].cpu().numpy(), ref["w"], rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_constant_schedule_is_saa_solve(prec):
    from paper_2404_11631_gb300 import saa
    d, N, M = 64, 5000, 3
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=8)
    w0 = torch.tensor(inputs.fw_start(d), device="cuda")
    a = saa.saa_solve_adaptive(gp, w0, [N] * 4, M=M, prec=prec)
    b = saa.saa_solve(gp, w0, T=4 * M, M=M, prec=prec)
    assert torch.equal(a["w"], b["w"]) and torch.equal(a["f_trace"], b["f_trace"])


def test_split_schedule_resumes_bitwise():
    from paper_2404_11631_gb300 import saa
    d, M = 32, 2
    Ns = [1000, 3000, 3000, 9000]
    gp, op, inst = make(d, Ns[0], seed=6)
    w0 = torch.tensor(inputs.fw_start(d), device="cuda")
    full = saa.saa_solve_adaptive(gp, w0, Ns, M=M, prec="fp32")
    a = saa.saa_solve_adaptive(gp, w0, Ns[:1], M=M, prec="fp32")
    b = saa.saa_solve_adaptive(gp, a["w"], Ns[1:], M=M, k0=1, prec="fp32")
    assert torch.equal(b["w"], full["w"])
    assert torch.equal(torch.cat([a["f_trace"], b["f_trace"]]), full["f_trace"])
    assert torch.all(full["gap_trace"] >= 0)


def test_growing_schedule_converges():
    from paper_2404_11631_gb300 import saa
    d, M = 8, 25
    Ns = [min(500 * 2 ** k, 64_000) for k in range(12)]
    gp, op, inst = make(d, Ns[0], seed=1)
    S, mu = inst.sigma, inst.mu

    def f(w):
        return 0.5 * w @ S @ w - mu @ w

    res = minimize(f, np.full(d, 0.5 / d), jac=lambda w: S @ w - mu, method="SLSQP",
                   bounds=[(0, None)] * d, constraints=[{"type": "ineq", "fun": lambda w: 1 - w.sum()}],
                   options={"ftol": 1e-14, "maxiter": 500})
    out = saa.saa_solve_adaptive(gp, torch.tensor(inputs.fw_start(d), device="cuda"), Ns, M=M, prec="fp32")
    w = out["w"].cpu().numpy()
    assert np.all(w >= 0) and w.sum() <= 1 + 1e-12
    assert f(w) >= res.fun - 1e-9 and f(w) - res.fun < 2e-2 * abs(res.fun) + 1e-3


def test_bad_schedules_are_rejected():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(8, 100)
    w0 = torch.tensor(inputs.fw_start(8), device="cuda")
    with pytest.raises(saa.SAAError):
        saa.saa_solve_adaptive(gp, w0, [100, 1], M=2)
    with pytest.raises(saa.SAAError):
        saa.saa_solve_adaptive(gp, w0, [], M=2)
