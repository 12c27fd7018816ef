"""The diagonal-covariance path (chol None, Sigma = diag(sd^2): the
independent assets of Sec. 4.1) against the oracle's diagonal branch: value
and gradient over dimensions that cross the kernels' staging chunks (8192 /
K dimensions) with ragged ends, up to Sec. 4.1's largest d = 10^5, every law
and K = 1..4; the adjoint's sample store bitwise equal to drawing again;
Algorithm 1 teacher-forced at d = 5000, resumed bitwise and run with an
adaptive sample size; a bad spread reported on the device.

Tolerances are the FP32 path's (relative 1e-6): each 4-dimension block's
dot product rounds once in FP32 before a float-float sum, and the decision
image sd o w is rounded to FP32."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, est_err, grad_err
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _make(d, N, law=oracle.LAW_GAUSS, nu=4, lam=0.5, seed=0, epoch=0, inst_seed=0):
    from paper_2404_11631_gb300 import saa
    mu, sd = inputs.paper_assets(d, inst_seed)
    gp = saa.Problem(mu=torch.tensor(mu, device="cuda"), chol=None, sd=torch.tensor(sd, device="cuda"), N=N, law=law,
                     nu=nu, lam=lam, seed=seed, epoch=epoch)
    op = oracle.make_problem(d, N, mu, None, law=law, nu=nu, lam=lam, seed=seed, epoch=epoch, sd=sd)
    return gp, op, mu


def _check(d, N, K, law=oracle.LAW_GAUSS, grad=False, lam=0.5, seed=3):
    from paper_2404_11631_gb300 import saa
    gp, op, mu = _make(d, N, law=law, lam=lam, seed=seed)
    X = inputs.decisions(K, d, seed=d) / d   # on the scale of the simplex
    Xt = torch.tensor(X, device="cuda")
    out = saa.saa_grad(gp, Xt) if grad else saa.saa_eval(gp, Xt)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.saa(op, 32, X, grad=grad)
    e = est_err(out["f"], ref["f"], ref["var"], X, mu, lam)
    msg = f"d={d} N={N} K={K} law={law}: f {e:.2e}"
    if grad:
        eg = grad_err(out["grad"], ref["grad"])
        print(msg + f" grad {eg:.2e}")
        assert eg <= TOL_GRAD["fp32"]
    else:
        ep = est_err(out["pbar"], ref["pbar"], ref["var"], X, mu, lam)
        ev = float(np.max(np.abs(out["var"] - ref["var"]) / ref["var"]))
        print(msg + f" pbar {ep:.2e} var {ev:.2e}")
        assert ep <= TOL["fp32"] and ev <= TOL["fp32"]
    assert e <= TOL["fp32"]


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("d,N,K", [(1, 2, 1), (5, 1000, 3), (1000, 3001, 1), (2051, 999, 4), (4099, 700, 2),
                                   (8195, 333, 1), (20_000, 200, 3)])
def test_value_parity(d, N, K, law):
    _check(d, N, K, law=law)


@pytest.mark.parametrize("d,N,K,law", [(1, 3, 1, oracle.LAW_GAUSS), (7, 5000, 2, oracle.LAW_MIX),
                                       (1000, 3001, 1, oracle.LAW_STUDENT_T), (2051, 999, 4, oracle.LAW_MIX),
                                       (8195, 400, 1, oracle.LAW_GAUSS), (20_000, 300, 2, oracle.LAW_STUDENT_T)])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_grad_parity(d, N, K, law, lam):
    _check(d, N, K, law=law, grad=True, lam=lam)


def test_paper_largest_dimension():
    # Sec. 4.1's largest instance, 10^5 independent assets, on a small sample
    _check(100_000, 256, 1, grad=True)


def test_deterministic_and_unsupported_forms():
    from paper_2404_11631_gb300 import saa
    gp, op, mu = _make(3000, 20_000, law=oracle.LAW_MIX, seed=9)
    X = torch.tensor(inputs.decisions(3, 3000, seed=1) / 3000, device="cuda")
    a = [saa.saa_grad(gp, X) for _ in range(3)]
    for r in a[1:]:
        assert torch.equal(r["grad"], a[0]["grad"]) and torch.equal(r["f"], a[0]["f"])
    # the workspace query already refuses these (size 0, the reason in the message)
    for prec in ("fp64", "f16x3"):
        with pytest.raises(saa.SAAError) as e:
            saa.saa_eval(gp, X, prec)
        assert e.value.status in (saa.SAA_EINVAL, saa.SAA_EUNSUPPORTED) and "FP32 only" in str(e.value)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_eval(gp, torch.tensor(inputs.decisions(5, 3000, seed=1), device="cuda"))
    assert e.value.status in (saa.SAA_EINVAL, saa.SAA_EUNSUPPORTED) and "K <= 4" in str(e.value)


@pytest.mark.parametrize("d,N,K,law", [(7, 3001, 1, oracle.LAW_STUDENT_T), (2051, 999, 3, oracle.LAW_MIX),
                                       (9000, 517, 2, oracle.LAW_GAUSS)])
def test_sample_store_matches_redraw_bitwise(d, N, K, law):
    # the adjoint's normals from the store (forward pass) or drawn again: same bits
    from paper_2404_11631_gb300 import saa
    gp, op, mu = _make(d, N, law=law, seed=13)
    X = torch.tensor(inputs.decisions(K, d, seed=2) / d, device="cuda")
    kept = saa.saa_grad(gp, X)
    saa.saa_ctx_set_sample_store(0)
    try:
        assert saa.workspace_size(gp, K, "fp32", 1) < 4 * N * d
        redrawn = saa.saa_grad(gp, X)
    finally:
        saa.saa_ctx_set_sample_store(1 << 35)
    saa.saa_ctx_sync()
    assert saa.workspace_size(gp, K, "fp32", 1) >= 4 * N * d
    assert torch.equal(kept["grad"], redrawn["grad"]) and torch.equal(kept["f"], redrawn["f"])


def test_bad_spread_is_flagged():
    from paper_2404_11631_gb300 import saa
    gp, op, mu = _make(100, 500)
    sd = gp.sd.clone()
    sd[17] = -1.0
    bad = saa.Problem(mu=gp.mu, chol=None, sd=sd, N=500)
    saa.saa_eval(bad, torch.ones(1, 100, dtype=torch.float64, device="cuda") / 100)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()   # the word was cleared; the context still works
    saa.saa_eval(gp, torch.ones(1, 100, dtype=torch.float64, device="cuda") / 100)
    saa.saa_ctx_sync()


def test_solve_teacher_forced():
    from paper_2404_11631_gb300 import saa
    d, N, M = 5000, 2048, 3
    gp, op, mu = _make(d, N, law=oracle.LAW_STUDENT_T, seed=21)
    w = torch.tensor(inputs.fw_start(d), device="cuda")
    for t in range(7):
        out = saa.saa_solve(gp, w, T=1, M=M, t0=t)
        wt = w.cpu().numpy()
        ref = oracle.saa(op, 32, wt, grad=True, epoch=t // M)
        f_gpu = out["f_trace"].cpu().numpy()[0]
        assert abs(f_gpu - ref["f"][0]) <= TOL["fp32"] * max(abs(ref["f"][0]), 0.5 * ref["var"][0] + abs(wt @ mu))
        g = ref["grad"][0]
        js, gap, wn = oracle.fw_step(g, wt, t)
        w_next = out["w"].cpu().numpy()
        s_gpu = (w_next - (1 - 2.0 / (t + 2)) * wt) / (2.0 / (t + 2))
        assert s_gpu @ g <= g.min(initial=0.0) + TOL_GRAD["fp32"] * np.linalg.norm(g)
        assert abs(out["gap_trace"].cpu().numpy()[0] - gap) <= 1e-5 * max(1.0, abs(gap))
        w = out["w"]


def test_solve_resume_bitwise_and_adaptive():
    from paper_2404_11631_gb300 import saa
    d, N, M = 1200, 1500, 2
    gp, op, mu = _make(d, N, law=oracle.LAW_MIX, seed=5)
    w0 = torch.tensor(inputs.fw_start(d), device="cuda")
    full = saa.saa_solve(gp, w0, T=9, M=M)
    a = saa.saa_solve(gp, w0, T=4, M=M)
    b = saa.saa_solve(gp, a["w"], T=5, M=M, t0=4)
    assert torch.equal(b["w"], full["w"])
    assert torch.equal(torch.cat([a["f_trace"], b["f_trace"]]), full["f_trace"])
    assert torch.all(full["gap_trace"] >= 0)
    # a constant sample-size schedule is saa_solve itself
    c = saa.saa_solve_adaptive(gp, w0, [N] * 3, M=M)
    full6 = saa.saa_solve(gp, w0, T=3 * M, M=M)
    assert torch.equal(c["w"], full6["w"]) and torch.equal(c["f_trace"], full6["f_trace"])
    # a growing schedule, teacher-forced one epoch (M = 1 iteration) at a time
    w = w0
    for k, n in enumerate([300, 600, 1200, 2400]):
        out = saa.saa_solve_adaptive(gp, w, [n], M=1, k0=k)
        wt = w.cpu().numpy()
        r = oracle.saa(_make(d, n, law=oracle.LAW_MIX, seed=5)[1], 32, wt, epoch=k)
        f = out["f_trace"].cpu().numpy()[0]
        assert abs(f - r["f"][0]) <= TOL["fp32"] * max(abs(r["f"][0]), 0.5 * r["var"][0] + abs(wt @ mu))
        w = out["w"]
