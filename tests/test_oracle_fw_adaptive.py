"""Pins for the oracle's Algorithm 1 with an adaptive sample size (the
resampling step's remark that the sample size N_k may depend on the epoch k).

Epoch k draws N_k samples of resample index epoch + k and runs M iterations
at the global iteration count t = kM + m.  Checked by: a constant schedule
reproducing the plain run bit for bit; every iteration's traced value being
Eq. 4 on that epoch's own N_k samples; the steps following gamma_t =
2/(t+2) with the global t and the LMO vertex of the gradient on that epoch's
samples; a schedule split at an epoch boundary resuming bit for bit; and a
growing schedule converging to the optimum of Eq. 3 found by scipy's SLSQP
on the exact (Sigma, mu)."""
import numpy as np
from scipy.optimize import minimize

import oracle
from paper_2404_11631_gb300 import inputs


def _probs(d, Ns, law=oracle.LAW_GAUSS, seed=0):
    inst = inputs.instance(d, seed=0)
    return [oracle.make_problem(d, int(N), inst.mu, inst.chol, law=law, seed=seed) for N in Ns], inst


def test_constant_schedule_is_the_plain_run():
    d, M = 6, 3
    probs, inst = _probs(d, [1500] * 4)
    w0 = inputs.fw_start(d)
    a = oracle.fw_adaptive(probs, 64, w0, M)
    b = oracle.fw(probs[0], 64, w0, T=4 * M, M=M)
    assert np.array_equal(a["w"], b["w"])
    assert np.array_equal(a["f_trace"], b["f_trace"]) and np.array_equal(a["gap_trace"], b["gap_trace"])


def test_each_epoch_uses_its_own_sample_size_and_the_global_step():
    d, M = 5, 2
    Ns = [300, 700, 1600, 4000]
    probs, inst = _probs(d, Ns, law=oracle.LAW_STUDENT_T, seed=4)
    w0 = inputs.fw_start(d)
    out = oracle.fw_adaptive(probs, 64, w0, M, want_w_trace=True)
    wt = np.vstack([out["w_trace"], out["w"]])   # w_t for t = 0 .. T
    for t in range(len(Ns) * M):
        k = t // M
        ref = oracle.saa(probs[k], 64, wt[t], grad=True, epoch=k)
        assert out["f_trace"][t] == ref["f"][0]
        g = ref["grad"][0]
        j = int(np.argmin(g))
        s = np.eye(d)[j] if g[j] < 0 else np.zeros(d)
        gamma = 2.0 / (t + 2)
        assert np.allclose(wt[t + 1], wt[t] + gamma * (s - wt[t]), rtol=1e-14, atol=1e-16)
        # the same iterate on another epoch's sample size gives another value
        other = oracle.saa(probs[(k + 1) % len(Ns)], 64, wt[t], epoch=k)["f"][0]
        assert other != ref["f"][0]


def test_split_schedule_resumes_bitwise():
    d, M = 7, 3
    Ns = [400, 800, 800, 1600, 3200]
    probs, inst = _probs(d, Ns, law=oracle.LAW_MIX, seed=2)
    w0 = inputs.fw_start(d)
    full = oracle.fw_adaptive(probs, 32, w0, M)
    a = oracle.fw_adaptive(probs[:2], 32, w0, M)
    b = oracle.fw_adaptive(probs[2:], 32, a["w"], M, k0=2)
    assert np.array_equal(b["w"], full["w"])
    assert np.array_equal(np.concatenate([a["f_trace"], b["f_trace"]]), full["f_trace"])


def test_growing_schedule_converges_to_the_qp_optimum():
    d, M = 8, 25
    Ns = [min(500 * 2 ** k, 32_000) for k in range(12)]
    probs, inst = _probs(d, Ns, seed=1)
    S, mu = inst.sigma, inst.mu

    def f(w):
        return 0.5 * w @ S @ w - mu @ w

    res = minimize(f, np.full(d, 0.5 / d), jac=lambda w: S @ w - mu, method="SLSQP",
                   bounds=[(0, None)] * d, constraints=[{"type": "ineq", "fun": lambda w: 1 - w.sum()}],
                   options={"ftol": 1e-14, "maxiter": 500})
    out = oracle.fw_adaptive(probs, 64, inputs.fw_start(d), M)
    assert np.all(out["gap_trace"] >= 0)
    assert f(out["w"]) >= res.fun - 1e-9
    assert f(out["w"]) - res.fun < 2e-2 * abs(res.fun) + 1e-3
