"""Ragged batches of independent problems (Eq. 4 for each, Sec. 3.1) in one
persistent launch, against the oracle problem by problem: mixed d, N, K and
laws, ragged tails, and the full 4096-instance workload on sampled problems."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, est_err, var_err
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _build(rb, laws, prec):
    from paper_2404_11631_gb300 import saa
    probs, Xs, ops = [], [], []
    for b in range(len(rb.d)):
        inst, X = rb.instances[b], rb.X[b]
        d, N = int(rb.d[b]), int(rb.N[b])
        law = laws[b % len(laws)]
        probs.append(saa.Problem(mu=torch.tensor(inst.mu, device="cuda"), chol=torch.tensor(inst.chol, device="cuda"),
                                 N=N, law=law, nu=4, seed=int(rb.seeds[b]), instance=b))
        Xs.append(torch.tensor(X, device="cuda"))
        ops.append(oracle.make_problem(d, N, inst.mu, inst.chol, law=law, nu=4, seed=int(rb.seeds[b]), instance=b))
    return probs, Xs, ops


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_small_ragged_batch_matches_oracle(prec):
    from paper_2404_11631_gb300 import saa
    rb = inputs.ragged_batch(37, seed=5, d_range=(1, 300), logN_range=(0.4, 4.3), K_range=(1, 16))
    laws = [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T, oracle.LAW_LOGN_STD]
    probs, Xs, ops = _build(rb, laws, prec)
    assert min(rb.N) >= 2
    batch = saa.Batch(probs, Xs, prec)
    for _ in range(2):                       # autotuned first call, cached shape second
        out = batch.run()
    saa.saa_ctx_sync()
    for b in range(len(probs)):
        ref = oracle.saa(ops[b], 64 if prec == "fp64" else 32, rb.X[b])
        f = out["f"][b].cpu().numpy()
        v = out["var"][b].cpu().numpy()
        assert est_err(f, ref["f"], ref["var"], rb.X[b], rb.instances[b].mu, 0.5) <= TOL[prec], b
        assert var_err(v, ref["var"], ref["f"], rb.X[b], rb.instances[b].mu, 0.5) <= TOL[prec], b


def test_full_ragged_4096_sampled_instances():
    # 4096 instances, d ~ U{8..512}, N = floor(10^U[3,5]), K ~ U{1..16}, Gaussian
    from paper_2404_11631_gb300 import saa
    rb = inputs.ragged_batch(4096, seed=0)
    probs, Xs, ops = _build(rb, [oracle.LAW_GAUSS], "fp32")
    batch = saa.Batch(probs, Xs, "fp32")
    out = batch.run()
    out = batch.run()
    saa.saa_ctx_sync()
    for b in (0, 1, 777, 2048, 4095):
        ref = oracle.saa(ops[b], 32, rb.X[b])
        f = out["f"][b].cpu().numpy()
        assert est_err(f, ref["f"], ref["var"], rb.X[b], rb.instances[b].mu, 0.5) <= TOL["fp32"], b
    # every instance agrees with its single-problem evaluation
    for b in range(0, 4096, 97):
        single = saa.saa_eval(probs[b], Xs[b], "fp32")["f"]
        rel = ((out["f"][b] - single).abs() / (0.5 * out["var"][b] + (Xs[b] @ probs[b].mu).abs())).max().item()
        assert rel <= 1e-6, b
