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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_gradient_matches_oracle(prec):
    # value and gradient of Eq. 4 per problem from one graph-replayed batch
    from helpers import TOL_GRAD, grad_err
    from paper_2404_11631_gb300 import saa
    rb = inputs.ragged_batch(23, seed=9, d_range=(1, 260), logN_range=(0.4, 4.0), K_range=(1, 9))
    laws = [oracle.LAW_MIX, oracle.LAW_GAUSS, oracle.LAW_STUDENT_T]
    probs, Xs, ops = _build(rb, laws, prec)
    batch = saa.Batch(probs, Xs, prec, want_grad=True)
    out = batch.run()
    out = batch.run()
    saa.saa_ctx_sync()
    for b in range(len(probs)):
        ref = oracle.saa(ops[b], 64 if prec == "fp64" else 32, rb.X[b], grad=True)
        assert est_err(out["f"][b].cpu().numpy(), ref["f"], ref["var"], rb.X[b], rb.instances[b].mu,
                       0.5) <= TOL[prec], b
        assert grad_err(out["grad"][b].cpu().numpy(), ref["grad"]) <= TOL_GRAD[prec], b
    batch.close()


def test_graph_replay_reads_current_decisions_and_matches_one_shot():
    from paper_2404_11631_gb300 import saa
    rb = inputs.ragged_batch(9, seed=2, d_range=(4, 90), logN_range=(2.0, 3.5), K_range=(1, 6))
    probs, Xs, ops = _build(rb, [oracle.LAW_GAUSS, oracle.LAW_MIX], "fp32")
    g = saa.Batch(probs, Xs, "fp32")
    one = saa.saa_eval_batched(probs, Xs, "fp32")
    out = g.run()
    saa.saa_ctx_sync()
    for b in range(len(probs)):
        assert torch.equal(out["f"][b], one["f"][b]) and torch.equal(out["var"][b], one["var"][b])
    # new decisions written in place: the replayed graph evaluates them
    rng = np.random.default_rng(4)
    newX = []
    for b, X in enumerate(Xs):
        x = rng.uniform(0.0, 1.0, size=tuple(X.shape))
        X.copy_(torch.tensor(x, device="cuda"))
        newX.append(x)
    out = g.run()
    saa.saa_ctx_sync()
    for b in range(len(probs)):
        ref = oracle.saa(ops[b], 32, newX[b])
        assert est_err(out["f"][b].cpu().numpy(), ref["f"], ref["var"], newX[b], rb.instances[b].mu,
                       0.5) <= TOL["fp32"], b
    g.close()


def test_full_ragged_4096_gradient_sampled_instances():
    # the 4096-instance ragged workload with gradients; oracle on problems small enough to check
    from helpers import TOL_GRAD, grad_err
    from paper_2404_11631_gb300 import saa
    rb = inputs.ragged_batch(4096, seed=0)
    probs, Xs, ops = _build(rb, [oracle.LAW_GAUSS], "fp32")
    out = saa.saa_grad_batched(probs, Xs, "fp32")
    saa.saa_ctx_sync()
    cost = rb.N.astype(np.float64) * rb.d.astype(np.float64) ** 2
    picks = [int(b) for b in np.argsort(cost)[[0, 1, 500, 1500, 2500]]]
    for b in picks:
        ref = oracle.saa(ops[b], 32, rb.X[b], grad=True)
        assert grad_err(out["grad"][b].cpu().numpy(), ref["grad"]) <= TOL_GRAD["fp32"], b
