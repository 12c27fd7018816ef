"""The scenario-range partial sums on the GPU (saa_partials), their merge
(saa_partials_merge) and the estimate finalized from the totals
(saa_finalize_partials): the sums over i of Eq. 4 and Eq. 5 (Sec. 3.1)
split by scenario, the exchange a split of one problem's N across devices
needs.

* Each range's partials against the oracle's partials of the same range
  (every precision, value and gradient, ranges that cross the mixed law's
  split, ragged tiles and one-scenario ranges).
* N split into 2 to 4 ranges, merged in fixed order and finalized: equal to
  the single-call saa_eval / saa_grad within the tolerance and to the
  oracle; the merge does not depend on which range's row came from where.
* multirank.estimate_sharded on one GPU (no process group).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, ORACLE_PREC, est_err, grad_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b, scale):
    return float(np.max(np.abs(a - b) / scale))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3", "bf16x3"])
@pytest.mark.parametrize("grad", [False, True])
def test_range_partials_match_oracle(prec, grad):
    from paper_2404_11631_gb300 import saa
    d, N, K = 48, 9001, 5
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=6)
    X = inputs.decisions(K, d, seed=6)
    Xt = torch.tensor(X, device="cuda")
    for i0, n in ((0, 1), (17, 300), (4400, 300), (4500, 4501), (0, N)):
        got = saa.saa_partials(gp, i0, n, Xt, prec, grad=grad).cpu().numpy()
        ref = oracle.partials(op, ORACLE_PREC[prec], i0, n, X, grad=grad)
        # scales: P1, P2 by the range's sum of squares; P3, P4 by their own size
        p2 = np.abs(ref[K:2 * K])
        s1 = np.sqrt(n * p2) + 1e-300
        tol = 1e-12 if prec == "fp64" else (20 * TOL[prec])
        assert _rel(got[:K], ref[:K], s1) <= tol
        assert _rel(got[K:2 * K], ref[K:2 * K], p2 + 1e-300) <= tol
        p3 = ref[2 * K:2 * K + d]
        assert np.linalg.norm(got[2 * K:2 * K + d] - p3) <= tol * max(np.sqrt(n * d), 1.0)
        if grad:
            g, r = got[2 * K + d:].reshape(K, d), ref[2 * K + d:].reshape(K, d)
            scale = np.sqrt(p2)[:, None] * np.sqrt(n)
            assert np.max(np.linalg.norm(g - r, axis=1) / scale[:, 0]) <= tol


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "bf16x3", "fp64"])
@pytest.mark.parametrize("ranges", [2, 3, 4])
def test_split_merge_finalize_equals_single_call(prec, ranges):
    from paper_2404_11631_gb300 import multirank, saa
    d, N, K = 130, 20_011, 7
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, seed=8)
    X = inputs.decisions(K, d, seed=8)
    Xt = torch.tensor(X, device="cuda")
    rows = torch.stack([saa.saa_partials(gp, a, b - a, Xt, prec, grad=True)
                        for a, b in multirank.scenario_ranges(N, ranges)])
    tot = saa.saa_partials_merge(rows)
    out = saa.saa_finalize_partials(gp, Xt, tot, grad=True)
    one = saa.saa_grad(gp, Xt, prec)
    ev = saa.saa_eval(gp, Xt, prec)
    saa.saa_ctx_sync()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.saa(op, ORACLE_PREC[prec], X, grad=True)
    assert est_err(o["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    assert est_err(o["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5) <= TOL[prec]
    assert grad_err(o["grad"], ref["grad"]) <= TOL_GRAD[prec]
    assert est_err(o["f"], ev["f"].cpu().numpy(), ref["var"], X, inst.mu, 0.5) <= 2 * TOL[prec]
    assert grad_err(o["grad"], one["grad"].cpu().numpy()) <= 2 * TOL_GRAD[prec]


def test_merge_is_fixed_order_and_exact_for_permuted_production():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(20, 5000, seed=2)
    Xt = torch.tensor(inputs.decisions(3, 20, seed=2), device="cuda")
    a = saa.saa_partials(gp, 0, 2500, Xt, "fp32", grad=True)
    b = saa.saa_partials(gp, 2500, 2500, Xt, "fp32", grad=True)
    b2 = saa.saa_partials(gp, 2500, 2500, Xt, "fp32", grad=True)   # produced later: same bits
    t1 = saa.saa_partials_merge(torch.stack([a, b]))
    t2 = saa.saa_partials_merge(torch.stack([a, b2]))
    assert torch.equal(t1, t2)
    # the merge of one row is that row
    assert torch.equal(saa.saa_partials_merge(a[None].contiguous()), a)


def test_estimate_sharded_one_gpu():
    from paper_2404_11631_gb300 import multirank, saa
    gp, op, inst = make(64, 30_000, law=oracle.LAW_MIX, seed=9)
    X = inputs.decisions(4, 64, seed=9)
    out = multirank.estimate_sharded(gp, torch.tensor(X, device="cuda"), "f16x3", grad=True)
    ref = oracle.saa(op, 32, X, grad=True)
    assert est_err(out["f"].cpu().numpy(), ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL["f16x3"]
    assert grad_err(out["grad"].cpu().numpy(), ref["grad"]) <= TOL_GRAD["f16x3"]


def test_partials_reject_bad_ranges():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(8, 1000)
    Xt = torch.tensor(inputs.decisions(2, 8, seed=0), device="cuda")
    for i0, n in ((-1, 10), (0, 0), (990, 11)):
        with pytest.raises(saa.SAAError) as e:
            saa.saa_partials(gp, i0, n, Xt, "fp32")
        assert e.value.status == saa.SAA_EINVAL
