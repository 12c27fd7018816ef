"""saa_eval_static: the value estimate for callers that cannot allocate
device memory (real-time loops that cannot take cudaMalloc's implicit device
synchronisation, plug-ins inside a framework that owns the device heap).
Its scratch is a fixed array in the library, so the test calls it through
the C ABI twice in a row and checks both results against saa_eval, which
uses a caller workspace, and against the CPU oracle; that a warm call leaves
the device's free memory unchanged; that a bad Cholesky diagonal gives NaN
outputs (this path has no context to report it through); and that the
diagonal form is rejected.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from helpers import ORACLE_PREC, TOL, est_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_eval(gp, X, prec, out=None):
    from paper_2404_11631_gb300 import saa
    L = saa.lib()
    L.saa_eval_static.argtypes = [C.POINTER(saa._CProblem), C.c_int32, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
    L.saa_eval_static.restype = C.c_int
    K = X.shape[0]
    if out is None:
        out = [torch.full((K,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    f, pb, vr = out
    cp = gp.c_struct()
    rc = L.saa_eval_static(C.byref(cp), K, X.data_ptr(), saa.PRECS[prec], f.data_ptr(), pb.data_ptr(),
                           vr.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, f, pb, vr


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_static_scratch_matches_workspace_path_twice(prec):
    from paper_2404_11631_gb300 import saa
    cases = [(128, 100_000, 64, oracle.LAW_MIX, 1), (37, 5003, 3, oracle.LAW_STUDENT_T, 2)]
    for d, N, K, law, seed in cases:        # two calls in a row, different sizes
        gp, op, inst = make(d, N, law=law, seed=seed)
        Xn = inputs.decisions(K, d, seed=seed)
        X = torch.tensor(Xn, device="cuda")
        rc, f, pb, vr = _static_eval(gp, X, prec)
        assert rc == saa.SAA_OK, saa.lib().saa_last_error()
        ref = saa.saa_eval(gp, X, prec)
        torch.cuda.synchronize()
        var = ref["var"].cpu().numpy()
        scale = np.maximum(np.abs(ref["f"].cpu().numpy()), 0.5 * var + np.abs(Xn @ inst.mu))
        for a, b in ((f, ref["f"]), (pb, ref["pbar"])):
            assert np.max(np.abs(a.cpu().numpy() - b.cpu().numpy()) / scale) <= TOL[prec]
        assert np.max(np.abs(vr.cpu().numpy() - var) / var) <= TOL[prec]
        # and against the CPU oracle on the same scenarios
        o = oracle.saa(op, ORACLE_PREC[prec], Xn)
        assert est_err(f.cpu().numpy(), o["f"], o["var"], Xn, inst.mu, 0.5) <= TOL[prec]
        assert est_err(pb.cpu().numpy(), o["pbar"], o["var"], Xn, inst.mu, 0.5) <= TOL[prec]


def test_static_call_leaves_free_memory_unchanged():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(64, 50_000, seed=4)
    X = torch.tensor(inputs.decisions(8, 64, seed=4), device="cuda")
    rc, *_ = _static_eval(gp, X, "fp32")          # warm: the module and its array are loaded
    assert rc == saa.SAA_OK
    torch.cuda.synchronize()
    out = [torch.empty(8, dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, f, pb, vr = _static_eval(gp, X, "fp32", out=out)
        assert rc == saa.SAA_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_bad_cholesky_diagonal_gives_nan():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(16, 4096, seed=5)
    X = torch.tensor(inputs.decisions(4, 16, seed=5), device="cuda")
    bad = gp.chol.clone()
    bad[3, 3] = -abs(float(bad[3, 3]))
    gb = saa.Problem(mu=gp.mu, chol=bad, N=gp.N, seed=5)
    rc, f, pb, vr = _static_eval(gb, X, "fp32")
    assert rc == saa.SAA_OK
    torch.cuda.synchronize()
    assert torch.isnan(f).all() and torch.isnan(pb).all() and torch.isnan(vr).all()
    # the next call with a good factor clears the word and gives numbers again
    rc, f, pb, vr = _static_eval(gp, X, "fp32")
    assert rc == saa.SAA_OK
    torch.cuda.synchronize()
    assert torch.isfinite(f).all() and torch.isfinite(vr).all()


def test_static_scratch_rejects_oversized_and_diagonal_problems():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(1024, 10_000, seed=3)
    X = torch.zeros(8192, 1024, dtype=torch.float64, device="cuda")
    rc, f, pb, vr = _static_eval(gp, X, "fp32")
    assert rc == saa.SAA_ENOMEM
    assert b"static array" in saa.lib().saa_last_error()
    dp = saa.Problem(mu=gp.mu, chol=None, sd=torch.ones(1024, dtype=torch.float64, device="cuda"), N=1000)
    rc, f, pb, vr = _static_eval(dp, X[:1], "fp32")
    assert rc == saa.SAA_EUNSUPPORTED
    assert b"diagonal form" in saa.lib().saa_last_error()
