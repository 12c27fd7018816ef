"""saa_eval_static: the value estimate for callers that cannot allocate
device memory (host callbacks, stream capture, real-time loops, plug-ins in
a framework that owns the device heap).  Its scratch is a fixed array in
the library, so the test calls it through the C ABI twice in a row and
checks both results against saa_eval, which uses a caller workspace.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_eval(gp, X, prec):
    from paper_2404_11631_gb300 import saa
    L = saa.lib()
    L.saa_eval_static.argtypes = [C.POINTER(saa._CProblem), C.c_int32, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
    L.saa_eval_static.restype = C.c_int
    K = X.shape[0]
    f = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    pb = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    vr = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
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
        X = torch.tensor(inputs.decisions(K, d, seed=seed), device="cuda")
        rc, f, pb, vr = _static_eval(gp, X, prec)
        assert rc == saa.SAA_OK, saa.lib().saa_last_error()
        ref = saa.saa_eval(gp, X, prec)
        torch.cuda.synchronize()
        var = ref["var"].cpu().numpy()
        scale = np.maximum(np.abs(ref["f"].cpu().numpy()), 0.5 * var + np.abs(X.cpu().numpy() @ inst.mu))
        for a, b in ((f, ref["f"]), (pb, ref["pbar"])):
            assert np.max(np.abs(a.cpu().numpy() - b.cpu().numpy()) / scale) <= TOL[prec]
        assert np.max(np.abs(vr.cpu().numpy() - var) / var) <= TOL[prec]


def test_static_scratch_rejects_oversized_problems():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(1024, 10_000, seed=3)
    X = torch.zeros(8192, 1024, dtype=torch.float64, device="cuda")
    rc, f, pb, vr = _static_eval(gp, X, "fp32")
    assert rc == saa.SAA_ENOMEM
    assert b"static array" in saa.lib().saa_last_error()
