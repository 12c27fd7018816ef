"""Algorithm 1 on the GPU (graph-replayed Frank-Wolfe iterations) against
the oracle: teacher-forced step checks, bitwise resume, and the oracle's own
straight run on the FP64 path."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, TOL_GRAD, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_teacher_forced_steps(prec):
    from paper_2404_11631_gb300 import saa
    d, N, M = 16, 4000, 3
    gp, op, inst = make(d, N, law=oracle.LAW_STUDENT_T, seed=21)
    w = torch.tensor(inputs.fw_start(d), device="cuda")
    oprec = 64 if prec == "fp64" else 32
    for t in range(8):
        out = saa.saa_solve(gp, w, T=1, M=M, t0=t, prec=prec)
        wt = w.cpu().numpy()
        ref = oracle.saa(op, oprec, wt, grad=True, epoch=t // M)
        f_gpu = out["f_trace"].cpu().numpy()[0]
        assert abs(f_gpu - ref["f"][0]) <= TOL[prec] * max(abs(ref["f"][0]), 0.5 * ref["var"][0] + abs(wt @ inst.mu))
        g = ref["grad"][0]
        js, gap, wn = oracle.fw_step(g, wt, t)
        w_next = out["w"].cpu().numpy()
        # the GPU's vertex must be optimal for the oracle's gradient up to the tolerance
        s_gpu = (w_next - (1 - 2.0 / (t + 2)) * wt) / (2.0 / (t + 2))
        assert s_gpu @ g <= g.min(initial=0.0) + TOL_GRAD[prec] * np.linalg.norm(g)
        assert abs(out["gap_trace"].cpu().numpy()[0] - gap) <= 1e-5 * max(1.0, abs(gap))
        w = out["w"]


def test_straight_run_matches_oracle_fp64():
    from paper_2404_11631_gb300 import saa
    d, N, T, M = 10, 10_000, 40, 4
    gp, op, inst = make(d, N, seed=0)
    w0 = inputs.fw_start(d)
    out = saa.saa_solve(gp, torch.tensor(w0, device="cuda"), T=T, M=M, prec="fp64")
    ref = oracle.fw(op, 64, w0, T=T, M=M)
    assert np.allclose(out["f_trace"].cpu().numpy(), ref["f_trace"], rtol=1e-10, atol=1e-12)
    assert np.allclose(out["w"].cpu().numpy(), ref["w"], rtol=1e-10, atol=1e-13)


def test_resume_is_bitwise():
    from paper_2404_11631_gb300 import saa
    d, N, M = 32, 3000, 2
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=5)
    w0 = torch.tensor(inputs.fw_start(d), device="cuda")
    full = saa.saa_solve(gp, w0, T=9, M=M, prec="fp32")
    a = saa.saa_solve(gp, w0, T=4, M=M, prec="fp32")
    b = saa.saa_solve(gp, a["w"], T=5, M=M, t0=4, prec="fp32")
    assert torch.equal(b["w"], full["w"])
    assert torch.equal(torch.cat([a["f_trace"], b["f_trace"]]), full["f_trace"])
    assert torch.all(full["gap_trace"] >= 0)
