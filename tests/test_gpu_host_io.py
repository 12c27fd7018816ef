"""saa_eval_host: Eq. 4 with mu, C, the decisions and the outputs in host
memory.  The library copies in, evaluates and copies back; its results must
be bitwise those of saa_eval on the same inputs (same kernels, same
workspace layout), for pinned and pageable host arrays, dense and diagonal
problems."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, est_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "fp64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_match_device_call(prec, pinned):
    from paper_2404_11631_gb300 import saa
    d, N, K = 96, 40_000, 12
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=7)
    Xn = inputs.decisions(K, d, seed=7)
    dev = saa.saa_eval(gp, torch.tensor(Xn, device="cuda"), prec)
    torch.cuda.synchronize()

    def host(a):
        t = torch.tensor(a)
        return t.pin_memory() if pinned else t
    hp = saa.Problem(mu=host(inst.mu), chol=host(inst.chol), N=N, law=oracle.LAW_MIX, seed=7)
    out = saa.saa_eval_host(hp, host(Xn), prec)
    for k in ("f", "pbar", "var"):
        assert torch.equal(out[k], dev[k].cpu()), k
    o = oracle.saa(op, 64 if prec == "fp64" else 32, Xn)
    assert est_err(out["f"].numpy(), o["f"], o["var"], Xn, inst.mu, 0.5) <= TOL[prec]


def test_host_buffers_diagonal_problem_and_optional_outputs():
    from paper_2404_11631_gb300 import saa
    d, N = 3000, 4096
    mu, sd = inputs.paper_assets(d, 0)
    w = inputs.fw_start(d)[None]
    dp = saa.Problem(mu=torch.tensor(mu, device="cuda"), chol=None, sd=torch.tensor(sd, device="cuda"), N=N)
    dev = saa.saa_eval(dp, torch.tensor(w, device="cuda"), "fp32")
    torch.cuda.synchronize()
    hp = saa.Problem(mu=torch.tensor(mu), chol=None, sd=torch.tensor(sd), N=N)
    out = {"f": torch.empty(1, dtype=torch.float64)}
    saa.saa_eval_host(hp, torch.tensor(w), "fp32", out=out)
    assert torch.equal(out["f"], dev["f"].cpu())


def test_host_call_reports_a_bad_cholesky_diagonal():
    from paper_2404_11631_gb300 import saa
    d, N = 8, 1000
    inst = inputs.instance(d, 0)
    ch = np.array(inst.chol)
    ch[2, 2] = 0.0
    hp = saa.Problem(mu=torch.tensor(inst.mu), chol=torch.tensor(ch), N=N)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_eval_host(hp, torch.tensor(inputs.decisions(2, d, 0)), "fp32")
    assert e.value.status == saa.SAA_EDEVICE
    # the call read and cleared the word: the context works on
    inst_ok = saa.Problem(mu=torch.tensor(inst.mu), chol=torch.tensor(inst.chol), N=N)
    out = saa.saa_eval_host(inst_ok, torch.tensor(inputs.decisions(2, d, 0)), "fp32")
    assert torch.isfinite(out["f"]).all()
