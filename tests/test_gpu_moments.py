"""saa_generate_moments: per-dimension sums of the generator's innovations
and their squares.  Parity with sums of the oracle's own draws (both
generator modes), the standardised laws' mean 0 and variance 1 at 2^24
scenarios (the samples of Sec. 3.1 at a scale the host cannot draw),
determinism and argument checks."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,oprec,tol", [("fp32", 32, 2e-6), ("fp64", 64, 1e-12)])
@pytest.mark.parametrize("d,n,i0", [(10, 5000, 0), (129, 777, 100), (1000, 300, 7)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
def test_moments_match_oracle_draws(prec, oprec, tol, d, n, i0, law):
    from paper_2404_11631_gb300 import saa
    N = i0 + n + 11
    gp, op, inst = make(d, N, law=law, seed=12)
    out = saa.saa_generate_moments(gp, i0, n, prec)
    saa.saa_ctx_sync()
    z, s, _ = oracle.generate(op, oprec, i0, n)
    for key, ref in (("sum", z.sum(axis=0)), ("sumsq", (z * z).sum(axis=0))):
        got = out[key].cpu().numpy()
        scale = np.abs(z).sum(axis=0) if key == "sum" else (z * z).sum(axis=0)
        assert np.all(np.abs(got - ref) <= tol * np.maximum(scale, 1.0)), key


# fourth moments: Gaussian 3; standardised lognormal (sigma = 1): e^4 + 2e^3 + 3e^2 - 3
KURT = {oracle.LAW_GAUSS: 3.0, oracle.LAW_LOGN_STD: math.exp(4) + 2 * math.exp(3) + 3 * math.exp(2) - 3}


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_LOGN_STD, oracle.LAW_MIX])
def test_standardised_laws_at_scale(law):
    from paper_2404_11631_gb300 import saa
    d, n = 16, 1 << 24
    gp, op, inst = make(d, n, law=law, seed=3)
    out = saa.saa_generate_moments(gp, 0, n, "fp32")
    saa.saa_ctx_sync()
    mean = out["sum"].cpu().numpy() / n
    var = out["sumsq"].cpu().numpy() / n - mean * mean
    k4 = KURT[law] if law != oracle.LAW_MIX else 0.5 * (KURT[oracle.LAW_GAUSS] + KURT[oracle.LAW_LOGN_STD])
    assert np.all(np.abs(mean) <= 5.0 / math.sqrt(n))
    assert np.all(np.abs(var - 1.0) <= 5.0 * math.sqrt(k4 - 1.0) / math.sqrt(n))


def test_moments_deterministic_and_checked():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(64, 100_000, law=oracle.LAW_MIX, seed=1)
    a = saa.saa_generate_moments(gp, 0, 100_000, "fp32")
    b = saa.saa_generate_moments(gp, 0, 100_000, "fp32")
    saa.saa_ctx_sync()
    assert torch.equal(a["sum"], b["sum"]) and torch.equal(a["sumsq"], b["sumsq"])
    with pytest.raises(saa.SAAError):
        saa.saa_generate_moments(gp, 99_990, 20, "fp32")
    with pytest.raises(saa.SAAError):
        saa.saa_generate_moments(gp, 0, 10, "bf16x3")
