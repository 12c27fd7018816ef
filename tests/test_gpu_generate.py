"""GPU scenario generator against the oracle: bit-exact innovations, scales
and samples for every law, both scenario precisions, ragged ranges and odd
dimensions (the samples R_i of Sec. 3.1)."""
import numpy as np
import pytest

import oracle
from helpers import make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_LOGN_STD, oracle.LAW_STUDENT_T, oracle.LAW_MIX])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d", [1, 7, 130])
def test_generate_bit_exact(law, prec, d):
    from paper_2404_11631_gb300 import saa
    N = 3001
    gp, op, inst = make(d, N, law=law, nu=6, seed=0x1234_5678_9ABC, instance=77, epoch=5)
    i0, n = 1200, 601   # straddles the Gaussian / lognormal boundary of the mixture
    out = saa.saa_generate(gp, i0, n, prec, want_xi=True)
    z_or, s_or, xi_or = oracle.generate(op, 64 if prec == "fp64" else 32, i0, n, want_xi=True)
    np_t = np.float64 if prec == "fp64" else np.float32
    z = out["z"].cpu().numpy()
    s = out["s"].cpu().numpy()
    xi = out["xi"].cpu().numpy()
    assert np.array_equal(z.view(np.uint64 if prec == "fp64" else np.uint32),
                          z_or.astype(np_t).view(np.uint64 if prec == "fp64" else np.uint32))
    assert np.array_equal(s, s_or.astype(np_t))
    assert np.array_equal(xi, xi_or.astype(np_t))


def test_generate_full_range_sampled_rows():
    # the full-size stream of the d=128, N=2^20 workload: sampled rows
    from paper_2404_11631_gb300 import saa
    N = 1 << 20
    gp, op, inst = make(128, N, law=oracle.LAW_MIX, seed=1)
    for i0 in (0, N // 2 - 3, N - 5):
        out = saa.saa_generate(gp, i0, 5, "fp32")
        z_or, s_or, _ = oracle.generate(op, 32, i0, 5)
        assert np.array_equal(out["z"].cpu().numpy(), z_or.astype(np.float32))


def test_generator_arithmetic_is_ieee_on_its_whole_domain():
    # the LOG quotient and the Box-Muller root, formed by Markstein's
    # correction of the hardware approximations, against the IEEE
    # round-to-nearest results for all 2^23 FP32 uniforms
    from paper_2404_11631_gb300 import saa
    assert saa.saa_selftest_arith() == (0, 0)


def test_generate_many_rows_bit_exact():
    # 2^16 scenarios x 4 dimensions: 2^17 Box-Muller pairs through the
    # shortened arithmetic, every law, against the oracle
    from paper_2404_11631_gb300 import saa
    for law in (oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T):
        gp, op, inst = make(4, 1 << 16, law=law, nu=8, seed=99)
        out = saa.saa_generate(gp, 0, 1 << 16, "fp32")
        z_or, s_or, _ = oracle.generate(op, 32, 0, 1 << 16)
        assert np.array_equal(out["z"].cpu().numpy().view(np.uint32), z_or.astype(np.float32).view(np.uint32))
        assert np.array_equal(out["s"].cpu().numpy(), s_or.astype(np.float32))
