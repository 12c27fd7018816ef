"""Parity of the tcgen05 split-precision paths (SAA_F16X3, SAA_BF16X3) with
the oracle on the same FP32-mode samples (Eq. 4 and Eq. 5, Sec. 3.1).  Shapes cover a single
K block, several K blocks with a ragged last one, decision counts that are
not multiples of 32, ragged scenario tails and every law; the full d=128,
N=2^20, K=256 workload is checked on sampled decisions.  Above d = 256 the
values run on the cluster kernel without its adjoint (d <= 1024, K <= 64):
against the oracle, and bit for bit against saa_grad's values, which take
the same exchange.  More decisions than one launch takes run in chunks:
against the oracle, and each chunk bit for bit the call on its decisions."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, est_err, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu


def _tc(d, N, K, law=oracle.LAW_GAUSS, seed=3, nu=4, lam=0.5, prec="f16x3"):
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(d, N, law=law, seed=seed, nu=nu, lam=lam)
    X = inputs.decisions(K, d, seed=seed)
    out = saa.saa_eval(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    ref = oracle.saa(op, 32, X)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref, X, inst


@pytest.mark.parametrize("d,N,K", [(1, 4099, 1), (7, 5000, 3), (64, 20_000, 32), (100, 9_999, 33),
                                   (128, 40_000, 256), (256, 12_345, 64), (200, 30_000, 100)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_MIX, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_value_parity(d, N, K, law, prec):
    out, ref, X, inst = _tc(d, N, K, law=law, prec=prec)
    e_f = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    e_p = est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5)
    e_v = np.max(np.abs(out["var"] - ref["var"]) / ref["var"])
    print(f"{prec} d={d} N={N} K={K} law={law}: f {e_f:.2e} pbar {e_p:.2e} var {e_v:.2e}")
    assert e_f <= TOL[prec] and e_p <= TOL[prec] and e_v <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_small_N_edge(prec):
    # N = 2 (one partial tile, 126 zero rows) and a tile-exact N = 128
    for N in (2, 128, 129):
        out, ref, X, inst = _tc(16, N, 5, seed=N, prec=prec)
        assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL[prec] * 10


def test_tc_deterministic_and_close_to_fp32_path():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(128, 100_000, law=oracle.LAW_MIX, seed=7)
    X = torch.tensor(inputs.decisions(256, 128, seed=7), device="cuda")
    a = saa.saa_eval(gp, X, "f16x3")
    b = saa.saa_eval(gp, X, "f16x3")
    saa.saa_ctx_sync()
    assert torch.equal(a["f"], b["f"]) and torch.equal(a["var"], b["var"])
    c = saa.saa_eval(gp, X, "fp32")
    rel = ((a["f"] - c["f"]).abs() / (0.5 * c["var"] + (X @ gp.mu).abs())).max().item()
    assert rel <= 2e-6


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_full_size_sampled_decisions(prec):
    from paper_2404_11631_gb300 import saa
    d, N, K = 128, 1 << 20, 256
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=0)
    X = inputs.decisions(K, d, seed=0)
    out = saa.saa_eval(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    pick = [0, 131, 255]
    ref = oracle.saa(op, 32, X[pick])
    f = out["f"].cpu().numpy()[pick]
    v = out["var"].cpu().numpy()[pick]
    assert est_err(f, ref["f"], ref["var"], X[pick], inst.mu, 0.5) <= TOL[prec]
    assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= TOL[prec]


@pytest.mark.parametrize("d,N,K", [(300, 5_000, 17), (512, 4_099, 64), (1000, 3_000, 5), (1024, 2_500, 64)])
@pytest.mark.parametrize("law", [oracle.LAW_GAUSS, oracle.LAW_STUDENT_T])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_tc_value_parity_large_d(d, N, K, law, prec):
    from paper_2404_11631_gb300 import saa
    out, ref, X, inst = _tc(d, N, K, law=law, prec=prec)
    e_f = est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5)
    e_p = est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5)
    e_v = np.max(np.abs(out["var"] - ref["var"]) / ref["var"])
    print(f"{prec} d={d} N={N} K={K} law={law}: f {e_f:.2e} pbar {e_p:.2e} var {e_v:.2e}")
    assert e_f <= TOL[prec] and e_p <= TOL[prec] and e_v <= TOL[prec]
    gp, op, inst = make(d, N, law=law, seed=3)
    g = saa.saa_grad(gp, torch.tensor(X, device="cuda"), prec)
    saa.saa_ctx_sync()
    assert np.array_equal(g["f"].cpu().numpy(), out["f"])


def test_tc_value_large_d_many_tiles_sampled_decisions():
    from paper_2404_11631_gb300 import saa
    d, N, K = 1024, 1 << 18, 64
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=0)
    X = inputs.decisions(K, d, seed=0)
    out = saa.saa_eval(gp, torch.tensor(X, device="cuda"), "f16x3")
    saa.saa_ctx_sync()
    pick = [0, 37, 63]
    ref = oracle.saa(op, 32, X[pick])
    f = out["f"].cpu().numpy()[pick]
    assert est_err(f, ref["f"], ref["var"], X[pick], inst.mu, 0.5) <= TOL["f16x3"]


def test_tc_unsupported_shapes_are_rejected():
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(1025, 1000)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_eval(gp, torch.zeros(2, 1025, dtype=torch.float64, device="cuda"), "f16x3")
    assert e.value.status in (saa.SAA_EINVAL, saa.SAA_EUNSUPPORTED)   # the workspace query refuses it first


@pytest.mark.parametrize("d,K,chunk", [(128, 300, 256), (200, 150, 128), (512, 100, 64)])
def test_tc_values_in_decision_chunks(d, K, chunk):
    # more decisions than one launch takes: consecutive chunks in one
    # workspace; against the oracle, and each chunk bit for bit the call on
    # its own decisions
    from paper_2404_11631_gb300 import saa
    N = 4_001
    out, ref, X, inst = _tc(d, N, K, law=oracle.LAW_MIX, seed=d, prec="f16x3")
    assert est_err(out["f"], ref["f"], ref["var"], X, inst.mu, 0.5) <= TOL["f16x3"]
    assert est_err(out["pbar"], ref["pbar"], ref["var"], X, inst.mu, 0.5) <= TOL["f16x3"]
    assert np.max(np.abs(out["var"] - ref["var"]) / ref["var"]) <= TOL["f16x3"]
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=d)
    Xt = torch.tensor(X, device="cuda")
    for k0 in range(0, K, chunk):
        part = saa.saa_eval(gp, Xt[k0:k0 + chunk], "f16x3")
        saa.saa_ctx_sync()
        for key in ("f", "pbar", "var"):
            assert np.array_equal(part[key].cpu().numpy(), out[key][k0:k0 + chunk]), (key, k0)
