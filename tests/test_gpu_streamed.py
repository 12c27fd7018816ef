"""Streamed mode (saa_eval_samples): Eq. 4 on a sample set held in device
memory, read by TMA tensor loads and contracted on the tensor cores, against
the oracle's Eq. 4 on the same FP32 samples (oracle.saa_explicit).

Shapes cover the smallest row (d = 4) and N = 2, a second TMA box wholly
past d (d = 32) or partly past it (d = 36, 100), ragged scenario tails,
decision counts that are not multiples of 32, the largest decision image
(d = 256 with K = 128; d = 128 with K = 256) and heavy-tailed samples; the
d = 128, N = 2^20, K = 256 workload is checked on sampled decisions.  The
error measure is helpers.est_err's with the oracle's |pbar| in place of
|mu'w|: |a - b| / max(|b|, lambda V + |pbar|).

Without a center the contraction carries the mean: Q_ik = R_i'x_k instead
of (R_i - c)'x_k, and the tensor pipe's FP32 accumulation error of Q, which
is relative to |Q|, reaches V multiplied by (pbar^2 + V) / V.  Uncentred
cases are held to the tolerance times that factor."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu
LAM = 0.5


def _err(a, ref, key):
    scale = np.maximum(np.abs(ref[key]), LAM * ref["var"] + np.abs(ref["pbar"]))
    return float(np.max(np.abs(a - ref[key]) / scale))


def _run(R, X, prec, centred=True, lam=LAM):
    from paper_2404_11631_gb300 import saa
    Rg = torch.from_numpy(R).cuda()
    Xg = torch.tensor(X, device="cuda")
    kw = {}
    if centred:
        kw["center"] = torch.tensor(R.astype(np.float64).mean(axis=0), device="cuda")
        kw["sigma"] = torch.tensor(R.astype(np.float64).std(axis=0) + 1e-30, device="cuda")
    out = saa.saa_eval_samples(Rg, Xg, lam, prec, **kw)
    saa.saa_ctx_sync()
    return {k: out[k].cpu().numpy() for k in ("f", "pbar", "var")}


@pytest.mark.parametrize("d,N,K", [(4, 2, 1), (32, 1000, 17), (36, 1000, 3), (100, 9_999, 33), (64, 128, 64),
                                   (64, 129, 5), (128, 10_000, 256), (256, 3_000, 128)])
@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
@pytest.mark.parametrize("centred", [True, False])
def test_streamed_parity(d, N, K, prec, centred):
    R, inst = inputs.sample_matrix(N, d, seed=d + N)
    X = inputs.decisions(K, d, seed=d)
    out = _run(R, X, prec, centred)
    ref = oracle.saa_explicit(R.astype(np.float64), X, LAM)
    e = {k: _err(out[k], ref, k) for k in ("f", "pbar")}
    e_v = LAM * float(np.max(np.abs(out["var"] - ref["var"]) / (LAM * ref["var"] + np.abs(ref["pbar"]))))
    cond = 1.0 if centred else 1.0 + float(np.max(ref["pbar"] ** 2 / ref["var"]))
    print(f"{prec} d={d} N={N} K={K} centred={centred}: f {e['f']:.2e} pbar {e['pbar']:.2e} var {e_v:.2e} "
          f"cond {cond:.2f}")
    tol = TOL[prec] * cond
    assert e["f"] <= tol and e["pbar"] <= tol and e_v <= tol


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_streamed_heavy_tails(prec):
    R, inst = inputs.sample_matrix(20_000, 128, seed=5, heavy=True)
    X = inputs.decisions(64, 128, seed=5)
    out = _run(R, X, prec)
    ref = oracle.saa_explicit(R.astype(np.float64), X, LAM)
    assert _err(out["f"], ref, "f") <= TOL[prec] and _err(out["pbar"], ref, "pbar") <= TOL[prec]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3"])
def test_streamed_full_size_sampled_decisions(prec):
    d, N, K = 128, 1 << 20, 256
    R, inst = inputs.sample_matrix(N, d, seed=0, heavy=True)
    X = inputs.decisions(K, d, seed=0)
    out = _run(R, X, prec)
    pick = [0, 131, 255]
    ref = oracle.saa_explicit(R.astype(np.float64), X[pick], LAM)
    sub = {k: v[pick] for k, v in out.items()}
    assert _err(sub["f"], ref, "f") <= TOL[prec] and _err(sub["pbar"], ref, "pbar") <= TOL[prec]


def test_streamed_deterministic_and_centre_free():
    from paper_2404_11631_gb300 import saa
    R, inst = inputs.sample_matrix(50_000, 128, seed=9)
    X = torch.tensor(inputs.decisions(100, 128, seed=9), device="cuda")
    Rg = torch.from_numpy(R).cuda()
    mu = torch.tensor(inst.mu, device="cuda")
    sd = torch.tensor(np.sqrt(np.diag(inst.sigma)), device="cuda")
    a = saa.saa_eval_samples(Rg, X, LAM, "f16x3", center=mu, sigma=sd)
    b = saa.saa_eval_samples(Rg, X, LAM, "f16x3", center=mu, sigma=sd)
    c = saa.saa_eval_samples(Rg, X, LAM, "f16x3", center=torch.zeros_like(mu))
    saa.saa_ctx_sync()
    assert torch.equal(a["f"], b["f"]) and torch.equal(a["var"], b["var"])
    ref = oracle.saa_explicit(R.astype(np.float64), X.cpu().numpy(), LAM)
    cond = 1.0 + float(np.max(ref["pbar"] ** 2 / ref["var"]))
    assert _err(a["f"].cpu().numpy(), ref, "f") <= TOL["f16x3"]
    assert _err(c["f"].cpu().numpy(), ref, "f") <= TOL["f16x3"] * cond


def test_streamed_matches_regenerated_samples():
    # the generator's own FP32 samples, streamed, against the in-kernel
    # regenerated estimate of the same scenarios (both CUDA paths: the
    # samples differ by their FP32 rounding only)
    from paper_2404_11631_gb300 import saa
    d, N, K = 128, 1 << 17, 64
    gp, op, inst = make(d, N, law=oracle.LAW_MIX, seed=4)
    X = torch.tensor(inputs.decisions(K, d, seed=4), device="cuda")
    xi = saa.saa_generate(gp, 0, N, "fp32", want_xi=True)["xi"]
    s = saa.saa_eval_samples(xi, X, gp.lam, "f16x3", center=gp.mu)
    g = saa.saa_eval(gp, X, "f16x3")
    saa.saa_ctx_sync()
    scale = gp.lam * g["var"] + g["pbar"].abs()
    assert ((s["f"] - g["f"]).abs() / scale).max().item() <= 1e-5


def test_streamed_scaling_keeps_bf16_exact_range():
    # a tiny sigma scales the columns up by 2^19: BF16 has FP32's range, so
    # the result is unchanged; at F16X3 the same scaling leaves FP16's range
    # and is reported on the next sync
    from paper_2404_11631_gb300 import saa
    R, inst = inputs.sample_matrix(4000, 64, seed=2)
    X = inputs.decisions(8, 64, seed=2)
    Rg, Xg = torch.from_numpy(R).cuda(), torch.tensor(X, device="cuda")
    tiny = torch.full((64,), 1e-6, dtype=torch.float64, device="cuda")
    mu = torch.tensor(R.astype(np.float64).mean(axis=0), device="cuda")
    out = saa.saa_eval_samples(Rg, Xg, LAM, "bf16x3", center=mu, sigma=tiny)
    saa.saa_ctx_sync()
    ref = oracle.saa_explicit(R.astype(np.float64), X, LAM)
    assert _err(out["f"].cpu().numpy(), ref, "f") <= TOL["bf16x3"]
    saa.saa_eval_samples(Rg, Xg, LAM, "f16x3", center=mu, sigma=tiny)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()


def test_streamed_rejects_bad_arguments():
    from paper_2404_11631_gb300 import saa
    R = torch.zeros(100, 8, dtype=torch.float32, device="cuda")
    X = torch.zeros(2, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(saa.SAAError):
        saa.saa_eval_samples(R, X, LAM, "fp32")                                      # tensor cores only
    with pytest.raises(saa.SAAError):
        saa.saa_eval_samples(R[:, :6].contiguous(), X[:, :6].contiguous(), LAM)      # d % 4
    with pytest.raises(saa.SAAError):
        saa.saa_eval_samples(R, torch.zeros(257, 8, dtype=torch.float64, device="cuda"), LAM)   # K > 256
    with pytest.raises(saa.SAAError):
        saa.saa_eval_samples(torch.zeros(10, 260, dtype=torch.float32, device="cuda"),
                             torch.zeros(1, 260, dtype=torch.float64, device="cuda"), LAM)      # d > 256
    bad = torch.ones(8, dtype=torch.float64, device="cuda")
    bad[3] = 0.0
    saa.saa_eval_samples(R, X, LAM, "bf16x3", sigma=bad)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()
