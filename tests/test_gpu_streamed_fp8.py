"""Streamed mode at SAA_FP8X: the E4M3 contraction (samples split hi + lo,
decisions in three terms, four products on kind::f8f6f4) against the
oracle's Eq. 4 on the same FP32 samples (oracle.saa_explicit).

Two kinds of check.  From N of a few thousand the estimates are held to
1e-4 (the precision target of the FP8 contraction): the sample-side rounding,
2^-8 of each element, changes sign from scenario to scenario and averages out
of V, and the decision side, whose rounding is shared by every scenario, is
kept in three terms (2^-12).  At any N, including N = 2, every result is held
to an a-priori rounding bound computed from the samples: per element
|delta(v y)| <= eps |v| |y| plus E4M3's subnormal spacing, with eps = 1.5 2^-7
covering the split residuals and the omitted A2 (B2 + B3), summed over the
dimensions, carried through V and f, plus the FP32 accumulation of the tensor
pipe.  A wrong operand layout or a missing product breaks one or both."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu
LAM = 0.5
TOL_FP8 = 1e-4


def _err(a, ref, key):
    scale = np.maximum(np.abs(ref[key]), LAM * ref["var"] + np.abs(ref["pbar"]))
    return float(np.max(np.abs(a - ref[key]) / scale))


def _spread(R):
    return R.astype(np.float64).std(axis=0) + 1e-30


def _run(R, X, center=True, sigma=True, lam=LAM):
    from paper_2404_11631_gb300 import saa
    Rg = torch.from_numpy(R).cuda()
    Xg = torch.tensor(X, device="cuda")
    kw = {}
    if center:
        kw["center"] = torch.tensor(R.astype(np.float64).mean(axis=0), device="cuda")
    if sigma:
        kw["sigma"] = torch.tensor(_spread(R), device="cuda")
    out = saa.saa_eval_samples(Rg, Xg, lam, "fp8x", **kw)
    saa.saa_ctx_sync()
    return {k: out[k].cpu().numpy() for k in ("f", "pbar", "var")}


def _a_priori_bound(R, X, lam=LAM):
    """Bound on |f - f_ref| per decision from the rounding analysis of the
    E4M3 split (see the module docstring), in the original units.  The kernel
    forms V = (S2 - S1^2 / N) / (N - 1) with S1 from the FP32 column sums, so
    the split's error enters through S2 = sum_i Q_i^2 alone."""
    N, d = R.shape
    c = R.astype(np.float64).mean(axis=0).astype(np.float32).astype(np.float64)
    D = R.astype(np.float64) - c                         # the centred samples
    sig = _spread(R)
    a = np.ceil(np.log2(sig))                            # 2^(a-1) < sigma <= 2^a
    nkb = (d + 63) // 64
    eps = 1.5 * 2.0 ** -7
    absv = 2.0 ** -9 * np.exp2(a)                        # E4M3 subnormal spacing of v, in R's units
    M = np.max(np.abs(X) * np.exp2(a), axis=1)           # largest scaled decision entry, per decision
    absd = 2.0 ** -16 * ((np.abs(D) * np.exp2(-a)).sum(axis=1)[:, None] * M[None, :])
    DX = np.abs(D) @ np.abs(X).T
    E = eps * DX + absv @ np.abs(X).T + absd             # [N, K] bound on |delta Q_ik|
    E += 2.0 * (8 * nkb + 32) * 2.0 ** -23 * DX          # FP32 accumulation in TMEM
    Q = D @ X.T
    dV = (2.0 * np.sum(np.abs(Q) * E, axis=0) + np.sum(E * E, axis=0)) / (N - 1)
    ref = oracle.saa_explicit(R.astype(np.float64), X, lam)
    scale = lam * ref["var"] + np.abs(ref["pbar"])
    return lam * dV + 1e-6 * scale, ref


@pytest.mark.parametrize("d,N,K", [(32, 1 << 14, 17), (36, 20_000, 3), (100, 1 << 14, 33), (64, 1 << 14, 64),
                                   (128, 1 << 15, 256), (256, 1 << 14, 128)])
@pytest.mark.parametrize("heavy", [False, True])
def test_fp8_streamed_parity(d, N, K, heavy):
    R, inst = inputs.sample_matrix(N, d, seed=d + N, heavy=heavy)
    X = inputs.decisions(K, d, seed=d)
    out = _run(R, X)
    ref = oracle.saa_explicit(R.astype(np.float64), X, LAM)
    e = {k: _err(out[k], ref, k) for k in ("f", "pbar")}
    e_v = LAM * float(np.max(np.abs(out["var"] - ref["var"]) / (LAM * ref["var"] + np.abs(ref["pbar"]))))
    print(f"fp8x d={d} N={N} K={K} heavy={heavy}: f {e['f']:.2e} pbar {e['pbar']:.2e} var {e_v:.2e}")
    assert e["f"] <= TOL_FP8 and e["pbar"] <= TOL_FP8 and e_v <= TOL_FP8


@pytest.mark.parametrize("d,N,K", [(4, 2, 1), (32, 1000, 17), (36, 1000, 3), (64, 128, 64), (64, 129, 5),
                                   (100, 9_999, 33), (256, 3_000, 128)])
def test_fp8_streamed_within_rounding_bound(d, N, K):
    R, inst = inputs.sample_matrix(N, d, seed=d + N)
    X = inputs.decisions(K, d, seed=d)
    out = _run(R, X)
    bound, ref = _a_priori_bound(R, X)
    err = np.abs(out["f"] - ref["f"])
    print(f"fp8x d={d} N={N} K={K}: max err / bound {float(np.max(err / bound)):.3f}")
    assert np.all(err <= bound)


def test_fp8_streamed_full_size_sampled_decisions():
    d, N, K = 128, 1 << 20, 256
    R, inst = inputs.sample_matrix(N, d, seed=0, heavy=True)
    X = inputs.decisions(K, d, seed=0)
    out = _run(R, X)
    pick = [0, 131, 255]
    ref = oracle.saa_explicit(R.astype(np.float64), X[pick], LAM)
    sub = {k: v[pick] for k, v in out.items()}
    assert _err(sub["f"], ref, "f") <= TOL_FP8 and _err(sub["pbar"], ref, "pbar") <= TOL_FP8


def test_fp8_streamed_deterministic():
    R, inst = inputs.sample_matrix(20_000, 128, seed=3)
    X = inputs.decisions(40, 128, seed=3)
    a, b = _run(R, X), _run(R, X)
    assert all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("center,sigma", [(False, True), (True, False), (False, False)])
def test_fp8_needs_center_and_sigma(center, sigma):
    from paper_2404_11631_gb300 import saa
    R, inst = inputs.sample_matrix(1000, 32, seed=1)
    X = inputs.decisions(4, 32, seed=1)
    with pytest.raises(saa.SAAError) as e:
        _run(R, X, center=center, sigma=sigma)
    assert e.value.status == saa.SAA_EINVAL


def test_fp8_range_violation_is_reported():
    # a spread 2^12 below the samples' own puts |R - c| 2^-a far above E4M3's
    # 448: flagged by the converters, reported by the next sync
    from paper_2404_11631_gb300 import saa
    R, inst = inputs.sample_matrix(4000, 64, seed=2)
    X = inputs.decisions(8, 64, seed=2)
    Rg, Xg = torch.from_numpy(R).cuda(), torch.tensor(X, device="cuda")
    mu = torch.tensor(R.astype(np.float64).mean(axis=0), device="cuda")
    small = torch.tensor(_spread(R) * 2.0 ** -12, device="cuda")
    saa.saa_eval_samples(Rg, Xg, LAM, "fp8x", center=mu, sigma=small)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_EDEVICE
    saa.saa_ctx_sync()


def test_fp8_regenerated_entry_points_refuse_it():
    # the C call returns SAA_EUNSUPPORTED (test_gpu_errors); the binding's
    # workspace query fails first and carries the library's reason
    from helpers import make
    from paper_2404_11631_gb300 import saa
    gp, op, inst = make(16, 1000)
    X = torch.tensor(inputs.decisions(2, 16, seed=0), device="cuda")
    with pytest.raises(saa.SAAError, match="streamed mode only"):
        saa.saa_eval(gp, X, "fp8x")
