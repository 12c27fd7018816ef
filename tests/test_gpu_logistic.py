"""The binary-classification task of Sec. 3.3 on the GPU against the
oracle: the synthetic data set bit for bit (features and labels, ragged
feature counts and row offsets), then the objective, its gradient and the
sub-sampled Hessian product over full data sets and index samples (Sec.
4.1's b = 50 and b_H = 600 with repeats) for several parameter vectors,
up to the paper's largest size n = 5000, N = 150000.

Tolerances: F within 1e-6 relative; gradient and Hessian product within
2e-6 in L2 relative error per vector.  The forward contraction rounds the
parameter vectors to FP32 (relative 2^-24 per weight) and sums them in
float-float; the adjoint sums at most 128 samples per lane in FP32 before
FP64 merges."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_F, TOL_G = 1e-6, 2e-6


def _bits_to_features(Xw, n):
    w = Xw.cpu().numpy().view(np.uint32)
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(w.shape[0], -1)[:, :n].astype(np.uint8)


def _both(n, N, seed=3, instance=0, flip=oracle.LABEL_NOISE_10PCT):
    from paper_2404_11631_gb300 import saa
    w = inputs.logistic_weights(n, seed)
    gpu = saa.saa_logistic_generate(n, N, torch.tensor(w, device="cuda"), seed=seed, instance=instance, flip=flip)
    op = oracle.make_logistic(n, N, w, seed=seed, instance=instance, flip=flip)
    return gpu, op


@pytest.mark.parametrize("n", [1, 31, 32, 33, 127, 128, 129, 300, 5000])
def test_data_bit_exact(n):
    from paper_2404_11631_gb300 import saa
    N = 700
    gpu, op = _both(n, N, seed=n, instance=2)
    saa.saa_ctx_sync()
    x, z = oracle.logistic_data(op)
    assert np.array_equal(_bits_to_features(gpu["X"], n), x)
    assert np.array_equal(gpu["z"].cpu().numpy(), z)
    # padding bits and words are zero
    full = gpu["X"].cpu().numpy().view(np.uint32)
    assert np.all(((full[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(N, -1)[:, n:] == 0)


def test_data_row_offset():
    from paper_2404_11631_gb300 import saa
    n, N = 200, 1000
    w = inputs.logistic_weights(n, 1)
    part = saa.saa_logistic_generate(n, N, torch.tensor(w, device="cuda"), seed=9, i0=613, rows=100)
    saa.saa_ctx_sync()
    x, z = oracle.logistic_data(oracle.make_logistic(n, N, w, seed=9), i0=613, rows=100)
    assert np.array_equal(_bits_to_features(part["X"], n), x) and np.array_equal(part["z"].cpu().numpy(), z)


def _err(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def _check(n, N, K, idx=None, seed=3, scale=0.05):
    from paper_2404_11631_gb300 import saa
    gpu, op = _both(n, N, seed=seed)
    rng = np.random.default_rng([n, K, seed])
    W = scale * rng.normal(size=(K, n))
    V = rng.normal(size=(K, n))
    ix = None if idx is None else torch.tensor(idx, dtype=torch.int64, device="cuda")
    out = saa.saa_logistic_eval(gpu["X"], gpu["z"], n, torch.tensor(W, device="cuda"), torch.tensor(V, device="cuda"),
                                idx=ix)
    saa.saa_ctx_sync()
    ref = oracle.logistic_eval(op, W, V=V, idx=idx)
    e_f = float(np.max(np.abs(out["F"].cpu().numpy() - ref["F"]) / np.abs(ref["F"])))
    e_g = _err(out["grad"].cpu().numpy(), ref["grad"])
    e_h = _err(out["hvp"].cpu().numpy(), ref["hvp"])
    print(f"n={n} N={N} K={K} b={'all' if idx is None else len(idx)}: F {e_f:.2e} grad {e_g:.2e} hvp {e_h:.2e}")
    assert e_f <= TOL_F and e_g <= TOL_G and e_h <= TOL_G
    return out


@pytest.mark.parametrize("n,K", [(1, 1), (50, 1), (50, 3), (129, 2), (500, 5), (1000, 1)])
def test_full_data_parity(n, K):
    _check(n, 30 * n, K)


@pytest.mark.parametrize("b", [1, 50, 600, 3000])
def test_index_samples_with_repeats(b):
    n, N = 500, 15_000
    idx = np.random.default_rng(b).integers(0, N, size=b)
    if b > 1:
        idx[1] = idx[0]   # a repeat
    _check(n, N, 2, idx=idx)


def test_paper_largest_size():
    # Sec. 4.1's largest binary-classification run: n = 5000 features, N = 30 n points
    _check(5000, 150_000, 1, scale=0.02)


def test_deterministic_and_without_hvp():
    from paper_2404_11631_gb300 import saa
    n, N = 300, 9000
    gpu, op = _both(n, N, seed=11)
    W = torch.tensor(0.05 * np.random.default_rng(0).normal(size=(2, n)), device="cuda")
    a = saa.saa_logistic_eval(gpu["X"], gpu["z"], n, W)
    b = saa.saa_logistic_eval(gpu["X"], gpu["z"], n, W)
    c = saa.saa_logistic_eval(gpu["X"], gpu["z"], n, W, want_grad=False)
    saa.saa_ctx_sync()
    assert torch.equal(a["F"], b["F"]) and torch.equal(a["grad"], b["grad"]) and torch.equal(a["F"], c["F"])
    assert "hvp" not in a and "grad" not in c
    ref = oracle.logistic_eval(op, W.cpu().numpy(), want=("F", "grad"))
    assert _err(a["grad"].cpu().numpy(), ref["grad"]) <= TOL_G


def test_bad_arguments():
    from paper_2404_11631_gb300 import saa
    with pytest.raises(saa.SAAError):
        saa.saa_logistic_generate(60_000, 10, torch.zeros(60_000, dtype=torch.int32, device="cuda"))
        saa.saa_logistic_eval(torch.zeros(10, saa.lib().saa_logistic_pitch(60_000), dtype=torch.int32, device="cuda"),
                              torch.zeros(10, dtype=torch.uint8, device="cuda"), 60_000,
                              torch.zeros(1, 60_000, dtype=torch.float64, device="cuda"))


def test_sqn_on_the_device_follows_the_oracle():
    # Algorithm 3 with the device's mini-batch gradients and Hessian products
    # against the same run with the oracle's (same sample draws)
    from paper_2404_11631_gb300 import saa
    from paper_2404_11631_gb300.sqn import device_callables, sqn
    n, N, L = 100, 3000, 10
    wstar = inputs.logistic_weights(n, 4)
    gpu = saa.saa_logistic_generate(n, N, torch.tensor(wstar, device="cuda"), seed=4)
    op = oracle.make_logistic(n, N, wstar, seed=4)
    g_dev, h_dev = device_callables(gpu["X"], gpu["z"], n)
    g_or = lambda w, idx: oracle.logistic_eval(op, w[None], idx=idx, want=("F", "grad"))["grad"][0]
    h_or = lambda w, v, idx: oracle.logistic_eval(op, w[None], V=v[None], idx=idx, want=("F", "hvp"))["hvp"][0]
    a = sqn(g_dev, h_dev, np.zeros(n), N, iters=6 * L, L=L, rng=np.random.default_rng(1))
    b = sqn(g_or, h_or, np.zeros(n), N, iters=6 * L, L=L, rng=np.random.default_rng(1))
    assert a.pairs_used == b.pairs_used >= 3
    assert np.linalg.norm(a.w - b.w) <= 1e-2 * np.linalg.norm(b.w)
    F = float(oracle.logistic_eval(op, a.w[None], want=("F",))["F"][0])
    assert F < 0.8 * np.log(2.0)
