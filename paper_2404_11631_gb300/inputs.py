"""Seeded synthetic inputs for the mean-variance SAA workloads.

This module only draws instance parameters with numpy's seeded PCG64
generator; it holds none of the estimator's arithmetic.  Both the CUDA path
and the CPU oracle receive the arrays it returns.

Law parameters follow the mean-variance task of Sec. 3.1 (R ~ N(mu, Sigma)):

* ``instance``: mu ~ U[-1,1]^d, Sigma = L L' + 0.1 I with L_ij ~ N(0, 1/d),
  C = the lower Cholesky factor of Sigma (numpy.linalg.cholesky).
* ``paper_instance``: the setup of Sec. 4.1 for the asset task,
  mu_i ~ U(-1,1), sigma_i ~ U(0, 0.025), diagonal Sigma.
* ``decisions``: K candidate decisions x ~ U[0,1]^d.
* ``logistic_weights``: the random linear combination that labels the
  binary-classification data set (Sec. 4.1's Task 3 setup): integer weights
  in [-3, 3], so the rule is exact in any arithmetic.  ``logistic_sizes``
  lists Sec. 4.1's feature counts with N = 30 n.
* ``sample_matrix``: a materialised sample set {R_i} (FP32 rows) for the
  streamed mode, R_i = mu + C z_i with z_i drawn by numpy (standard normal,
  or Student-t with 4 degrees of freedom for the second half when
  ``heavy``).  These are plain numpy draws standing in for scenario data the
  caller already holds; they are not the estimator's in-kernel law.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LAW_GAUSS, LAW_LOGN_STD, LAW_STUDENT_T, LAW_MIX = 0, 1, 2, 3


@dataclass
class Instance:
    d: int
    mu: np.ndarray      # [d] float64
    sigma: np.ndarray   # [d, d] float64, symmetric positive definite
    chol: np.ndarray    # [d, d] float64, lower triangular, chol @ chol.T == sigma


def instance(d: int, seed: int = 0) -> Instance:
    """mu ~ U[-1,1]^d, Sigma = L L' + 0.1 I, L_ij ~ N(0, 1/d)."""
    rng = np.random.default_rng([seed, d, 1])
    mu = rng.uniform(-1.0, 1.0, size=d)
    L = rng.normal(0.0, 1.0 / np.sqrt(d), size=(d, d))
    sigma = L @ L.T + 0.1 * np.eye(d)
    sigma = 0.5 * (sigma + sigma.T)
    chol = np.linalg.cholesky(sigma)
    return Instance(d, mu, sigma, np.ascontiguousarray(chol))


def paper_assets(d: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 4.1 asset setup as (mu, sd): mu_i ~ U(-1,1), sigma_i ~ U(0,0.025),
    independent assets (Sigma = diag(sd^2)); no d x d matrix is formed."""
    rng = np.random.default_rng([seed, d, 2])
    mu = rng.uniform(-1.0, 1.0, size=d)
    sd = rng.uniform(0.0, 0.025, size=d)
    return mu, np.maximum(sd, 1e-6)


def paper_instance(d: int, seed: int = 0) -> Instance:
    """The assets of :func:`paper_assets` with dense Sigma and C."""
    mu, sd = paper_assets(d, seed)
    return Instance(d, mu, np.diag(sd * sd), np.diag(sd))


def decisions(K: int, d: int, seed: int = 0) -> np.ndarray:
    """K candidate decisions x ~ U[0,1]^d, row-major [K, d]."""
    rng = np.random.default_rng([seed, d, K, 3])
    return rng.uniform(0.0, 1.0, size=(K, d))


def sample_matrix(N: int, d: int, seed: int = 0, inst_seed: int = 0, heavy: bool = False,
                  chunk: int = 1 << 16) -> tuple[np.ndarray, Instance]:
    """(R [N, d] float32 row-major, the Instance whose mu and C shaped it)."""
    inst = instance(d, inst_seed)
    rng = np.random.default_rng([seed, N, d, 4])
    R = np.empty((N, d), dtype=np.float32)
    for i0 in range(0, N, chunk):
        n = min(chunk, N - i0)
        z = rng.standard_normal((n, d))
        if heavy:
            tail = np.arange(i0, i0 + n) >= N // 2
            z[tail] = rng.standard_t(4.0, size=(int(tail.sum()), d))
        R[i0:i0 + n] = inst.mu + z @ inst.chol.T
    return R, inst


def logistic_weights(n: int, seed: int = 0) -> np.ndarray:
    """Integer weights w* in [-3, 3]^n of the labelling rule z = [2 x'w* > 1'w*]."""
    rng = np.random.default_rng([seed, n, 5])
    return rng.integers(-3, 4, size=n).astype(np.int32)


def logistic_sizes() -> list[tuple[int, int]]:
    """(n, N) of Sec. 4.1's binary-classification runs: n features, N = 30 n points."""
    return [(n, 30 * n) for n in (50, 500, 1000, 5000)]


def fw_start(d: int) -> np.ndarray:
    """Starting point w0 = (0.5/d) 1, an interior point of W = {w >= 0, 1'w <= 1}."""
    return np.full(d, 0.5 / d)


@dataclass
class RaggedBatch:
    d: np.ndarray        # [B] int
    N: np.ndarray        # [B] int
    K: np.ndarray        # [B] int
    seeds: np.ndarray    # [B] uint64 Philox seeds
    instances: list = field(default_factory=list)   # Instance per problem
    X: list = field(default_factory=list)           # [K_b, d_b] decisions per problem


def ragged_batch(B: int, seed: int = 0, d_range=(8, 512), logN_range=(3.0, 5.0), K_range=(1, 16),
                 materialise: bool = True) -> RaggedBatch:
    """B independent instances: d ~ U{d_range}, N = floor(10^U[logN_range]), K ~ U{K_range}."""
    rng = np.random.default_rng([seed, B, 4])
    d = rng.integers(d_range[0], d_range[1] + 1, size=B)
    N = np.floor(10.0 ** rng.uniform(logN_range[0], logN_range[1], size=B)).astype(np.int64)
    K = rng.integers(K_range[0], K_range[1] + 1, size=B)
    seeds = rng.integers(0, 2**63, size=B, dtype=np.uint64)
    rb = RaggedBatch(d, N, K, seeds)
    if materialise:
        for b in range(B):
            rb.instances.append(instance(int(d[b]), seed=seed * 1_000_003 + b))
            rb.X.append(decisions(int(K[b]), int(d[b]), seed=seed * 1_000_003 + b))
    return rb


# Named workloads (sizes of the five configurations this library is measured on).
WORKLOADS = {
    "plain_fp64_d10": dict(d=10, N=10_000, K=1, law=LAW_GAUSS, prec="fp64"),
    "batched_d128_N1M_K256_mix": dict(d=128, N=1 << 20, K=256, law=LAW_MIX, prec="bf16x3"),
    "ragged_4096": dict(B=4096, prec="fp32"),
    "adjoint_d1024_N1M_K64": dict(d=1024, N=1 << 20, K=64, law=LAW_GAUSS, prec="bf16x3"),
    "fw_d1024_N4M_t4_T200": dict(d=1024, N=1 << 22, K=1, law=LAW_STUDENT_T, nu=4, T=200, M=1, prec="fp8x"),
}
