"""Shared test helpers: build the same seeded problem for the CUDA path and
the CPU oracle, and the error measures the parity tests use.

Tolerances (relative error, per result):
  FP32 path   <= 1e-6   (FP32 contraction, FP64 cross-block reduction)
  F16X3 path  <= 1e-6   (FP16 hi/lo split products: the decision operand is
                         represented to ~2^-22, identically for all samples)
  BF16X3 path <= 5e-5   (BF16 hi/lo: the decision operand's ~2^-16
                         representation error does not average over N)
  FP64 path   <= 1e-11  (only the summation order differs from the oracle)
Error of an estimate a against the oracle's b for decision k is
  |a - b| / max(|b|, lambda V_k + |mu'w_k|),
because f_hat and w'R_bar can be near zero while their terms are not.
Gradients use the L2 relative error ||a - b|| / ||b|| per decision.
The sample variance alone is scored as the variance term of f_hat,
  lambda |V_a - V_b| / max(|f_b|, lambda V_b + |mu'w_k|),
because an FP32 contraction's error scales with |a_i||y_k|, not with |Q_ik|:
a decision with a small variance but large y_k sees a larger relative error
in V than in f_hat.
"""
import numpy as np

import oracle
from paper_2404_11631_gb300 import inputs

TOL = {"fp32": 1e-6, "fp64": 1e-11, "f16x3": 1e-6, "bf16x3": 5e-5}
TOL_GRAD = {"fp32": 1e-6, "fp64": 1e-11, "f16x3": 1e-6, "bf16x3": 5e-5}
ORACLE_PREC = {"fp32": 32, "fp64": 64, "f16x3": 32, "bf16x3": 32}


def make(d, N, law=oracle.LAW_GAUSS, nu=4, lam=0.5, seed=0, instance=0, epoch=0, inst_seed=0, paper=False):
    """(gpu Problem, oracle problem, Instance) for the same law and stream."""
    import torch
    from paper_2404_11631_gb300 import saa
    inst = inputs.paper_instance(d, inst_seed) if paper else inputs.instance(d, inst_seed)
    mu = torch.tensor(inst.mu, dtype=torch.float64, device="cuda")
    ch = torch.tensor(inst.chol, dtype=torch.float64, device="cuda")
    gp = saa.Problem(mu=mu, chol=ch, N=N, law=law, nu=nu, lam=lam, seed=seed, instance=instance, epoch=epoch)
    op = oracle.make_problem(d, N, inst.mu, inst.chol, law=law, nu=nu, lam=lam, seed=seed, instance=instance,
                             epoch=epoch)
    return gp, op, inst


def est_err(a, b, var, X, mu, lam):
    scale = np.maximum(np.abs(b), lam * var + np.abs(X @ mu))
    return np.max(np.abs(a - b) / scale)


def var_err(va, vb, fb, X, mu, lam):
    scale = np.maximum(np.abs(fb), lam * vb + np.abs(X @ mu))
    return np.max(lam * np.abs(va - vb) / scale)


def grad_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1))
