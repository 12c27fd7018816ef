"""Algorithm 2 (Frank-Wolfe for the multi-product newsvendor of Sec. 3.2)
as host orchestration around the device's Monte Carlo gradient.

Epoch k draws fresh demand samples (the problem's epoch counter word is k)
and runs M iterations on them; iteration t = kM + m takes the gradient
estimate of Sec. 3.2 at x (from `saa_newsvendor_grad` through the callable
below), solves the linear subproblem s = argmin { s'g : A s <= C, s >= 0 }
and steps x <- x + gamma (s - x) with gamma = 2 / (t + 2).

The subproblem is a linear program, not a data-parallel step: with one
resource row it is solved exactly in O(n) (the best ratio g_j / a_j among
g_j < 0, at the vertex C / a_j on axis j, or s = 0), and with several rows
by scipy's HiGHS.  The Frank-Wolfe gap g'(x - s) >= 0 is returned per
iteration.
"""
from __future__ import annotations

from typing import Callable

import numpy as np


def lmo(g: np.ndarray, A: np.ndarray, C: np.ndarray) -> np.ndarray:
    """argmin over {s : A s <= C, s >= 0} of s'g (A [R, n] >= 0, C [R] > 0)."""
    A = np.atleast_2d(A)
    n = g.size
    if A.shape[0] == 1:
        s = np.zeros(n)
        neg = g < 0.0
        if not np.any(neg):
            return s
        ratio = np.where(neg, g / A[0], np.inf)   # cost per unit of the resource
        j = int(np.argmin(ratio))
        s[j] = C[0] / A[0, j]
        return s
    from scipy.optimize import linprog
    r = linprog(g, A_ub=A, b_ub=C, bounds=(0.0, None), method="highs")
    if r.status != 0:
        raise RuntimeError(f"linear subproblem failed: {r.message}")
    return np.asarray(r.x, dtype=np.float64)


def newsvendor_fw(grad: Callable[[np.ndarray, int], np.ndarray], A: np.ndarray, C: np.ndarray, x0: np.ndarray,
                  epochs: int, M: int) -> dict:
    """Algorithm 2 for `epochs` epochs of M iterations from x0 (x0 must satisfy
    A x0 <= C, x0 >= 0).  grad(x, k) is the gradient estimate on epoch k's
    demand samples.  Returns x and the per-iteration gap trace."""
    x = np.array(x0, dtype=np.float64, copy=True)
    gaps = []
    for k in range(epochs):
        for m in range(M):
            g = grad(x, k)
            s = lmo(g, A, C)
            gaps.append(float(g @ (x - s)))
            gamma = 2.0 / (k * M + m + 2)
            x = x + gamma * (s - x)
    return {"x": x, "gap_trace": np.array(gaps)}


def device_gradient(prob):
    """grad(x, k) of `newsvendor_fw` evaluated by the CUDA kernel on epoch
    k's demand samples; prob is a `saa.Newsvendor` (its epoch is replaced)."""
    import dataclasses

    import torch

    from . import saa
    dev = prob.mu.device

    def grad(x, k):
        p = dataclasses.replace(prob, epoch=int(k))
        return saa.saa_newsvendor_grad(p, torch.tensor(x[None], device=dev))[0].cpu().numpy()

    return grad
