"""Algorithm 3 (stochastic quasi-Newton for the binary-classification task of
Sec. 3.3) and Algorithm 4 (its inverse-Hessian update), as host
orchestration around the device kernels.

Per iteration k the mini-batch gradient over a sample S of b points comes
from the device (`saa_logistic_eval` through the callables below); the
first 2L iterations take plain stochastic-gradient steps w <- w - (beta/k) g,
later ones w <- w - (beta/k) H_t g.  Every L iterations the average of the
last L iterates closes a block; from the second block on, the correction
pair is s_t = (difference of the last two block averages) and
y_t = (sub-sampled Hessian over b_H points at the newest average) s_t, the
Hessian product again from the device.

Algorithm 4 builds H_t from H = (s_t'y_t / y_t'y_t) I by the BFGS update
with the last min(t, M) pairs, oldest first.  Only H_t g is ever needed, and
the two-loop recursion computes that product from the same pairs and the
same initial scaling in O(M n) (identical in exact arithmetic; the dense n x n
update would cost O(M n^2) per iteration).  These O(M n) vector steps run in
numpy on the host; the data-parallel parts (the sample averages over the
data set) run in the CUDA kernels.

Readings: the paper's "sample sets" are uniform draws with replacement
(the caller's generator); the block average that the correction pairs use is
kept while the next block accumulates (the reset clears the accumulator).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np


def two_loop(g: np.ndarray, pairs: list[tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """H g for the BFGS inverse-Hessian of Algorithm 4: initial matrix
    (s'y / y'y) I from the newest pair, then the updates with `pairs`
    (oldest first).  Pairs with s'y <= 0 must not be passed."""
    q = np.array(g, dtype=np.float64, copy=True)
    alphas = []
    for s, y in reversed(pairs):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        alphas.append((rho, a))
        q -= a * y
    s_t, y_t = pairs[-1]
    r = (float(s_t @ y_t) / float(y_t @ y_t)) * q
    for (s, y), (rho, a) in zip(pairs, reversed(alphas)):
        bcoef = rho * float(y @ r)
        r += (a - bcoef) * s
    return r


def dense_h(pairs: list[tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """Algorithm 4 written out densely (n x n): for checking two_loop."""
    s_t, y_t = pairs[-1]
    n = s_t.size
    H = (float(s_t @ y_t) / float(y_t @ y_t)) * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / float(y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@dataclass
class SQNResult:
    w: np.ndarray
    pairs_used: int
    skipped_pairs: int
    w_trace: list = field(default_factory=list)


def sqn(grad: Callable[[np.ndarray, np.ndarray], np.ndarray],
        hvp: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray],
        w0: np.ndarray, N: int, iters: int, L: int = 10, M: int = 25, beta: float = 2.0, b: int = 50,
        b_H: int = 600, rng: np.random.Generator | None = None, trace_every: int = 0) -> SQNResult:
    """Algorithm 3 for `iters` iterations from w0.

    grad(w, idx)   -> mini-batch gradient of F at w over rows idx (int64 [b])
    hvp(w, v, idx) -> sub-sampled Hessian of F at w times v over rows idx
    A pair whose curvature s'y is not positive (possible only through
    rounding, the sub-sampled Hessian being positive semi-definite) is not
    stored; the count is returned."""
    rng = np.random.default_rng(0) if rng is None else rng
    w = np.array(w0, dtype=np.float64, copy=True)
    acc = np.zeros_like(w)
    prev_avg = None
    pairs: list[tuple[np.ndarray, np.ndarray]] = []
    skipped = 0
    trace = []
    for k in range(1, iters + 1):
        idx = rng.integers(0, N, size=b)
        g = grad(w, idx)
        acc += w
        alpha = beta / k
        if k <= 2 * L or not pairs:
            w = w - alpha * g
        else:
            w = w - alpha * two_loop(g, pairs[-M:])
        if k % L == 0:
            avg = acc / L
            if prev_avg is not None:
                s = avg - prev_avg
                y = hvp(avg, s, rng.integers(0, N, size=b_H))
                if float(s @ y) > 0.0:
                    pairs.append((s, y))
                    pairs = pairs[-M:]
                else:
                    skipped += 1
            prev_avg = avg
            acc = np.zeros_like(w)
        if trace_every and k % trace_every == 0:
            trace.append(w.copy())
    return SQNResult(w=w, pairs_used=len(pairs), skipped_pairs=skipped, w_trace=trace)


def device_callables(X, z, n: int):
    """grad and hvp callables of `sqn` over a device data set (the feature
    bits X and labels z of `saa_logistic_generate`), evaluated by the CUDA
    kernels; vectors cross the host boundary as float64 [n]."""
    import torch

    from . import saa
    dev = X.device

    def grad(w, idx):
        out = saa.saa_logistic_eval(X, z, n, torch.tensor(w[None], device=dev),
                                    idx=torch.tensor(idx, dtype=torch.int64, device=dev))
        return out["grad"][0].cpu().numpy()

    def hvp(w, v, idx):
        out = saa.saa_logistic_eval(X, z, n, torch.tensor(w[None], device=dev), torch.tensor(v[None], device=dev),
                                    idx=torch.tensor(idx, dtype=torch.int64, device=dev))
        return out["hvp"][0].cpu().numpy()

    return grad, hvp
