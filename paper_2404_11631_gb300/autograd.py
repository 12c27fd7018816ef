"""torch.autograd.Function for the SAA estimate (Eq. 4, Sec. 3.1).

``SAAFunction.apply(X, problem, prec)`` returns f_hat(w_k) for the K rows of
X.  When X requires a gradient, the forward pass runs ``saa_grad``: one pass
of the sample kernel computes the value and the adjoint contraction
sum_i a_i Q_ik, so the gradient
    grad f_hat(w) = lambda 2/(N-1) sum_i (R_i - R_bar)(R_i - R_bar)'w - R_bar
is available without storing any of the N samples (they are regenerated
in-kernel).  ``backward`` scales it by the incoming gradient of each f_k.
There is no CPU fallback.
"""
from __future__ import annotations

import torch

from . import saa


class SAAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X: torch.Tensor, problem: "saa.Problem", prec: str = "fp32") -> torch.Tensor:
        Xc = X.detach().contiguous()
        if ctx.needs_input_grad[0]:
            out = saa.saa_grad(problem, Xc, prec)
            ctx.save_for_backward(out["grad"])
        else:
            out = saa.saa_eval(problem, Xc, prec, pbar=False, var=False)
        return out["f"]

    @staticmethod
    def backward(ctx, g_f: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return g_f.to(grad.dtype).unsqueeze(1) * grad, None, None


def saa_objective(X: torch.Tensor, problem: "saa.Problem", prec: str = "fp32") -> torch.Tensor:
    """Differentiable f_hat for the K decisions in X ([K, d] float64 CUDA)."""
    if X.dim() == 1:
        return SAAFunction.apply(X.unsqueeze(0), problem, prec)[0]
    return SAAFunction.apply(X, problem, prec)
