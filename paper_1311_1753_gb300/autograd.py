"""torch.autograd wrapper of the fused NLL + gradient evaluation.

``nll(ctx, theta)`` returns the negative log-likelihood as a 0-d tensor whose backward
pass uses the gradient the library computed in the same event pass (no extra device
work in backward).  theta is a 1-d float64 tensor of the free parameters (gf_free_params
order); any torch optimiser can then drive the fit.
"""
from __future__ import annotations

import numpy as np
import torch


class GooNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, theta: torch.Tensor, gctx):
        th = theta.detach().to("cpu", torch.float64).numpy()
        f, g = gctx.nll_grad(np.ascontiguousarray(th))
        ctx_.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(f, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx_, grad_out):
        (g,) = ctx_.saved_tensors
        return grad_out * g, None


def nll(gctx, theta: torch.Tensor) -> torch.Tensor:
    return GooNLL.apply(theta, gctx)
