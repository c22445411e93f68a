"""torch.autograd.Function around sv_adjoint_grad.

Forward returns f_b = <0|U^dag(theta_b) H U(theta_b)|0> for each row of a
(batch, n_params) parameter tensor; the library computes the gradients in the
same call (adjoint sweep, no tape), and backward scales them by the upstream
gradient: d loss / d theta_b = (d loss / d f_b) * grad_b.  This is the
batched-template, per-parameter-gradient path of the paper's QML layers
(Sec. 8.2), with the adjoint in place of autograd through every gate.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class AdjointExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, n, dtype, gates, terms, checkpoint_every):
        p = params.detach().to("cpu", torch.float64).numpy()
        val, grad = B.sv_adjoint_grad(n, dtype, gates, p, terms, checkpoint_every)
        ctx.save_for_backward(torch.from_numpy(grad).to(params.device, params.dtype))
        return torch.from_numpy(val).to(params.device, params.dtype)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout.unsqueeze(-1) * grad, None, None, None, None, None


def adjoint_expectation(params: torch.Tensor, n: int, gates, terms, dtype: int = B.SV_C64,
                        checkpoint_every: int = 0) -> torch.Tensor:
    """Differentiable batch of expectations; params is (batch, n_params) or (n_params,)."""
    squeeze = params.dim() == 1
    p = params.unsqueeze(0) if squeeze else params
    g = gates if isinstance(gates, B.Gates) else B.Gates(gates)
    t = B.pauli_terms(terms) if not isinstance(terms, type(B.pauli_terms([]))) else terms
    out = AdjointExpectation.apply(p, n, dtype, g, t, checkpoint_every)
    return out[0] if squeeze else out
