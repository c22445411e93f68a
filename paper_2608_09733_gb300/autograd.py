"""torch.autograd.Function around the adjoint gradient.

Forward returns f_b = <0|U^dag(theta_b) H U(theta_b)|0> for each row of a
(batch, n_params) parameter tensor.  When the parameters need a gradient the
library computes it in the same call (adjoint sweep, no tape) and backward
scales it by the upstream gradient: d loss / d theta_b = (d loss / d f_b) *
grad_b; otherwise only the values are computed (forward pass and H psi, no
reverse pass).  CUDA parameter tensors go through the device-array entry
points: parameters, gradients and values stay on the GPU, and no host copy
sits on the step.  This is the batched-template, per-parameter-gradient path
of the paper's QML layers (Sec. 8.2), with the adjoint in place of autograd
through every gate.
"""

from __future__ import annotations

from collections import namedtuple

import numpy as np
import torch

from . import binding as B


class AdjointExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, n, dtype, gates, terms, checkpoint_every):
        want_grad = ctx.needs_input_grad[0]
        if params.is_cuda:
            p = params.detach().to(torch.float64).contiguous()
            val, grad = B.sv_adjoint_grad_device(n, dtype, gates, p, terms, checkpoint_every=checkpoint_every,
                                                 values_only=not want_grad)
        else:
            p = params.detach().to(torch.float64).numpy()
            v, g = B.sv_adjoint_grad(n, dtype, gates, p, terms, checkpoint_every)
            val, grad = torch.from_numpy(v), torch.from_numpy(g)
        if want_grad:
            ctx.save_for_backward(grad.to(params.dtype))
        return val.to(params.dtype)

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


_Term = namedtuple("_Term", "paulis qubits coeff")


class _BatchLayerFn(torch.autograd.Function):
    """Forward: <Z_q> of every qubit for every input row (one batched
    forward pass).  Backward: one batched adjoint pass whose Hamiltonian for
    row b is sum_q (dL/d<Z_q>_b) Z_q, which gives dL/dtheta_b directly."""

    @staticmethod
    def forward(ctx, x, w, n, dtype, gates, checkpoint_every):
        dev = x.device if x.is_cuda else torch.device("cpu")
        xb = x.detach().to(dev, torch.float64)
        wb = w.detach().to(dev, torch.float64).reshape(1, -1).expand(xb.shape[0], -1)
        params = torch.cat([xb, wb], dim=1).contiguous()
        if params.is_cuda:  # the parameters stay on the device
            z = B.sv_batch_expect_z_device(n, dtype, gates, params)[:, :n]
        else:
            z = torch.from_numpy(B.sv_batch_expect_z(n, dtype, gates, params.numpy())[:, :n])
        ctx.params, ctx.n, ctx.dtype, ctx.gates, ctx.ckpt = params, n, dtype, gates, checkpoint_every
        ctx.n_data = x.shape[1]
        ctx.devices = (x.device, x.dtype, w.device, w.dtype)
        return z.to(x.device, x.dtype)

    @staticmethod
    def backward(ctx, gz):
        n = ctx.n
        terms = B.pauli_terms([_Term("Z", [q], 1.0) for q in range(n)])
        xdev, xdt, wdev, wdt = ctx.devices
        if ctx.params.is_cuda:  # upstream gradient, gradients and the weight sum on the device
            coeffs = gz.detach().to(ctx.params.device, torch.float64).contiguous()
            _, g = B.sv_adjoint_grad_device(n, ctx.dtype, ctx.gates, ctx.params, terms, row_coeffs=coeffs,
                                            checkpoint_every=ctx.ckpt)
        else:
            coeffs = gz.detach().to("cpu", torch.float64).contiguous().numpy()
            _, grad = B.sv_adjoint_grad_rows(n, ctx.dtype, ctx.gates, ctx.params.numpy(), terms, coeffs, ctx.ckpt)
            g = torch.from_numpy(grad)
        dx = g[:, :ctx.n_data].to(xdev, xdt)
        dw = g[:, ctx.n_data:].sum(dim=0).to(wdev, wdt)
        return dx, dw, None, None, None, None


class BatchLayer(torch.nn.Module):
    """A fixed circuit template as a torch layer (Sec. 5.4 BatchLayer): the
    template's parameter slots 0 .. n_data-1 take each input row's data,
    slots n_data .. n_data+n_weights-1 the layer's trainable weights; the
    output is <Z_q> for every qubit of every row, (batch, n).  All rows run
    as one batched state; backward is one batched adjoint pass (no
    parameter-shift loop).  With CUDA inputs (and the layer on the GPU) the
    whole step stays in device memory.  Parameterised gates must be
    one-parameter rotations (RX, RY, RZ, P, RXX, RYY, RZZ, EXC1, EXC2)."""

    def __init__(self, gates, n_qubits: int, n_data: int, n_weights: int, dtype: int = B.SV_C64,
                 checkpoint_every: int = 0, init_scale: float = 0.1, seed: int = 0):
        super().__init__()
        self.gates = gates if isinstance(gates, B.Gates) else B.Gates(gates)
        self.n, self.n_data, self.dtype, self.ckpt = n_qubits, n_data, dtype, checkpoint_every
        gen = torch.Generator().manual_seed(seed)
        self.weight = torch.nn.Parameter(init_scale * torch.randn(n_weights, generator=gen, dtype=torch.float64))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        if x.dim() != 2 or x.shape[1] != self.n_data:
            raise ValueError("expected input rows of %d data values" % self.n_data)
        return _BatchLayerFn.apply(x, self.weight, self.n, self.dtype, self.gates, self.ckpt)
