"""torch.autograd.Function over the hand-written DPF adjoint (dpf_loss_backward).

The forward returns the batch loss  sum_k L_k  (L_k the MSE of Alg. 1 for
case k, FP64 evaluation); the backward returns, scaled by the incoming
gradient, dL/dtheta and dL/d|V| (zero at non-learnable entries), dL/dP_spec,
dL/dQ_spec and the branch gradients dL/dg, dL/db of the series admittance --
all from the CUDA kernels; PyTorch only routes the tensors.
"""
from __future__ import annotations

import torch

from . import _abi
from .dpf import Workspace, Ybus, dpf_loss_backward


class DPFLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, va, vm, p_spec, q_spec, g_series, b_series, ybus: Ybus, ws: Workspace,
                precision: int = _abi.FP32):
        want = ["loss", "d_va", "d_vm", "d_p", "d_q"]
        if g_series is not None:
            want += ["d_g", "d_b"]
        out = dpf_loss_backward(ybus, ws, va.detach().contiguous(), vm.detach().contiguous(),
                                None if p_spec is None else p_spec.detach().contiguous(),
                                None if q_spec is None else q_spec.detach().contiguous(),
                                g_series=None if g_series is None else g_series.detach().contiguous(),
                                b_series=None if b_series is None else b_series.detach().contiguous(),
                                precision=precision, want=want)
        ctx.grads = out
        ctx.has_spec = p_spec is not None
        ctx.has_branch = g_series is not None
        return out["loss"].sum()

    @staticmethod
    def backward(ctx, grad):
        o = ctx.grads
        g = grad.to(torch.float64)
        gp = g * o["d_p"] if ctx.has_spec else None
        gq = g * o["d_q"] if ctx.has_spec else None
        gg = g * o["d_g"] if ctx.has_branch else None
        gb = g * o["d_b"] if ctx.has_branch else None
        return g * o["d_va"], g * o["d_vm"], gp, gq, gg, gb, None, None, None


def dpf_loss(va, vm, ybus, ws, p_spec=None, q_spec=None, g_series=None, b_series=None, precision=_abi.FP32):
    """Differentiable batch loss sum_k L_k."""
    return DPFLoss.apply(va, vm, p_spec, q_spec, g_series, b_series, ybus, ws, precision)
