"""Branch-parameter identification by gradient descent on the power mismatch.

The paper motivates DPF by end-to-end gradients from the power mismatches to
the simulation parameters, which "allows these parameters to be identified"
(abstract, Sec. 1), without an experiment.  Here: given K measured operating
points (V = |V| e^{j theta} and the injections P, Q at every bus), the series
admittances g + jb of every branch are adjusted by Adam to minimise the sum
over operating points of the DPF loss of Alg. 1 at those fixed voltages.
The operating points are staged once (dpf_paramid_begin); each step takes
the branch gradient from dpf_paramid_step (Y values rebuilt by k_ybus_values,
forward pass, branch adjoint k_edge_grad) and the step from dpf_adam_update;
the learning rate of each parameter is scaled by its starting magnitude, so a
step is a relative change of about `lr`.
"""
from __future__ import annotations

import torch

from . import _abi
from .dpf import Workspace, Ybus, dpf_adam_update, dpf_paramid_begin, dpf_paramid_step


def identify_branches(y: Ybus, ws: Workspace, va, vm, p, q, g0, b0, iters: int, lr: float = 3e-3,
                      betas=(0.9, 0.999), precision=_abi.FP32, record_every: int = 0, stream=None):
    """Returns (g, b, history); g0, b0 are [M] float64 CUDA tensors, the others [K][N]."""
    g = g0.clone()
    b = b0.clone()
    mg, vg, mb, vb = (torch.zeros_like(g0) for _ in range(4))
    sg, sb = g0.abs(), b0.abs()
    hist = []
    dpf_paramid_begin(y, ws, va, vm, p, q, precision=precision, stream=stream)
    bufs = {}
    for t in range(1, iters + 1):
        want = ("d_g", "d_b", "loss") if (record_every and t % record_every == 0) else ("d_g", "d_b")
        out = dpf_paramid_step(y, ws, g, b, want=want, out=bufs, stream=stream)
        bufs.update(out)
        if "loss" in out:
            hist.append((t, float(out["loss"].sum().item())))
        dpf_adam_update(g, out["d_g"], mg, vg, t, lr, betas[0], betas[1], lr_scale=sg, stream=stream)
        dpf_adam_update(b, out["d_b"], mb, vb, t, lr, betas[0], betas[1], lr_scale=sb, stream=stream)
    return g, b, hist
