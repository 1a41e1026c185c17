"""The DPF loop (Alg. 1), plain FP64 (oracle; test infrastructure).

Per iteration (Alg. 1): S_calc <- V (Y V)^*; out/target; loss = MSE;
gradient of the loss w.r.t. the learnables theta[pv,pq], |V|[pq];
optimizer.step(); scheduler.step(); stop test.

Readings where Alg. 1 is silent or loose:
  * initialisation "V <- ones" is the flat start: theta = 0 except the slack's
    set angle, |V| = set-point at pv and slack buses, 1 at pq buses;
  * the stop test is the max-abs FP64 mismatch max|f| <= tol, evaluated on the
    current iterate before its update, every `check_every` iterations (t = 0,
    k, 2k, ...); a converged case returns that iterate and the number of
    optimizer steps taken so far;
  * after max_iter steps the final iterate is evaluated once more; it counts as
    converged if it meets tol;
  * the scheduler receives the loss of the iterate the step was taken from.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .gradient import loss_grad
from .optim import SGD, Adam, ConstantLR, ReduceLROnPlateau, RMSprop, StepLR
from .power import PQ, PV, SLACK, learnable_sets, mismatch

CONVERGED, MAX_ITER, DIVERGED = 0, 1, 2


@dataclasses.dataclass
class DPFOptions:
    lr: float = 1e-2
    optimizer: str = "adam"  # "adam" | "sgd" | "rmsprop" (the optimisers of Sec. 5.3)
    momentum: float = 0.0  # SGD
    alpha: float = 0.99  # RMSprop
    beta1: float = 0.979  # Table 2
    beta2: float = 0.963
    eps: float = 1e-8
    sched: str = "plateau"  # "plateau" | "step" | "const"
    factor: float = 0.547  # Table 2 plateau parameters
    patience: int = 41
    threshold: float = 0.0673
    cooldown: int = 97
    min_lr: float = 0.0
    step_size: int = 100  # Table 3 StepLR parameters
    gamma: float = 0.773
    max_iter: int = 1000
    tol: float = 1e-6
    check_every: int = 1


def flat_start(bus_type, vm_set, va_slack=0.0):
    """Flat start (reading of Alg. 1's initialisation)."""
    bus_type = np.asarray(bus_type)
    n = bus_type.size
    va = np.zeros(n)
    va[bus_type == SLACK] = va_slack
    vm = np.ones(n)
    fixed = (bus_type == PV) | (bus_type == SLACK)
    vm[fixed] = np.asarray(vm_set, np.float64)[fixed]
    return va, vm


def dpf_solve(Y, p_spec, q_spec, bus_type, vm_set, opts: DPFOptions,
              va0=None, vm0=None, va_slack=0.0, history=False):
    """Run Alg. 1.  Returns dict(va, vm, iters, status, max_mismatch, loss)."""
    bus_type = np.asarray(bus_type)
    fva, fvm = flat_start(bus_type, vm_set, va_slack)
    va = fva if va0 is None else np.asarray(va0, np.float64).copy()
    vm = fvm if vm0 is None else np.asarray(vm0, np.float64).copy()
    # the specified quantities are not learnable: enforce them
    fixed_vm = (bus_type == PV) | (bus_type == SLACK)
    vm[fixed_vm] = np.asarray(vm_set, np.float64)[fixed_vm]
    va[bus_type == SLACK] = va_slack
    pvpq, pq = learnable_sets(bus_type)
    npv = pvpq.size
    nx = npv + pq.size
    if opts.optimizer == "sgd":
        opt = SGD(nx, opts.lr, opts.momentum)
    elif opts.optimizer == "rmsprop":
        opt = RMSprop(nx, opts.lr, opts.alpha, opts.eps)
    else:
        opt = Adam(nx, opts.lr, (opts.beta1, opts.beta2), opts.eps)
    if opts.sched == "plateau":
        sched = ReduceLROnPlateau(opt, opts.factor, opts.patience, opts.threshold,
                                  opts.cooldown, opts.min_lr)
    elif opts.sched == "step":
        sched = StepLR(opt, opts.step_size, opts.gamma)
    else:
        sched = ConstantLR(opt)
    losses = []
    status = MAX_ITER
    iters = opts.max_iter
    for t in range(opts.max_iter):
        f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
        if not np.all(np.isfinite(f)):
            status, iters = DIVERGED, t
            break
        if t % opts.check_every == 0 and np.max(np.abs(f)) <= opts.tol:
            status, iters = CONVERGED, t
            break
        L, d_va, d_vm = loss_grad(Y, va, vm, p_spec, q_spec, bus_type)
        if history:
            losses.append(L)
        x = np.concatenate([va[pvpq], vm[pq]])
        g = np.concatenate([d_va[pvpq], d_vm[pq]])
        x = opt.step(x, g)
        va[pvpq] = x[:npv]
        vm[pq] = x[npv:]
        sched.step(L)
    f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
    mx = float(np.max(np.abs(f))) if f.size else 0.0
    if status == MAX_ITER and mx <= opts.tol:
        status = CONVERGED
    return dict(va=va, vm=vm, iters=iters, status=status, max_mismatch=mx,
                loss=float(f @ f) / max(f.size, 1), losses=losses, lr=opt.lr)
