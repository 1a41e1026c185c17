"""Loss gradients (oracle; test infrastructure).

Voltage gradient.  Sec. 4.1 states that for L = 1/2 ||F||^2 the gradient is
J^T F.  With the MSE of Alg. 1, L = (1/m) f^T f, the chain rule gives
dL/dx = (2/m) J_f^T f with x = [theta(pvpq); |V|(pq)] (the learnables of
Alg. 1 and Eq. pf_optimization_problem).  J_f is built from Alg. 2's partials.

Parameter gradient.  The paper claims gradients with respect to simulation
parameters (Sec. 1, abstract) without a formula.  The oracle differentiates
S_calc directly: for a branch parameter p, dY/dp is the derivative of the
branch's pi-model block (oracle/ybus.py), dS/dp = V (dY/dp V)^*, and
dL/dp = (2/m) [sum_{pvpq} dP_i (Re dS_i/dp) + sum_{pq} dQ_i (Im dS_i/dp)].
Parameters: series conductance g and susceptance b (y_s = g + j b) and total
charging b_ch.  For the specified injections dL/dP_i = -(2/m) dP_i (i in pvpq)
and dL/dQ_i = -(2/m) dQ_i (i in pq).
"""
from __future__ import annotations

import numpy as np

from .jacobian import jacobian_f
from .power import learnable_sets, mismatch, voltage


def loss_grad(Y, va, vm, p_spec, q_spec, bus_type):
    """(L, dL/dtheta [N], dL/d|V| [N]); zero at non-learnable entries."""
    f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
    m = f.size
    J = jacobian_f(Y, va, vm, bus_type)
    gx = (2.0 / m) * (J.T @ f)
    pvpq, pq = learnable_sets(bus_type)
    n = len(bus_type)
    d_va = np.zeros(n)
    d_vm = np.zeros(n)
    d_va[pvpq] = gx[: pvpq.size]
    d_vm[pq] = gx[pvpq.size:]
    return float(f @ f) / m, d_va, d_vm


def param_grad(Y, va, vm, p_spec, q_spec, bus_type, f_bus, t_bus, tap):
    """Gradients of L w.r.t. branch g, b, b_ch [M] and specified P, Q [N].

    Y must be the admittance matrix built from the same branches.  The
    derivative blocks of branch ell (from ybus.branch_blocks, tau = tap):
      dY/dg    = [[1/tau^2, -1/tau], [-1/tau, 1]]
      dY/db    = j dY/dg
      dY/db_ch = [[j/(2 tau^2), 0], [0, j/2]]
    """
    pvpq, pq = learnable_sets(bus_type)
    n = len(bus_type)
    V = voltage(va, vm)
    S = V * np.conj(Y @ V)
    dP = np.zeros(n)
    dQ = np.zeros(n)
    dP[pvpq] = (S.real - p_spec)[pvpq]
    dQ[pq] = (S.imag - q_spec)[pq]
    m = pvpq.size + pq.size
    tau = np.where(np.asarray(tap) == 0.0, 1.0, np.asarray(tap, np.float64))

    def dl(i, dS_i):
        return (2.0 / m) * (dP[i] * dS_i.real + dQ[i] * dS_i.imag)

    M = len(f_bus)
    d_g = np.zeros(M)
    d_b = np.zeros(M)
    d_bc = np.zeros(M)
    for ell in range(M):
        f, t, tl = int(f_bus[ell]), int(t_bus[ell]), tau[ell]
        Vf, Vt = V[f], V[t]
        # (dY/dg V) at f and t
        uf = Vf / tl ** 2 - Vt / tl
        ut = -Vf / tl + Vt
        d_g[ell] = dl(f, Vf * np.conj(uf)) + dl(t, Vt * np.conj(ut))
        d_b[ell] = dl(f, Vf * np.conj(1j * uf)) + dl(t, Vt * np.conj(1j * ut))
        cf = 0.5j * Vf / tl ** 2
        ct = 0.5j * Vt
        d_bc[ell] = dl(f, Vf * np.conj(cf)) + dl(t, Vt * np.conj(ct))
    d_p = -(2.0 / m) * dP
    d_q = -(2.0 / m) * dQ
    return d_g, d_b, d_bc, d_p, d_q
