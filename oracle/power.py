"""Power balance, mismatch and loss (oracle; test infrastructure).

Eq. powerbalance: S_calc = V (Y_bus V)^*.
Eq. pf_equation_full: P must match at pv and pq buses, Q at pq buses; |V| is
fixed at pv buses and V at the slack.
Alg. 1: the loss is the MSE between out = [P_calc[pv,pq], Q_calc[pq]] and
target = [P[pv,pq], Q[pq]], i.e. L = (1/m) sum f^2 with m = |pv| + 2|pq|.
The mismatch is taken as calculated minus specified (Alg. 2's f); the sign
does not change the loss.
"""
from __future__ import annotations

import numpy as np

PQ, PV, SLACK = 0, 1, 2


def learnable_sets(bus_type):
    """(pvpq, pq): the buses whose angle, and whose magnitude, are unknown.

    pvpq lists the pv buses then the pq buses, each in ascending order
    (Alg. 1 and Alg. 2 index lists).
    """
    bus_type = np.asarray(bus_type)
    pv = np.flatnonzero(bus_type == PV)
    pq = np.flatnonzero(bus_type == PQ)
    return np.concatenate([pv, pq]), pq


def voltage(va, vm):
    """V = |V| e^{j theta} (Sec. 4, polar parameterisation)."""
    return np.asarray(vm, np.float64) * np.exp(1j * np.asarray(va, np.float64))


def s_calc(Y, V):
    """S_calc = V (Y V)^* (Eq. powerbalance)."""
    return V * np.conj(Y @ V)


def mismatch(Y, va, vm, p_spec, q_spec, bus_type):
    """f = [(P_calc - P)[pvpq], (Q_calc - Q)[pq]] (Alg. 2) and S_calc."""
    pvpq, pq = learnable_sets(bus_type)
    S = s_calc(Y, voltage(va, vm))
    f = np.concatenate([(S.real - p_spec)[pvpq], (S.imag - q_spec)[pq]])
    return f, S


def loss(Y, va, vm, p_spec, q_spec, bus_type):
    """L = MSE(out, target) = (1/m) ||f||^2 (Alg. 1)."""
    f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
    return float(f @ f) / f.size
