"""Jacobian of the power mismatch (oracle; test infrastructure).

Alg. 2 (Newton-Raphson) writes the partial derivatives of S_calc element-wise:

  dS_i/d|V|_j = V_i Y_ij^* V_j^* / |V_j|                      (i != j)
              = V_i/|V_i| I_i^* + V_i Y_ii^* V_i^* / |V_i|     (i == j)
  dS_i/dtheta_j = -j V_i Y_ij^* V_j^*                          (i != j)
                = j V_i I_i^* - j V_i Y_ii^* V_i^*             (i == j)

and selects J_f = [[dP/dtheta[pvpq,pvpq], dP/d|V|[pvpq,pq]],
                   [dQ/dtheta[pq,pvpq],   dQ/d|V|[pq,pq]]].
Here the element-wise rules are written as sparse matrix products: the
off-diagonal rule applied to every (i, j) of Y's pattern is
diag(V) conj(Y) diag(conj(V)/|V|) (resp. -j diag(V) conj(Y) diag(conj(V))), and
the diagonal rule adds diag(V/|V| conj(I)) (resp. j diag(V conj(I))).

|V| in these denominators is the magnitude variable itself (Alg. 1: the
learnable real factor in V = |V| e^{j theta}), not the modulus of V: the two
agree while the variable is positive, and using the variable keeps the
partials those of S with respect to the learnable when an iterate's
magnitude turns negative.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .power import learnable_sets, voltage


def dS_dVm_dVa(Y, va, vm):
    """(dS/d|V|, dS/dtheta) as complex sparse matrices (Alg. 2)."""
    vm = np.asarray(vm, np.float64)
    V = voltage(va, vm)
    I = Y @ V
    Yc = Y.conj()
    dV = sp.diags(V)
    d_vm = dV @ Yc @ sp.diags(np.conj(V) / vm) + sp.diags(V / vm * np.conj(I))
    d_va = -1j * (dV @ Yc @ sp.diags(np.conj(V))) + sp.diags(1j * V * np.conj(I))
    return d_vm.tocsr(), d_va.tocsr()


def jacobian_f(Y, va, vm, bus_type):
    """J_f (real sparse CSC), rows [P(pvpq); Q(pq)], cols [theta(pvpq); |V|(pq)]."""
    pvpq, pq = learnable_sets(bus_type)
    d_vm, d_va = dS_dVm_dVa(Y, va, vm)
    j11 = d_va[pvpq][:, pvpq].real
    j12 = d_vm[pvpq][:, pq].real
    j21 = d_va[pq][:, pvpq].imag
    j22 = d_vm[pq][:, pq].imag
    return sp.bmat([[j11, j12], [j21, j22]]).tocsc()
