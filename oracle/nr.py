"""Newton-Raphson power flow (Alg. 2), the ground-truth solver (oracle).

Alg. 2: evaluate f = [(P_calc - P)[pvpq], (Q_calc - Q)[pq]]; while its norm is
above tol, build dS/d|V| and dS/dtheta, select J_f, solve J_f dx = -f and
update [theta[pvpq]; |V|[pq]] <- [...] + dx.  The tolerance test uses the
infinity norm.  The linear solve is scipy.sparse.linalg.spsolve (a library
primitive standing in for LightSim2Grid's KLU).  Start: flat (the DC start of
Alg. 2 is an optional refinement not used here).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .dpf import flat_start
from .jacobian import jacobian_f
from .power import learnable_sets, mismatch


def nr_solve(Y, p_spec, q_spec, bus_type, vm_set, va_slack=0.0, tol=1e-10,
             max_iter=50, va0=None, vm0=None):
    """Returns dict(va, vm, iters, converged, norms) with norms[k] = ||f_k||_inf."""
    fva, fvm = flat_start(bus_type, vm_set, va_slack)
    va = fva if va0 is None else np.asarray(va0, np.float64).copy()
    vm = fvm if vm0 is None else np.asarray(vm0, np.float64).copy()
    pvpq, pq = learnable_sets(bus_type)
    npv = pvpq.size
    norms = []
    f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
    it = 0
    while True:
        nrm = float(np.max(np.abs(f))) if f.size else 0.0
        norms.append(nrm)
        if nrm < tol:
            return dict(va=va, vm=vm, iters=it, converged=True, norms=norms)
        if it >= max_iter or not np.isfinite(nrm):
            return dict(va=va, vm=vm, iters=it, converged=False, norms=norms)
        J = jacobian_f(Y, va, vm, bus_type)
        dx = spla.spsolve(J, -f)
        va = va.copy()
        vm = vm.copy()
        va[pvpq] += dx[:npv]
        vm[pq] += dx[npv:]
        it += 1
        f, _ = mismatch(Y, va, vm, p_spec, q_spec, bus_type)
