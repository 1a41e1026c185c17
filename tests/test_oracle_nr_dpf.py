"""Pins for the oracle's Newton-Raphson solver and DPF loop (CPU).

* two-bus closed form: slack E at angle 0 feeding a load P + jQ through
  z = r + jx.  From V1 conj(V2) = |V2|^2 + z conj(S_L):
      |V2|^2 = ((E^2 - 2a) + sqrt((E^2 - 2a)^2 - 4 |z|^2 |S_L|^2)) / 2,
      theta2 = -atan2(b, |V2|^2 + a),  a = rP + xQ, b = xP - rQ;
* NR against scipy.optimize.fsolve on the same equations (library routine);
* NR's local quadratic convergence;
* at the solution the loss and its gradient vanish and the slack/PV
  unknowns (P at the slack, Q at PV buses) balance the branch losses;
* DPF (Alg. 1) reaches the NR solution on the two-bus line and on the
  30-bus workload.
"""
import math

import numpy as np
import pytest
import scipy.optimize

import gridgen
import oracle
from oracle.ybus import grid_ybus
from conftest import small_grid


def two_bus_closed_form(P, Q, r, x, E=1.0):
    a, b = r * P + x * Q, x * P - r * Q
    c = E * E - 2 * a
    u2 = 0.5 * (c + math.sqrt(c * c - 4 * (r * r + x * x) * (P * P + Q * Q)))
    return math.sqrt(u2), -math.atan2(b, u2 + a)


@pytest.mark.parametrize("P,Q,r,x", [(0.5, 0.2, 0.01, 0.1), (1.2, 0.4, 0.02, 0.25), (0.8, -0.3, 0.05, 0.08)])
def test_nr_two_bus_closed_form(P, Q, r, x):
    g = gridgen.two_bus(P, Q, r, x)
    Y = grid_ybus(g)
    res = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    assert res["converged"]
    u, th = two_bus_closed_form(P, Q, r, x)
    assert abs(res["vm"][1] - u) < 1e-11
    assert abs(res["va"][1] - th) < 1e-11


@pytest.mark.parametrize("n,seed,npv", [(3, 1, 1), (4, 2, 1), (5, 3, 2)])
def test_nr_matches_fsolve(n, seed, npv):
    g = small_grid(n, seed, n_pv=npv, load_scale=0.5)
    Y = grid_ybus(g)
    res = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    assert res["converged"]
    pvpq, pq = oracle.learnable_sets(g.bus_type)
    va0, vm0 = oracle.flat_start(g.bus_type, g.vm_set)

    def F(x):
        va, vm = va0.copy(), vm0.copy()
        va[pvpq] = x[: pvpq.size]
        vm[pq] = x[pvpq.size:]
        return oracle.mismatch(Y, va, vm, g.p_spec, g.q_spec, g.bus_type)[0]

    x0 = np.concatenate([va0[pvpq], vm0[pq]])
    xs, info, ier, msg = scipy.optimize.fsolve(F, x0, xtol=1e-13, full_output=True)
    assert ier == 1, msg
    np.testing.assert_allclose(xs[: pvpq.size], res["va"][pvpq], atol=1e-9)
    np.testing.assert_allclose(xs[pvpq.size:], res["vm"][pq], atol=1e-9)


def test_nr_quadratic_convergence_and_solution_properties():
    g = gridgen.config_grid("c1_30bus_fp64")
    Y = grid_ybus(g)
    res = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set, tol=1e-13)
    assert res["converged"]
    e = res["norms"]
    # once in the quadratic regime, e_{k+1} <= C e_k^2 with a moderate C
    ratios = [e[k + 1] / e[k] ** 2 for k in range(len(e) - 1) if 1e-12 < e[k + 1] and e[k] < 1e-2]
    assert ratios and max(ratios) < 1e3
    L, d_va, d_vm = oracle.loss_grad(Y, res["va"], res["vm"], g.p_spec, g.q_spec, g.bus_type)
    assert L < 1e-26
    assert max(np.abs(d_va).max(), np.abs(d_vm).max()) < 1e-10
    # slack P and PV Q are outputs: total injection equals total branch loss (> 0)
    S = oracle.s_calc(Y, res["vm"] * np.exp(1j * res["va"]))
    assert S.real.sum() > 0
    assert abs(S.real.sum() - (S.real[g.slack] + g.p_spec[g.bus_type != gridgen.SLACK].sum())) < 1e-9


def test_dpf_two_bus_reaches_closed_form():
    P, Q, r, x = 0.5, 0.2, 0.01, 0.1
    g = gridgen.two_bus(P, Q, r, x)
    Y = grid_ybus(g)
    opts = oracle.DPFOptions(lr=1e-2, max_iter=20000, tol=1e-9)
    res = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set, opts)
    assert res["status"] == 0
    u, th = two_bus_closed_form(P, Q, r, x)
    assert abs(res["vm"][1] - u) < 1e-8
    assert abs(res["va"][1] - th) < 1e-8


def test_dpf_30bus_reaches_nr():
    """The 30-bus FP64 workload: Adam (lr 1e-2, Table 2 betas and plateau) to 1e-6 p.u."""
    g = gridgen.config_grid("c1_30bus_fp64")
    Y = grid_ybus(g)
    nr = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    res = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set,
                           oracle.DPFOptions(lr=1e-2, max_iter=20000, tol=1e-6))
    assert res["status"] == 0 and res["max_mismatch"] <= 1e-6
    assert np.abs(res["vm"] - nr["vm"]).max() < 1e-5
    assert np.abs(res["va"] - nr["va"]).max() < 1e-5
