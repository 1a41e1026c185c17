"""Pins of the oracle's DC approximation (oracle/dc.py) to things other than
itself: a closed form, edge-wise flow conservation, the lossless small-angle
limit of the AC power flow (Newton-Raphson oracle, pinned in its own tests),
outage plumbing and bus-order invariance."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.power import PQ, PV, SLACK
from oracle.ybus import grid_ybus


def test_two_bus_closed_form():
    # slack at angle a0 feeding injection P2 through reactance x behind tap tau:
    # P2 = (theta2 - a0) / (x tau)  =>  theta2 = a0 + P2 x tau
    for tau in (1.0, 1.07, 0.0):
        th = oracle.dc_solve(2, [0], [1], [0.2], [tau], [SLACK, PQ], [0.0, -0.8], va_slack=0.1)
        t = 1.0 if tau == 0.0 else tau
        assert th[0] == 0.1
        assert abs(th[1] - (0.1 - 0.8 * 0.2 * t)) < 1e-15


def test_flow_conservation_and_island_balance():
    g = gridgen.make_grid(60, 3, load_scale=0.2)
    th = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec, va_slack=0.05)
    F = oracle.dc_branch_flows(g.f_bus, g.t_bus, g.x, g.tap, th)
    net = np.zeros(g.n_bus)
    np.add.at(net, g.f_bus, F)
    np.add.at(net, g.t_bus, -F)
    u = g.bus_type != SLACK
    assert np.abs(net[u] - g.p_spec[u]).max() < 1e-10
    # lossless: the slack takes the island's net injection
    assert abs(net[~u].sum() + g.p_spec[u].sum()) < 1e-10


def test_lossless_small_angle_limit_of_ac():
    g = gridgen.make_grid(40, 11, load_scale=1.0)
    rng = np.random.default_rng(2)
    g.r = np.zeros_like(g.r)
    g.b_ch = np.zeros_like(g.b_ch)
    g.tap = rng.uniform(0.9, 1.1, g.n_branch)
    # |V| = 1 everywhere (every non-slack bus a pv bus at set-point 1): the AC
    # active flow is then exactly sin(theta_f - theta_t) / (x tau)
    g.bus_type = np.where(g.bus_type == SLACK, SLACK, PV).astype(g.bus_type.dtype)
    g.vm_set = np.ones(g.n_bus)
    g.p_spec = 0.01 * g.p_spec
    g.q_spec = np.zeros(g.n_bus)
    nr = oracle.nr_solve(grid_ybus(g), g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    assert nr["converged"]
    th = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec)
    scale = np.abs(nr["va"]).max()
    assert scale > 1e-3
    assert np.abs(nr["va"] - th).max() <= 1e-3 * scale  # O(theta^3) apart
    # the tap enters as 1/(x tau): dropping it (or squaring it) is far off
    th_wrong = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, np.ones(g.n_branch), g.bus_type, g.p_spec)
    assert np.abs(nr["va"] - th_wrong).max() > 1e-2 * scale


def test_outage_equals_removed_branch():
    g = gridgen.make_grid(50, 4, load_scale=0.2)
    ell = int(gridgen.n1_outages(g)[3])
    th = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec, outage=ell)
    keep = np.arange(g.n_branch) != ell
    th2 = oracle.dc_solve(g.n_bus, g.f_bus[keep], g.t_bus[keep], g.x[keep], g.tap[keep], g.bus_type, g.p_spec)
    assert np.abs(th - th2).max() < 1e-12


def test_bus_order_invariance():
    g = gridgen.make_grid(50, 6, load_scale=0.2)
    perm = np.random.default_rng(1).permutation(g.n_bus)
    inv = np.argsort(perm)
    th = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec)
    thp = oracle.dc_solve(g.n_bus, inv[g.f_bus], inv[g.t_bus], g.x, g.tap, g.bus_type[perm], g.p_spec[perm])
    assert np.abs(thp - th[perm]).max() < 1e-12


def test_outage_shift_is_superposition_of_dc_solutions():
    """DC linearity: the base-case DC angles plus the outage shift of those
    angles are the DC angles of the outage case (the shift's right-hand side
    is the injection the removed branch carried)."""
    g = gridgen.make_grid(80, 7, load_scale=0.3)
    th0 = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec, va_slack=0.2)
    for ell in gridgen.n1_outages(g)[::9]:
        d = oracle.dc_outage_shift(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, th0, int(ell))
        th1 = oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, g.p_spec, va_slack=0.2,
                              outage=int(ell))
        assert np.abs(th0 + d - th1).max() < 1e-10
        assert np.all(d[g.bus_type == SLACK] == 0.0)


def test_outage_shift_keeps_the_injections_of_arbitrary_angles():
    """For any angles (here random, as AC angles would be), the shifted angles
    over the remaining branches give every non-slack bus the net injection
    the original angles gave it over all branches; no outage: no shift."""
    g = gridgen.make_grid(60, 2, load_scale=0.2)
    th = np.random.default_rng(5).normal(0.0, 0.3, g.n_bus)
    ell = int(gridgen.n1_outages(g)[11])
    d = oracle.dc_outage_shift(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, th, ell)

    def net(f, t, x, tap, theta):
        F = oracle.dc_branch_flows(f, t, x, tap, theta)
        n = np.zeros(g.n_bus)
        np.add.at(n, f, F)
        np.add.at(n, t, -F)
        return n

    keep = np.arange(g.n_branch) != ell
    before = net(g.f_bus, g.t_bus, g.x, g.tap, th)
    after = net(g.f_bus[keep], g.t_bus[keep], g.x[keep], g.tap[keep], th + d)
    u = g.bus_type != SLACK
    assert np.abs(after[u] - before[u]).max() < 1e-10 * max(1.0, np.abs(before).max())
    assert np.abs(d).max() > 1e-3  # the removed flow did move the angles
    assert np.all(oracle.dc_outage_shift(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, th, -1) == 0.0)
