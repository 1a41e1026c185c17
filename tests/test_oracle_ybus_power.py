"""Pins for the oracle's Y_bus and S_calc (CPU).

* branch currents from circuit analysis of the pi-model with an ideal
  transformer (not from the oracle's block formula);
* the power-balance identity: for ANY voltage vector, the power injected at
  all buses equals the power absorbed by the branches
  (series z|I_s|^2 plus the charging halves at the line-side voltages);
* structural facts: symmetry, nnz = N + 2M, zero row sums without shunts.
"""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.ybus import grid_ybus
from conftest import small_grid


def _branch_absorbed(grid, V):
    """Complex power absorbed by each branch, from circuit analysis."""
    tau = np.where(grid.tap == 0, 1.0, grid.tap)
    vf_line = V[grid.f_bus] / tau  # ideal transformer at the from-bus
    vt = V[grid.t_bus]
    z = grid.r + 1j * grid.x
    i_series = (vf_line - vt) / z
    series = z * np.abs(i_series) ** 2
    charging = -1j * grid.b_ch / 2 * (np.abs(vf_line) ** 2 + np.abs(vt) ** 2)
    return series + charging


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (5, 2), (30, 0), (300, 5)])
def test_power_balance_identity_any_voltage(n, seed):
    g = small_grid(n, seed) if n < 30 else gridgen.make_grid(n, seed)
    Y = grid_ybus(g)
    rng = np.random.default_rng(seed)
    V = (1 + 0.1 * rng.standard_normal(n)) * np.exp(1j * 0.3 * rng.standard_normal(n))
    S = oracle.s_calc(Y, V)
    lhs = S.sum()
    rhs = _branch_absorbed(g, V).sum()
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, np.abs(S).sum())


def test_branch_currents_from_circuit():
    # one transformer branch with charging between bus 0 (from) and bus 1 (to)
    r, x, b, tau = 0.012, 0.09, 0.03, 1.04
    Y = oracle.build_ybus(2, [0], [1], [r], [x], [b], [tau])
    Vf, Vt = 1.02 * np.exp(0.1j), 0.97 * np.exp(-0.05j)
    z = r + 1j * x
    i_s = (Vf / tau - Vt) / z
    i_from = (i_s + 0.5j * b * Vf / tau) / tau  # primary current of the ideal transformer
    i_to = -i_s + 0.5j * b * Vt
    I = Y @ np.array([Vf, Vt])
    assert abs(I[0] - i_from) < 1e-12
    assert abs(I[1] - i_to) < 1e-12


@pytest.mark.parametrize("n,seed", [(30, 0), (2000, 2)])
def test_ybus_structure(n, seed):
    g = gridgen.make_grid(n, seed)
    Y = grid_ybus(g)
    assert Y.nnz == g.n_bus + 2 * g.n_branch
    assert abs(Y - Y.T).max() < 1e-15
    # remove charging and taps: every row of a pure series network sums to 0
    Y0 = oracle.build_ybus(g.n_bus, g.f_bus, g.t_bus, g.r, g.x, 0 * g.b_ch, np.ones(g.n_branch))
    assert np.abs(np.asarray(Y0.sum(axis=1))).max() < 1e-9
    # charging only (tau = 1): row sum = j * half the charging of incident branches
    Yc = oracle.build_ybus(g.n_bus, g.f_bus, g.t_bus, g.r, g.x, g.b_ch, np.ones(g.n_branch))
    want = np.zeros(g.n_bus)
    np.add.at(want, g.f_bus, g.b_ch / 2)
    np.add.at(want, g.t_bus, g.b_ch / 2)
    assert np.abs(np.asarray(Yc.sum(axis=1)).ravel() - 1j * want).max() < 1e-9


def test_mismatch_sets_and_loss_normalisation():
    g = small_grid(5, 3, n_pv=2)
    Y = grid_ybus(g)
    va = np.linspace(-0.1, 0.1, 5)
    vm = np.linspace(0.95, 1.05, 5)
    f, S = oracle.mismatch(Y, va, vm, g.p_spec, g.q_spec, g.bus_type)
    pv, pq = g.pv, g.pq
    assert f.size == pv.size + 2 * pq.size
    want = np.concatenate([(S.real - g.p_spec)[pv], (S.real - g.p_spec)[pq],
                           (S.imag - g.q_spec)[pq]])
    np.testing.assert_allclose(f, want, rtol=0, atol=0)
    assert oracle.loss(Y, va, vm, g.p_spec, g.q_spec, g.bus_type) == pytest.approx(np.mean(want ** 2), rel=1e-15)


def test_rejects_phase_shift():
    with pytest.raises(ValueError):
        oracle.build_ybus(2, [0], [1], [0.01], [0.1], [0.0], [1.0], shift=[0.1])
