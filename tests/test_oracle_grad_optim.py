"""Pins for the oracle's gradients and optimiser (CPU).

* central finite differences (step 1e-6, FP64) of the loss at every
  coordinate of 3-5 bus grids (voltage learnables, branch g/b/b_ch, P, Q, and
  r/x through the chain rule);
* Adam, ReduceLROnPlateau and StepLR against torch.optim on the same gradient
  / loss sequences (library special case);
* the default hyper-parameters against the values printed in Tables 2-3.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.ybus import grid_ybus
from conftest import small_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hyperparameters.json")


def _rand_state(g, seed):
    rng = np.random.default_rng(seed)
    va = 0.2 * rng.standard_normal(g.n_bus)
    vm = 1.0 + 0.05 * rng.standard_normal(g.n_bus)
    return va, vm


@pytest.mark.parametrize("n,seed,npv,neg", [(3, 1, 1, False), (4, 2, 1, False), (5, 3, 2, False),
                                            (5, 9, 1, False), (5, 9, 1, True)])
def test_voltage_gradient_fd(n, seed, npv, neg):
    g = small_grid(n, seed, n_pv=npv)
    Y = grid_ybus(g)
    va, vm = _rand_state(g, seed)
    if neg:  # an iterate whose magnitude variable went negative
        vm[g.pq[0]] = -0.3
    L, d_va, d_vm = oracle.loss_grad(Y, va, vm, g.p_spec, g.q_spec, g.bus_type)
    h = 1e-6
    pvpq, pq = oracle.learnable_sets(g.bus_type)
    lf = lambda a, m: oracle.loss(Y, a, m, g.p_spec, g.q_spec, g.bus_type)
    scale = max(np.abs(d_va).max(), np.abs(d_vm).max())
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd_a = (lf(va + e, vm) - lf(va - e, vm)) / (2 * h)
        fd_m = (lf(va, vm + e) - lf(va, vm - e)) / (2 * h)
        # non-learnable coordinates must report zero
        want_a = fd_a if i in pvpq else 0.0
        want_m = fd_m if i in pq else 0.0
        assert abs(d_va[i] - want_a) <= 1e-7 * scale
        assert abs(d_vm[i] - want_m) <= 1e-7 * scale


@pytest.mark.parametrize("n,seed", [(3, 1), (5, 3), (6, 4)])
def test_param_gradient_fd(n, seed):
    g = small_grid(n, seed, n_pv=1)
    va, vm = _rand_state(g, seed + 100)
    Y = grid_ybus(g)
    d_g, d_b, d_bc, d_p, d_q = oracle.param_grad(Y, va, vm, g.p_spec, g.q_spec, g.bus_type,
                                                 g.f_bus, g.t_bus, g.tap)
    ys = 1.0 / (g.r + 1j * g.x)

    def L_of(gs, bs, bc, p, q):
        z = 1.0 / (gs + 1j * bs)
        Yp = oracle.build_ybus(g.n_bus, g.f_bus, g.t_bus, z.real, z.imag, bc, g.tap)
        return oracle.loss(Yp, va, vm, p, q, g.bus_type)

    base = [ys.real.copy(), ys.imag.copy(), g.b_ch.copy(), g.p_spec.copy(), g.q_spec.copy()]
    grads = [d_g, d_b, d_bc, d_p, d_q]
    h = 1e-6
    for which in range(5):
        scale = max(np.abs(grads[which]).max(), 1e-12)
        for j in range(base[which].size):
            up = [b.copy() for b in base]
            dn = [b.copy() for b in base]
            up[which][j] += h
            dn[which][j] -= h
            fd = (L_of(*up) - L_of(*dn)) / (2 * h)
            assert abs(grads[which][j] - fd) <= 2e-7 * scale + 1e-12, (which, j)


def test_param_gradient_chain_rule_r_x():
    """dL/dr, dL/dx from (dL/dg, dL/db) and g + jb = 1/(r + jx), against FD on r, x."""
    g = small_grid(5, 7, n_pv=1)
    va, vm = _rand_state(g, 7)
    Y = grid_ybus(g)
    d_g, d_b, *_ = oracle.param_grad(Y, va, vm, g.p_spec, g.q_spec, g.bus_type, g.f_bus, g.t_bus, g.tap)
    r, x = g.r, g.x
    den = r * r + x * x
    dg_dr, dg_dx = (x * x - r * r) / den ** 2, -2 * r * x / den ** 2
    db_dr, db_dx = 2 * r * x / den ** 2, (x * x - r * r) / den ** 2
    d_r = d_g * dg_dr + d_b * db_dr
    d_x = d_g * dg_dx + d_b * db_dx
    h = 1e-7
    for j in range(g.n_branch):
        for arr, dd in ((r, d_r), (x, d_x)):
            up, dn = arr.copy(), arr.copy()
            up[j] += h
            dn[j] -= h
            rr = (up, x) if arr is r else (r, up)
            rd = (dn, x) if arr is r else (r, dn)
            Lu = oracle.loss(oracle.build_ybus(g.n_bus, g.f_bus, g.t_bus, rr[0], rr[1], g.b_ch, g.tap), va, vm, g.p_spec, g.q_spec, g.bus_type)
            Ld = oracle.loss(oracle.build_ybus(g.n_bus, g.f_bus, g.t_bus, rd[0], rd[1], g.b_ch, g.tap), va, vm, g.p_spec, g.q_spec, g.bus_type)
            fd = (Lu - Ld) / (2 * h)
            assert abs(dd[j] - fd) <= 1e-6 * max(abs(fd), 1.0)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    n = 17
    x0 = rng.standard_normal(n)
    grads = rng.standard_normal((300, n)) * np.logspace(0, -6, 300)[:, None]
    for betas in [(0.979, 0.963), (0.9, 0.999), (0.7847, 0.6624)]:
        opt = oracle.Adam(n, 3e-3, betas)
        x = x0.copy()
        p = torch.tensor(x0.copy(), dtype=torch.float64, requires_grad=True)
        topt = torch.optim.Adam([p], lr=3e-3, betas=betas, eps=1e-8, foreach=False)
        for gk in grads:
            x = opt.step(x, gk)
            p.grad = torch.tensor(gk, dtype=torch.float64)
            topt.step()
        np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_sgd_rmsprop_match_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    n = 11
    x0 = rng.standard_normal(n)
    grads = rng.standard_normal((200, n)) * np.logspace(0, -4, 200)[:, None]
    for make, tmake in [
        (lambda: oracle.SGD(n, 1e-2, 0.9), lambda p: torch.optim.SGD([p], lr=1e-2, momentum=0.9)),
        (lambda: oracle.SGD(n, 1e-2, 0.0), lambda p: torch.optim.SGD([p], lr=1e-2)),
        (lambda: oracle.RMSprop(n, 1e-3, 0.99), lambda p: torch.optim.RMSprop([p], lr=1e-3, alpha=0.99, eps=1e-8)),
    ]:
        opt = make()
        x = x0.copy()
        p = torch.tensor(x0.copy(), dtype=torch.float64, requires_grad=True)
        topt = tmake(p)
        for gk in grads:
            x = opt.step(x, gk)
            p.grad = torch.tensor(gk, dtype=torch.float64)
            topt.step()
        np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_schedulers_match_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    losses = np.concatenate([np.linspace(1, 0.5, 50), 0.5 + 0.01 * rng.random(400),
                             np.linspace(0.5, 0.1, 100), 0.1 + 0.001 * rng.random(300)])
    for kw in [dict(factor=0.547, patience=41, threshold=0.0673, cooldown=97),
               dict(factor=0.8, patience=2, threshold=0.0388, cooldown=4),
               dict(factor=0.5, patience=10, threshold=1e-4, cooldown=0)]:
        opt = oracle.Adam(1, 0.01)
        sch = oracle.ReduceLROnPlateau(opt, **kw)
        p = torch.zeros(1, requires_grad=True)
        topt = torch.optim.SGD([p], lr=0.01)
        tsch = torch.optim.lr_scheduler.ReduceLROnPlateau(topt, mode="min", threshold_mode="rel", **kw)
        for L in losses:
            sch.step(L)
            tsch.step(L)
            assert opt.lr == pytest.approx(topt.param_groups[0]["lr"], rel=1e-15)
    opt = oracle.Adam(1, 0.03564)
    sch = oracle.StepLR(opt, 100, 0.773)
    p = torch.zeros(1, requires_grad=True)
    topt = torch.optim.SGD([p], lr=0.03564)
    tsch = torch.optim.lr_scheduler.StepLR(topt, 100, 0.773)
    for _ in range(1000):
        topt.step()
        sch.step()
        tsch.step()
        assert opt.lr == pytest.approx(topt.param_groups[0]["lr"], rel=1e-12)


def test_defaults_are_table2():
    t2 = json.load(open(GOLDEN))["table2_static"]
    o = oracle.DPFOptions()
    assert (o.beta1, o.beta2) == tuple(t2["betas"])
    assert (o.factor, o.patience, o.threshold, o.cooldown) == (
        t2["factor"], t2["patience"], t2["threshold"], t2["cooldown"])
    assert o.max_iter == t2["max_iter"]
