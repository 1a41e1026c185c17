"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
  * FP64 kernels: results agree with the oracle to rounding, 1e-10 relative
    to the largest magnitude involved (sums of O(10) terms of size |Y| ~ 300
    in a different order);
  * FP32 kernels: S_calc within 1e-4 p.u. absolute (terms |Y_ij V_j| <= ~300,
    FP32 epsilon 6e-8, a few terms per row), gradients within 1e-4 of the
    gradient's max-abs (the required 1e-4 relative, norm-wise);
  * the FP64 convergence test (loss, max mismatch) runs in FP64 in both
    modes: 1e-12 relative.
"""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.ybus import grid_ybus

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_28203_gb300 as dpf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2603_28203_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    dpf.lib()


def _states(n_case, n_bus, seed, spread=0.2):
    rng = np.random.default_rng(seed)
    va = spread * rng.standard_normal((n_case, n_bus))
    vm = 1.0 + 0.05 * rng.standard_normal((n_case, n_bus))
    return va, vm


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


GRIDS = {
    "c1": lambda: gridgen.config_grid("c1_30bus_fp64"),
    "g300": lambda: gridgen.make_grid(300, 5, load_scale=0.1),
    "c3": lambda: gridgen.config_grid("c3_n1_2kbus"),
}


@pytest.mark.parametrize("gname", ["c1", "g300", "c3"])
@pytest.mark.parametrize("precision", [dpf.FP64, dpf.FP32])
@pytest.mark.parametrize("K", [1, 5, 37])
def test_power_parity(gname, precision, K):
    g = GRIDS[gname]()
    Y = grid_ybus(g)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    va, vm = _states(K, g.n_bus, 1)
    p, q = dpf.dpf_power(y, ws, _t(va), _t(vm), precision=precision)
    p, q = p.cpu().numpy(), q.cpu().numpy()
    for k in range(K):
        S = oracle.s_calc(Y, vm[k] * np.exp(1j * va[k]))
        scale = np.abs(S).max()
        tol = 1e-10 * scale if precision == dpf.FP64 else 1e-4
        assert np.abs(p[k] - S.real).max() <= tol
        assert np.abs(q[k] - S.imag).max() <= tol


@pytest.mark.parametrize("gname", ["c1", "g300"])
@pytest.mark.parametrize("precision", [dpf.FP64, dpf.FP32])
def test_loss_backward_parity(gname, precision):
    g = GRIDS[gname]()
    Y = grid_ybus(g)
    K = 6
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    va, vm = _states(K, g.n_bus, 2, spread=0.05)
    rng = np.random.default_rng(3)
    P = g.p_spec[None, :] * (1 + 0.1 * rng.standard_normal((K, g.n_bus)))
    Q = g.q_spec[None, :] * (1 + 0.1 * rng.standard_normal((K, g.n_bus)))
    out = dpf.dpf_loss_backward(y, ws, _t(va), _t(vm), _t(P), _t(Q), precision=precision,
                                want=("loss", "d_va", "d_vm", "d_p", "d_q", "d_g", "d_b", "d_bch"))
    o = {k: v.cpu().numpy() for k, v in out.items()}
    sum_g = np.zeros(g.n_branch)
    sum_b = np.zeros(g.n_branch)
    sum_bc = np.zeros(g.n_branch)
    rel = 1e-10 if precision == dpf.FP64 else 1e-4
    for k in range(K):
        L, d_va, d_vm = oracle.loss_grad(Y, va[k], vm[k], P[k], Q[k], g.bus_type)
        assert abs(o["loss"][k] - L) <= 1e-12 * L
        sc = max(np.abs(d_va).max(), np.abs(d_vm).max())
        assert np.abs(o["d_va"][k] - d_va).max() <= rel * sc
        assert np.abs(o["d_vm"][k] - d_vm).max() <= rel * sc
        dg, db, dbc, dp, dq = oracle.param_grad(Y, va[k], vm[k], P[k], Q[k], g.bus_type, g.f_bus, g.t_bus, g.tap)
        sc = max(np.abs(dp).max(), np.abs(dq).max())
        assert np.abs(o["d_p"][k] - dp).max() <= rel * sc
        assert np.abs(o["d_q"][k] - dq).max() <= rel * sc
        sum_g += dg
        sum_b += db
        sum_bc += dbc
    for got, want in ((o["d_g"], sum_g), (o["d_b"], sum_b), (o["d_bch"], sum_bc)):
        assert np.abs(got - want).max() <= rel * np.abs(want).max()


def test_modified_branch_parameters():
    """g_series / b_series replace the series admittance (parameter identification)."""
    g = GRIDS["g300"]()
    K = 4
    rng = np.random.default_rng(9)
    gp = gridgen.perturb_branches(g, 5)
    ys = 1.0 / (gp.r + 1j * gp.x)
    Yp = grid_ybus(gp)
    y = dpf.dpf_build_ybus(g)  # the as-built grid; parameters come in per call
    ws = dpf.dpf_workspace_create(y, K)
    va, vm = _states(K, g.n_bus, 4, spread=0.05)
    out = dpf.dpf_loss_backward(y, ws, _t(va), _t(vm), g_series=_t(ys.real), b_series=_t(ys.imag),
                                precision=dpf.FP64, want=("loss", "d_g", "d_b"))
    sg = np.zeros(g.n_branch)
    for k in range(K):
        L = oracle.loss(Yp, va[k], vm[k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(out["loss"][k].item() - L) <= 1e-12 * L
        sg += oracle.param_grad(Yp, va[k], vm[k], g.p_spec, g.q_spec, g.bus_type, g.f_bus, g.t_bus, g.tap)[0]
    assert np.abs(out["d_g"].cpu().numpy() - sg).max() <= 1e-10 * np.abs(sg).max()


@pytest.mark.parametrize("precision", [dpf.FP64, dpf.FP32])
def test_n1_correction_parity(precision):
    """Shared Y + per-case branch-removal correction == Y rebuilt without the branch."""
    g = GRIDS["c3"]()
    outs = gridgen.n1_outages(g)
    rng = np.random.default_rng(5)
    ells = np.concatenate([[-1], rng.choice(outs, 40, replace=False)]).astype(np.int32)
    K = ells.size
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    va, vm = _states(K, g.n_bus, 6, spread=0.1)
    p, q = dpf.dpf_power(y, ws, _t(va), _t(vm), outage=_t(ells, torch.int32), precision=precision)
    out = dpf.dpf_loss_backward(y, ws, _t(va), _t(vm), outage=_t(ells, torch.int32), precision=precision,
                                want=("loss", "d_va", "d_vm"))
    p, q = p.cpu().numpy(), q.cpu().numpy()
    rel = 1e-10 if precision == dpf.FP64 else 1e-4
    for k in range(K):
        gk = g if ells[k] < 0 else g.without_branch(int(ells[k]))
        Yk = grid_ybus(gk)
        S = oracle.s_calc(Yk, vm[k] * np.exp(1j * va[k]))
        tol = 1e-10 * np.abs(S).max() if precision == dpf.FP64 else 1e-4
        assert np.abs(p[k] - S.real).max() <= tol and np.abs(q[k] - S.imag).max() <= tol
        L, d_va, d_vm = oracle.loss_grad(Yk, va[k], vm[k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(out["loss"][k].item() - L) <= 1e-12 * L
        sc = max(np.abs(d_va).max(), np.abs(d_vm).max())
        assert np.abs(out["d_va"][k].cpu().numpy() - d_va).max() <= rel * sc
        assert np.abs(out["d_vm"][k].cpu().numpy() - d_vm).max() <= rel * sc


def _solve(y, ws, K, opts, **kw):
    N = y.n_bus
    res = dict(va=torch.zeros((K, N), dtype=torch.float64, device=DEV),
               vm=torch.zeros((K, N), dtype=torch.float64, device=DEV),
               iters=torch.zeros(K, dtype=torch.int32, device=DEV),
               status=torch.zeros(K, dtype=torch.int32, device=DEV),
               max_mismatch=torch.zeros(K, dtype=torch.float64, device=DEV),
               loss=torch.zeros(K, dtype=torch.float64, device=DEV))
    for k in ("va", "vm"):
        if k + "0" in kw:
            res[k].copy_(kw.pop(k + "0"))
    dpf.dpf_solve_batch(y, ws, opts, n_case=K, **res, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


@pytest.mark.parametrize("sched", ["plateau", "step", "const"])
@pytest.mark.parametrize("lanes", [0, 1, 4])
def test_solve_trajectory_fp64(sched, lanes):
    """FP64 batched iterations follow the oracle's Alg. 1 loop step for step."""
    g = GRIDS["c1"]()
    Y = grid_ybus(g)
    K = 5
    rng = np.random.default_rng(11)
    P = g.p_spec[None, :] * (1 + 0.05 * rng.standard_normal((K, g.n_bus)))
    Q = g.q_spec[None, :] * (1 + 0.05 * rng.standard_normal((K, g.n_bus)))
    code = dict(plateau=dpf.SCHED_PLATEAU, step=dpf.SCHED_STEP, const=dpf.SCHED_CONST)[sched]
    kw = dict(lr=2e-2, sched=sched, factor=0.5, patience=3, threshold=1e-3, cooldown=2, step_size=7, gamma=0.8)
    opts = dpf.SolveOpts(precision=dpf.FP64, max_iter=150, check_every=1, lanes=lanes, lr=2e-2, sched=code,
                         factor=0.5, patience=3, threshold=1e-3, cooldown=2, step_size=7, gamma=0.8, tol=1e-6)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    r = _solve(y, ws, K, opts, p_spec=_t(P), q_spec=_t(Q))
    for k in range(K):
        ref = oracle.dpf_solve(Y, P[k], Q[k], g.bus_type, g.vm_set,
                               oracle.DPFOptions(max_iter=150, tol=1e-6, **kw))
        assert r["iters"][k] == ref["iters"] and r["status"][k] == ref["status"]
        assert np.abs(r["va"][k] - ref["va"]).max() < 1e-9
        assert np.abs(r["vm"][k] - ref["vm"]).max() < 1e-9
        assert abs(r["max_mismatch"][k] - ref["max_mismatch"]) <= 1e-9
        assert abs(r["loss"][k] - ref["loss"]) <= 1e-9 * max(ref["loss"], 1e-12)


@pytest.mark.parametrize("opt", ["sgd", "rmsprop"])
def test_other_optimisers_trajectory_fp64(opt):
    """SGD (momentum) and RMSprop, the other optimisers of Sec. 5.3, step for step vs the oracle."""
    g = GRIDS["c1"]()
    Y = grid_ybus(g)
    K = 3
    code = dict(sgd=dpf.OPT_SGD, rmsprop=dpf.OPT_RMSPROP)[opt]
    lr = 1e-3 if opt == "sgd" else 5e-3
    kw = dict(lr=lr, momentum=0.9, alpha=0.95, sched=dpf.SCHED_PLATEAU, factor=0.5, patience=3, threshold=1e-3,
              cooldown=2)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP64, max_iter=120, check_every=1, optimizer=code, **kw))
    ref = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set,
                           oracle.DPFOptions(optimizer=opt, lr=lr, momentum=0.9, alpha=0.95, sched="plateau",
                                             factor=0.5, patience=3, threshold=1e-3, cooldown=2, max_iter=120))
    for k in range(K):
        assert np.abs(r["va"][k] - ref["va"]).max() < 1e-9
        assert np.abs(r["vm"][k] - ref["vm"]).max() < 1e-9
        assert r["iters"][k] == ref["iters"]


def test_c1_converges_to_nr_fp64():
    """30-bus workload: FP64 DPF (lr 1e-2, Table 2 betas/plateau) to 1e-6 p.u., matches NR."""
    g = GRIDS["c1"]()
    Y = grid_ybus(g)
    nr = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 1)
    r = _solve(y, ws, 1, dpf.SolveOpts(precision=dpf.FP64, max_iter=20000, check_every=1, lr=1e-2))
    assert r["status"][0] == dpf.CASE_CONVERGED and r["max_mismatch"][0] <= 1e-6
    assert np.abs(r["vm"][0] - nr["vm"]).max() < 1e-5
    assert np.abs(r["va"][0] - nr["va"]).max() < 1e-5
    ref = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set, oracle.DPFOptions(lr=1e-2, max_iter=20000))
    # same algorithm in FP64; rounding may flip a late plateau decision
    assert abs(int(r["iters"][0]) - ref["iters"]) <= 0.1 * ref["iters"]


def test_plain_form_matches_batched():
    g = GRIDS["c1"]()
    K = 3
    rng = np.random.default_rng(12)
    P = g.p_spec[None, :] * (1 + 0.05 * rng.standard_normal((K, g.n_bus)))
    Q = g.q_spec[None, :] * (1 + 0.05 * rng.standard_normal((K, g.n_bus)))
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(precision=dpf.FP64, max_iter=300, check_every=1, lr=1e-2)
    a = _solve(y, ws, K, dpf.SolveOpts(**base), p_spec=_t(P), q_spec=_t(Q))
    b = _solve(y, ws, K, dpf.SolveOpts(plain=1, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (a["iters"] == b["iters"]).all()
    assert np.abs(a["va"] - b["va"]).max() == 0.0 and np.abs(a["vm"] - b["vm"]).max() == 0.0


def test_fp32_iterations_track_fp64():
    """FP32 iterations (double-float master) stay close to the oracle's FP64
    trajectory (Alg. 1, same settings): 1e-3 on the iterates after 200 steps
    at a constant rate."""
    g = GRIDS["g300"]()
    K = 8
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(max_iter=200, check_every=10, lr=1e-3, sched=dpf.SCHED_CONST)
    b = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP32, **base))
    Y = grid_ybus(g)
    ref = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set,
                           oracle.DPFOptions(lr=1e-3, max_iter=200, check_every=10, sched="const"))
    assert np.abs(b["va"] - ref["va"][None]).max() < 1e-3
    assert np.abs(b["vm"] - ref["vm"][None]).max() < 1e-3
    # the reported FP64 mismatch is the oracle's mismatch of the returned state
    for k in range(K):
        f, _ = oracle.mismatch(Y, b["va"][k], b["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(b["max_mismatch"][k] - np.abs(f).max()) <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("outages", [False, True])
def test_pair_kernels_match_single(outages):
    """FP32 batches >= 64 cases run two cases per thread; same iterates as one per thread."""
    g = GRIDS["c3"]()
    K = 100
    kw = {}
    if outages:
        ells = np.concatenate([[-1], np.random.default_rng(8).choice(gridgen.n1_outages(g), K - 1, replace=False)])
        kw["outage"] = _t(ells.astype(np.int32), torch.int32)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(precision=dpf.FP32, max_iter=100, check_every=10, lr=1e-3)
    a = _solve(y, ws, K, dpf.SolveOpts(pair_cases=1, **base), **kw)
    b = _solve(y, ws, K, dpf.SolveOpts(pair_cases=0, **base), **kw)
    assert np.abs(a["va"] - b["va"]).max() < 1e-4 and np.abs(a["vm"] - b["vm"]).max() < 1e-4
    assert np.abs(a["max_mismatch"] - b["max_mismatch"]).max() < 1e-4 * np.abs(b["max_mismatch"]).max()
    assert (a["iters"] == b["iters"]).all()


def test_autotune_shape_is_valid_and_equivalent():
    g = GRIDS["c3"]()
    K = 130
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dpf.SolveOpts(precision=dpf.FP32, max_iter=60, check_every=10, lr=1e-3)
    tuned = dpf.dpf_autotune(y, ws, base, iters=10, n_case=K)
    # row_blocks 0 is the automatic (wave-aligned) choice
    assert tuned.lanes in (8, 16, 32) and tuned.warps in (4, 8) and tuned.row_blocks >= 0
    assert tuned.pair_cases in (0, 1, 2, 3)
    again = dpf.dpf_autotune(y, ws, base, iters=10, n_case=K)  # cached
    assert (again.lanes, again.warps, again.row_blocks, again.pair_cases) == \
        (tuned.lanes, tuned.warps, tuned.row_blocks, tuned.pair_cases)
    a = _solve(y, ws, K, tuned)
    b = _solve(y, ws, K, base)
    assert np.abs(a["va"] - b["va"]).max() < 1e-4 and np.abs(a["vm"] - b["vm"]).max() < 1e-4


def test_warm_start_and_host_io():
    g = GRIDS["g300"]()
    K = 3
    Y = grid_ybus(g)
    nr = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set)
    assert nr["converged"]
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    va0 = np.tile(nr["va"], (K, 1))
    vm0 = np.tile(nr["vm"], (K, 1))
    opts = dpf.SolveOpts(precision=dpf.FP64, flat_start=0, max_iter=10, check_every=1)
    r = _solve(y, ws, K, opts, va0=_t(va0), vm0=_t(vm0))
    # started at the NR solution: converged at the first test, nothing moved
    assert (r["iters"] == 0).all() and (r["status"] == dpf.CASE_CONVERGED).all()
    assert np.abs(r["va"] - va0).max() == 0.0
    # the same through host buffers
    h = {k: torch.zeros_like(torch.tensor(v)).pin_memory() for k, v in
         dict(va=va0, vm=vm0).items()}
    h["va"].copy_(torch.tensor(va0))
    h["vm"].copy_(torch.tensor(vm0))
    it = torch.zeros(K, dtype=torch.int32).pin_memory()
    st = torch.zeros(K, dtype=torch.int32).pin_memory()
    mx = torch.zeros(K, dtype=torch.float64).pin_memory()
    dpf.dpf_solve_batch(y, ws, opts, n_case=K, host_io=True, va=h["va"], vm=h["vm"], iters=it, status=st,
                        max_mismatch=mx)
    assert (it.numpy() == 0).all() and (st.numpy() == 0).all()
    assert np.abs(h["va"].numpy() - va0).max() == 0.0


def test_invalid_inputs_raise():
    g = GRIDS["c1"]()
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 2)
    br = dpf.dpf_ybus_bridges(y)
    bridge = int(np.flatnonzero(br)[0])
    va = torch.zeros((2, g.n_bus), dtype=torch.float64, device=DEV)
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_solve_batch(y, ws, None, n_case=2, va=va, vm=va.clone(),
                            outage=torch.tensor([bridge, -1], dtype=torch.int32, device=DEV))
    assert e.value.code == -2
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_solve_batch(y, ws, None, n_case=2, va=va, vm=va.clone(),
                            outage=torch.tensor([g.n_branch, -1], dtype=torch.int32, device=DEV))
    assert e.value.code == -1
    with pytest.raises(dpf.DPFError):
        dpf.dpf_solve_batch(y, ws, None, n_case=0, va=va, vm=va.clone())
    with pytest.raises(dpf.DPFError):
        dpf.dpf_solve_iterate(ws, 1)  # no begin
    # element offsets are 32-bit: n_bus * n_case >= 2^32 is rejected before any work
    big = 2 ** 32 // g.n_bus + 1
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_solve_batch(y, ws, None, n_case=big, va=va, vm=va.clone())
    assert e.value.code == -5


def test_diverged_case_is_flagged():
    """A NaN injection makes that case diverge; the others are unaffected."""
    g = GRIDS["c1"]()
    K = 3
    P = np.tile(g.p_spec, (K, 1))
    Q = np.tile(g.q_spec, (K, 1))
    P[1, g.pq[0]] = np.nan
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP64, max_iter=30, check_every=1), p_spec=_t(P), q_spec=_t(Q))
    assert r["status"][1] == dpf.CASE_DIVERGED
    ref = oracle.dpf_solve(grid_ybus(g), P[1], Q[1], g.bus_type, g.vm_set,
                           oracle.DPFOptions(max_iter=30), va_slack=g.va_slack)
    assert ref["status"] == oracle.dpf.DIVERGED and r["iters"][1] == ref["iters"]
    assert r["status"][0] == dpf.CASE_MAX_ITER and r["status"][2] == dpf.CASE_MAX_ITER
    assert r["iters"][0] == 30 and np.isfinite(r["va"][0]).all()
    # the same workspace, reused after a case diverged (and every case of a
    # batch stopped), solves a clean batch exactly as a fresh one does
    r_all = _solve(y, ws, K, dpf.SolveOpts(max_iter=40, check_every=5), p_spec=_t(np.full_like(P, np.nan)),
                   q_spec=_t(Q))
    assert (r_all["status"] == dpf.CASE_DIVERGED).all()
    opts = dpf.SolveOpts(max_iter=60, check_every=5)
    r1 = _solve(y, ws, K, opts, p_spec=_t(np.tile(g.p_spec, (K, 1))), q_spec=_t(Q))
    ws2 = dpf.dpf_workspace_create(y, K)
    r2 = _solve(y, ws2, K, opts, p_spec=_t(np.tile(g.p_spec, (K, 1))), q_spec=_t(Q))
    for key in ("va", "vm", "iters", "status"):
        assert np.array_equal(r1[key], r2[key]), key


def test_autograd_function():
    from paper_2603_28203_gb300.autograd import dpf_loss
    g = GRIDS["c1"]()
    Y = grid_ybus(g)
    K = 2
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    va, vm = _states(K, g.n_bus, 21, spread=0.05)
    tva = _t(va).requires_grad_(True)
    tvm = _t(vm).requires_grad_(True)
    L = dpf_loss(tva, tvm, y, ws, precision=dpf.FP64)
    (3.0 * L).backward()
    for k in range(K):
        Lk, d_va, d_vm = oracle.loss_grad(Y, va[k], vm[k], g.p_spec, g.q_spec, g.bus_type)
        assert np.abs(tva.grad[k].cpu().numpy() - 3 * d_va).max() <= 1e-10 * np.abs(d_va).max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_solve_repeats_bit_for_bit(precision):
    """Two identical batched solves give identical iterates, iteration counts,
    statuses and FP64 mismatches: the per-case loss that drives the scheduler
    is summed in a fixed order (no atomic sum), so no scheduling decision
    depends on the order in which CTAs finish."""
    g = GRIDS["c3"]()
    K = 130
    ells = np.concatenate([[-1], np.random.default_rng(12).choice(gridgen.n1_outages(g), K - 1, replace=False)])
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    prec = dict(fp32=dpf.FP32, fp64=dpf.FP64)[precision]
    opts = dpf.SolveOpts(precision=prec, max_iter=300, check_every=10, lr=1e-3)
    kw = dict(outage=_t(ells.astype(np.int32), torch.int32))
    a = _solve(y, ws, K, opts, **kw)
    b = _solve(y, ws, K, opts, **kw)
    for key in ("va", "vm", "iters", "status", "max_mismatch"):
        assert np.array_equal(a[key], b[key]), key


def test_c1_converges_to_nr_mixed():
    """DPF_MIXED (FP64 forward pass and voltages, FP32 adjoint and optimiser)
    reaches 1e-6 p.u. on the 30-bus grid, which FP32 iterations cannot (their
    current's cancellation error is ~1e-5 p.u. here), and lands on the NR
    solution; FP32 iterations of the same batch stall above 1e-6."""
    g = GRIDS["c1"]()
    Y = grid_ybus(g)
    K = 64
    rng = np.random.default_rng(5)
    sc = 1 + 0.05 * rng.uniform(-1, 1, (K, 1))
    P, Q = g.p_spec[None, :] * sc, g.q_spec[None, :] * sc
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(max_iter=20000, check_every=25, lr=1e-2)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.MIXED, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (r["status"] == dpf.CASE_CONVERGED).all() and (r["max_mismatch"] <= 1e-6).all()
    for k in (0, K // 2, K - 1):
        f, _ = oracle.mismatch(Y, r["va"][k], r["vm"][k], P[k], Q[k], g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12
        nr = oracle.nr_solve(Y, P[k], Q[k], g.bus_type, g.vm_set)
        assert np.abs(r["vm"][k] - nr["vm"]).max() < 1e-5
        assert np.abs(r["va"][k] - nr["va"]).max() < 1e-5
    f32 = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP32, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (f32["status"] != dpf.CASE_CONVERGED).all()


def test_mixed_n1_batch_against_oracle():
    """DPF_MIXED on N-1 cases of the 2,000-bus grid: the FP64 mismatch
    reported for each case equals the oracle's recomputation from the returned
    voltages, and the iterates stay within the FP32 bar of the oracle's FP64
    trajectory (the adjoint and the optimiser run in FP32)."""
    g = GRIDS["c3"]()
    K = 70
    outs = np.random.default_rng(13).choice(gridgen.n1_outages(g), K, replace=False).astype(np.int32)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.MIXED, max_iter=60, check_every=10, lr=1e-3),
               outage=_t(outs, torch.int32))
    for k in (0, K // 2, K - 1):
        keep = np.arange(g.n_branch) != outs[k]
        Yk = oracle.build_ybus(g.n_bus, g.f_bus[keep], g.t_bus[keep], g.r[keep], g.x[keep], g.b_ch[keep],
                               g.tap[keep])
        f, _ = oracle.mismatch(Yk, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-9
        ref = oracle.dpf_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set,
                               oracle.DPFOptions(lr=1e-3, max_iter=60, check_every=10), va_slack=g.va_slack)
        assert np.abs(r["va"][k] - ref["va"]).max() <= 5e-3
        assert np.abs(r["vm"][k] - ref["vm"]).max() <= 5e-3


@pytest.mark.parametrize("precision", ["fp32", "fp32r"])
def test_single_case_direct_rows_match_staged(precision):
    """A single-case FP32 solve reads its Y_bus rows straight from global
    memory (one wave of CTAs, no shared-memory staging); a batch of two runs
    the staged kernels.  With a constant rate (no loss-dependent schedule,
    whose sum order follows the row blocks) case 0 of the pair and the single
    case take identical steps: same iterates to the bit."""
    g = GRIDS["g300"]()
    prec = dict(fp32=dpf.FP32, fp32r=dpf.FP32R)[precision]
    opts = dpf.SolveOpts(precision=prec, max_iter=200, check_every=10, lr=1e-3, sched=dpf.SCHED_CONST)
    y = dpf.dpf_build_ybus(g)
    ws1 = dpf.dpf_workspace_create(y, 1)
    ws2 = dpf.dpf_workspace_create(y, 2)
    a = _solve(y, ws1, 1, opts)
    b = _solve(y, ws2, 2, opts)
    assert np.array_equal(a["va"][0], b["va"][0]) and np.array_equal(a["vm"][0], b["vm"][0])
    assert a["iters"][0] == b["iters"][0] and a["max_mismatch"][0] == b["max_mismatch"][0]
    c = _solve(y, ws1, 1, dpf.SolveOpts(stage_y=1, **{f: getattr(opts, f) for f in
                                                      ("precision", "max_iter", "check_every", "lr", "sched")}))
    assert np.array_equal(a["va"], c["va"]) and np.array_equal(a["vm"], c["vm"])
    Y = grid_ybus(g)
    f, _ = oracle.mismatch(Y, a["va"][0], a["vm"][0], g.p_spec, g.q_spec, g.bus_type)
    assert abs(np.abs(f).max() - a["max_mismatch"][0]) <= 1e-12 * np.abs(f).max()
