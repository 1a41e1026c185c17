"""GPU DC approximation (dpf_dc_solve, batched CG) against the oracle's
dc_solve: N-1 cases and per-case injections on the 2,000-bus grid, islands,
a single small case, the residual of the 10,000-bus grid computed by the
oracle, bridge outages rejected, and the DC start of the DPF solve."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.power import SLACK

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


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _oracle_dc(g, p, ell=-1):
    return oracle.dc_solve(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, p, va_slack=g.va_slack, outage=ell)


def test_dc_n1_and_per_case_injections_match_oracle():
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 40
    ells = np.concatenate([[-1], np.random.default_rng(3).choice(gridgen.n1_outages(g), K - 1, replace=False)])
    P, _ = gridgen.time_series(g, K, seed=9)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    out = dpf.dpf_dc_solve(y, ws, K, p_spec=_t(P), outage=_t(ells.astype(np.int32), torch.int32), tol=1e-12)
    th = out["va"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    assert (it > 0).all() and (out["rel_residual"].cpu().numpy() <= 1e-12).all()
    for k in range(K):
        ref = _oracle_dc(g, P[k], int(ells[k]))
        assert np.abs(th[k] - ref).max() <= 1e-7 * np.abs(ref).max(), k
        assert th[k][g.bus_type == SLACK][0] == g.va_slack


def test_dc_fp32_vectors_at_a_loose_tolerance():
    """tol >= 1e-5 runs the CG on FP32 vectors: every case stops with the
    recurrence's |r| / |r0| <= tol, and the true relative residual of the
    returned angles, recomputed by the oracle in FP64, stays within 10 tol
    (the FP32 recurrence drifts from it by rounding only)."""
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 40
    ells = np.concatenate([[-1], np.random.default_rng(5).choice(gridgen.n1_outages(g), K - 1, replace=False)])
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    tol = 1e-4
    out = dpf.dpf_dc_solve(y, ws, K, outage=_t(ells.astype(np.int32), torch.int32), tol=tol)
    th = out["va"].cpu().numpy()
    assert (out["rel_residual"].cpu().numpy() <= tol).all()
    u = np.where(g.bus_type != SLACK)[0]
    for k in range(K):
        B = oracle.dc_matrix(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, int(ells[k]))
        rhs = g.p_spec[u] - B[u][:, g.bus_type == SLACK] @ np.full((g.bus_type == SLACK).sum(), g.va_slack)
        true = np.linalg.norm((B[u][:, u] @ th[k][u]) - rhs) / np.linalg.norm(rhs)
        assert true <= 10 * tol, (k, true)
        assert th[k][g.bus_type == SLACK][0] == g.va_slack


def test_dc_islands_and_single_case():
    grids = [gridgen.make_grid(n, 40 + i, load_scale=0.2) for i, n in enumerate([30, 55, 80])]
    cat = gridgen.concat_grids(grids)
    cat.va_slack = 0.07
    y = dpf.dpf_build_ybus(cat)
    ws = dpf.dpf_workspace_create(y, 3)
    out = dpf.dpf_dc_solve(y, ws, 3, tol=1e-13)  # the grid's injections for every case
    ref = _oracle_dc(cat, cat.p_spec)
    for k in range(3):
        assert np.abs(out["va"][k].cpu().numpy() - ref).max() <= 1e-9
    g = gridgen.config_grid("c1_30bus_fp64")
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 1)
    out = dpf.dpf_dc_solve(y, ws, 1, tol=1e-14)
    assert np.abs(out["va"][0].cpu().numpy() - _oracle_dc(g, g.p_spec)).max() <= 1e-12


def test_dc_residual_at_10k_buses():
    g = gridgen.config_grid("c2_10kbus")
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 4)
    P = np.stack([g.p_spec * s for s in (1.0, 0.5, 1.5, 0.9)])
    out = dpf.dpf_dc_solve(y, ws, 4, p_spec=_t(P), tol=1e-11, max_iter=20000)
    B = oracle.dc_matrix(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap)
    u = g.bus_type != SLACK
    for k in range(4):
        th = out["va"][k].cpu().numpy()
        r = (B @ th - P[k])[u]
        assert np.abs(r).max() <= 1e-8 * np.abs(P[k][u]).max(), k


def test_dc_rejects_bridge_outage():
    g = gridgen.config_grid("c3_n1_2kbus")
    bridge = int(np.where(gridgen.bridges(g.n_bus, g.f_bus, g.t_bus))[0][0])
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 1)
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_dc_solve(y, ws, 1, outage=_t(np.array([bridge], np.int32), torch.int32))
    assert e.value.code == -2  # DPF_E_ISLANDED


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dpf_dc_start_begins_at_the_dc_angles(precision):
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 8
    ells = np.concatenate([[-1], gridgen.n1_outages(g)[:K - 1]]).astype(np.int32)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    prec = dict(fp64=dpf.FP64, fp32=dpf.FP32)[precision]
    res = dict(va=torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV),
               vm=torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV),
               iters=torch.zeros(K, dtype=torch.int32, device=DEV))
    dpf.dpf_solve_batch(y, ws, dpf.SolveOpts(precision=prec, max_iter=0, dc_start=1), n_case=K,
                        outage=_t(ells, torch.int32), **res)
    va = res["va"].cpu().numpy()
    vm = res["vm"].cpu().numpy()
    fva, fvm = oracle.flat_start(g.bus_type, g.vm_set, g.va_slack)
    for k in range(K):
        ref = _oracle_dc(g, g.p_spec, int(ells[k]))
        assert np.abs(va[k] - ref).max() <= 1e-8 * np.abs(ref).max()
        # |V| as flat-started (FP32 mode keeps it as a double-float, ~48 bits)
        assert np.abs(vm[k] - fvm).max() <= (0.0 if precision == "fp64" else 1e-14)


def _base_state(g):
    """The oracle's Newton solution of the intact grid (the N-1 batch's start)."""
    from oracle.ybus import grid_ybus
    r = oracle.nr_solve(grid_ybus(g), g.p_spec, g.q_spec, g.bus_type, g.vm_set, va_slack=g.va_slack, tol=1e-10)
    assert r["converged"]
    return r["va"], r["vm"]


def _shift(g, theta, ell):
    return oracle.dc_outage_shift(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, theta, int(ell))


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("shared", [True, False])
def test_dc_outage_shift_of_a_warm_start(precision, shared):
    """dc_start with a warm start and outages: every case begins at its start
    angles plus the oracle's DC outage shift of them (|V| as started; a case
    without an outage keeps its start), and the FP64 mismatch reported at
    that start is the oracle's.  300-bus grid: a shared start (the base
    case's Newton solution) or per-case starts (that solution perturbed)."""
    from oracle.ybus import grid_ybus
    g = gridgen.make_grid(300, 5, load_scale=0.1)
    outs = gridgen.n1_outages(g)
    K = 37
    ells = np.concatenate([[-1], outs[::max(1, outs.size // (K - 1))][:K - 1]]).astype(np.int32)
    va0, vm0 = _base_state(g)
    rng = np.random.default_rng(4)
    VA = np.tile(va0, (K, 1)) + (0.0 if shared else 1e-3 * rng.standard_normal((K, g.n_bus)))
    VM = np.tile(vm0, (K, 1))
    VA[:, g.bus_type == SLACK] = g.va_slack
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    prec = dict(fp64=dpf.FP64, fp32r=dpf.FP32R)[precision]
    res = dict(va=_t(VA), vm=_t(VM), iters=torch.zeros(K, dtype=torch.int32, device=DEV),
               status=torch.zeros(K, dtype=torch.int32, device=DEV),
               max_mismatch=torch.zeros(K, dtype=torch.float64, device=DEV))
    start = dict(va_start=_t(va0), vm_start=_t(vm0)) if shared else {}
    opts = dpf.SolveOpts(precision=prec, max_iter=0, flat_start=0, dc_start=1, dc_tol=1e-12)
    dpf.dpf_solve_batch(y, ws, opts, n_case=K, outage=_t(ells, torch.int32), **start, **res)
    va = res["va"].cpu().numpy()
    vm = res["vm"].cpu().numpy()
    mm = res["max_mismatch"].cpu().numpy()
    Y = grid_ybus(g)
    for k in range(K):
        d = _shift(g, VA[k], ells[k])
        ref = VA[k] + d
        assert np.abs(va[k] - ref).max() <= 1e-8 * max(np.abs(d).max(), 1e-6), k
        if ells[k] < 0:  # (the FP32R master is a double-float pair, ~48 bits)
            assert np.abs(va[k] - VA[k]).max() <= (0.0 if precision == "fp64" else 1e-14)
        assert np.abs(vm[k] - VM[k]).max() <= (0.0 if precision == "fp64" else 1e-14)
        # the reported FP64 mismatch of the start: the oracle's on Y_bus without the branch
        keep = np.arange(g.n_branch) != ells[k]
        Yk = Y if ells[k] < 0 else oracle.build_ybus(g.n_bus, g.f_bus[keep], g.t_bus[keep], g.r[keep], g.x[keep],
                                                       g.b_ch[keep], g.tap[keep])
        f, _ = oracle.mismatch(Yk, va[k], vm[k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - mm[k]) <= 1e-10 * max(1.0, np.abs(f).max()), k


def test_dc_outage_shift_through_host_buffers():
    """The shifted start through host_io (outage list and shared start from
    pinned host memory, results back to it: the benchmark's e2e path) equals
    the device-buffer call bit for bit, 200 refined FP32 iterations."""
    g = gridgen.make_grid(300, 5, load_scale=0.1)
    outs = gridgen.n1_outages(g)[:40].astype(np.int32)
    K, N = outs.size, g.n_bus
    va0, vm0 = _base_state(g)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    o = dpf.SolveOpts(precision=dpf.FP32R, max_iter=200, flat_start=0, dc_start=1, dc_tol=1e-4, dc_max_iter=100,
                      check_every=50, gate=5e-6)

    def outs_on(dev):
        mk = (lambda shape, dt: torch.zeros(shape, dtype=dt).pin_memory()) if dev == "cpu" else \
             (lambda shape, dt: torch.zeros(shape, dtype=dt, device=DEV))
        return dict(va=mk((K, N), torch.float64), vm=mk((K, N), torch.float64), iters=mk(K, torch.int32),
                    status=mk(K, torch.int32), max_mismatch=mk(K, torch.float64))

    d = outs_on("cuda")
    dpf.dpf_solve_batch(y, ws, o, n_case=K, outage=_t(outs, torch.int32), va_start=_t(va0), vm_start=_t(vm0), **d)
    h = outs_on("cpu")
    pin = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt).pin_memory()
    dpf.dpf_solve_batch(y, ws, o, n_case=K, host_io=True, outage=pin(outs, torch.int32), va_start=pin(va0),
                        vm_start=pin(vm0), **h)
    torch.cuda.synchronize()
    for k in d:
        assert torch.equal(d[k].cpu(), h[k]), k


def test_dc_outage_shift_full_n1_batch_in_the_benchmark_settings():
    """The whole 2,000-bus N-1 batch started as the benchmark starts it (the
    base case's Newton state shared, refined FP32, the shift's CG stopped at
    presets.N1_DC_START's relative residual or iteration cap).  Sampled
    cases: the oracle's relative residual of the returned shift,
    |B' dtheta - (B - B') theta| / |(B - B') theta| over the non-slack rows,
    is within the CG tolerance -- or, for a case the cap stopped, the error
    in the energy norm of B' (which CG lowers at every step, unlike the
    residual) is below half that of no shift -- slack angles and every |V|
    keep the base state, and the shift lowers the median starting mismatch
    of the batch."""
    from paper_2603_28203_gb300.presets import N1_DC_START
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g).astype(np.int32)
    K = outs.size
    va0, vm0 = _base_state(g)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)

    def start(dc):
        res = dict(va=torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV),
                   vm=torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV),
                   max_mismatch=torch.zeros(K, dtype=torch.float64, device=DEV))
        o = dpf.SolveOpts(precision=dpf.FP32R, max_iter=0, flat_start=0, **dict(N1_DC_START, dc_start=dc))
        dpf.dpf_solve_batch(y, ws, o, n_case=K, outage=_t(outs, torch.int32), va_start=_t(va0), vm_start=_t(vm0),
                            **res)
        return res["va"].cpu().numpy(), res["vm"].cpu().numpy(), res["max_mismatch"].cpu().numpy()

    va, vm, mm = start(1)
    _, _, mm0 = start(0)
    B = oracle.dc_matrix(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap)
    u = np.where(g.bus_type != SLACK)[0]
    for k in np.random.default_rng(2).choice(K, 8, replace=False):
        Bo = oracle.dc_matrix(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, int(outs[k]))
        d = va[k] - va0
        rhs = ((B - Bo) @ va0)[u]
        rel = np.linalg.norm((Bo @ d)[u] - rhs) / np.linalg.norm(rhs)
        ex = _shift(g, va0, outs[k])[u]
        Buu = Bo[u][:, u]
        e = d[u] - ex
        energy = np.sqrt(e @ (Buu @ e) / (ex @ (Buu @ ex)))
        assert rel <= 1.01 * N1_DC_START["dc_tol"] or energy < 0.5, (k, rel, energy)
        assert np.all(d[g.bus_type == SLACK] == 0.0)
        assert np.abs(vm[k] - vm0).max() <= 1e-14
    assert np.median(mm) < 0.8 * np.median(mm0)
