"""GPU parity of the refined FP32 iterations (DPF_FP32R) against the oracle.

DPF_FP32R keeps every per-iteration operation in FP32 but evaluates the
mismatch as a correction to the FP64 residual of the case's most recent
convergence test, so its iterations resolve mismatches far below the ~1e-5
p.u. at which plain FP32 iterations stall.  The bars: a converged case has an
FP64 max mismatch <= 1e-6 p.u. (recomputed by the oracle from the returned
voltages, 1e-12 absolute) and lies on the oracle's Newton-Raphson root
(Alg. 2, from the flat start: the high-voltage root).  On the 30-bus grid
that means |V| within 1e-5 p.u. and theta within 1e-5 rad of it.  On the
2,000-bus grid the Jacobian's smallest singular value is ~6e-4, so a state
whose residual is 1e-6 p.u. can lie ~1e-4 from the exact root: there the
test is that the gap is exactly the first-order image of the residual,
x_DPF - x_NR = J^-1 f(x_DPF) (same root, no other error).
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
from paper_2603_28203_gb300.presets import N1_WARM  # noqa: E402

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


def _solve(y, ws, K, opts, va0=None, vm0=None, **kw):
    N = y.n_bus
    res = dict(va=torch.zeros((K, N), dtype=torch.float64, device=DEV),
               vm=torch.zeros((K, N), dtype=torch.float64, device=DEV),
               iters=torch.zeros(K, dtype=torch.int32, device=DEV),
               status=torch.zeros(K, dtype=torch.int32, device=DEV),
               max_mismatch=torch.zeros(K, dtype=torch.float64, device=DEV),
               loss=torch.zeros(K, dtype=torch.float64, device=DEV))
    if va0 is not None:
        res["va"].copy_(va0)
        res["vm"].copy_(vm0)
    dpf.dpf_solve_batch(y, ws, opts, n_case=K, **res, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


def _ybus_without(g, ell):
    keep = np.arange(g.n_branch) != ell
    return oracle.build_ybus(g.n_bus, g.f_bus[keep], g.t_bus[keep], g.r[keep], g.x[keep], g.b_ch[keep], g.tap[keep])


def test_c1_batch_converges_to_nr():
    """30-bus grid, 64 load variants from the flat start (Table 2, lr 1e-2):
    every case reaches 1e-6 p.u. in FP32R and lands on the Newton solution;
    plain FP32 iterations of the same batch stall above 1e-6; FP32R needs
    about as many iterations as FP64 (same algorithm, same schedule)."""
    g = gridgen.config_grid("c1_30bus_fp64")
    Y = grid_ybus(g)
    K = 64
    rng = np.random.default_rng(5)
    sc = 1 + 0.05 * rng.uniform(-1, 1, (K, 1))
    P, Q = g.p_spec[None, :] * sc, g.q_spec[None, :] * sc
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(max_iter=20000, check_every=25, lr=1e-2)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP32R, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (r["status"] == dpf.CASE_CONVERGED).all() and (r["max_mismatch"] <= 1e-6).all()
    for k in range(K):
        f, _ = oracle.mismatch(Y, r["va"][k], r["vm"][k], P[k], Q[k], g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12
    for k in (0, 17, K // 2, K - 1):
        nr = oracle.nr_solve(Y, P[k], Q[k], g.bus_type, g.vm_set)
        assert nr["converged"]
        assert np.abs(r["vm"][k] - nr["vm"]).max() < 1e-5
        assert np.abs(r["va"][k] - nr["va"]).max() < 1e-5
    f64 = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP64, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (f64["status"] == dpf.CASE_CONVERGED).all()
    assert abs(np.median(r["iters"]) - np.median(f64["iters"])) <= 0.1 * np.median(f64["iters"])
    f32 = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP32, **base), p_spec=_t(P), q_spec=_t(Q))
    assert (f32["status"] != dpf.CASE_CONVERGED).all()


def test_n1_warm_start_converged_cases_match_newton():
    """2,000-bus N-1 batch, every case warm-started from the base case's
    solution (the base case solved by the library's Newton-Raphson), FP32R
    with the warm-start settings (presets.N1_WARM), 5,000 iterations.  At least 20 cases converge; for each converged case the
    reported FP64 mismatch equals the oracle's recomputation on Y_bus rebuilt
    without the outaged branch, and the state is the oracle's Newton solution
    of that case (same root) up to the first-order image of its residual:
    x_DPF - x_NR = J^-1 f(x_DPF) within 1e-7 (the gap itself reaches ~1e-4
    on this grid: ||J^-1||_inf ~1,300)."""
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g)
    K, N = outs.size, g.n_bus
    y = dpf.dpf_build_ybus(g)
    nrh = dpf.dpf_nr_create(y, 1)
    bva = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    bvm = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    bst = torch.zeros(1, dtype=torch.int32, device=DEV)
    dpf.dpf_nr_solve(nrh, precision=dpf.FP64, tol=1e-10, max_iter=20, n_case=1, va=bva, vm=bvm, status=bst)
    torch.cuda.synchronize()
    assert int(bst[0]) == dpf.CASE_CONVERGED
    nrh.free()
    ws = dpf.dpf_workspace_create(y, K)
    opts = dpf.SolveOpts(precision=dpf.FP32R, max_iter=5000, check_every=25, flat_start=0, **N1_WARM)
    r = _solve(y, ws, K, opts, va_start=bva[0], vm_start=bvm[0], outage=_t(outs, torch.int32))
    conv = np.nonzero(r["status"] == dpf.CASE_CONVERGED)[0]
    assert conv.size >= 20, conv.size
    assert (r["max_mismatch"][conv] <= 1e-6).all()
    import scipy.sparse.linalg as spla
    pvpq, pq = oracle.learnable_sets(g.bus_type)
    for k in conv:
        Yk = _ybus_without(g, int(outs[k]))
        f, _ = oracle.mismatch(Yk, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12, k
        nr = oracle.nr_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set, va_slack=g.va_slack)
        assert nr["converged"], k
        dx = np.concatenate([r["va"][k][pvpq] - nr["va"][pvpq], r["vm"][k][pq] - nr["vm"][pq]])
        lin = spla.spsolve(oracle.jacobian_f(Yk, nr["va"], nr["vm"], g.bus_type), f)
        assert np.abs(dx - lin).max() <= 1e-7, (k, np.abs(dx - lin).max(), np.abs(dx).max())
    # the cases left unconverged still report their true FP64 mismatch
    rest = np.setdiff1d(np.arange(K), conv)
    for k in rest[:: max(1, rest.size // 4)][:4]:
        f, _ = oracle.mismatch(_ybus_without(g, int(outs[k])), r["va"][k], r["vm"][k], g.p_spec, g.q_spec,
                               g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12 * max(1.0, np.abs(f).max()), k


def test_n1_benchmark_configuration_dc_shift():
    """The benchmark's N-1 step as bench.py runs it: the base case by the
    library's Newton-Raphson, every case's start shifted by the DC angle
    change of its outage, presets.N1_DC / N1_DC_START / N1_DC_TEST, the
    budget N1_DC_BUDGET, the autotuned launch shape.  At least 150 of the
    2,379 cases converge (219 when this was written; the count moves by
    ~10% with the last bits of the arithmetic).  Sampled converged cases: the
    reported FP64 mismatch is the oracle's on Y_bus rebuilt without the
    branch, and the state is the oracle's Newton root up to J^-1 f (1e-7);
    sampled unconverged cases report their true mismatch."""
    from paper_2603_28203_gb300.presets import N1_DC, N1_DC_BUDGET, N1_DC_START, N1_DC_TEST
    import scipy.sparse.linalg as spla
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g)
    K, N = outs.size, g.n_bus
    y = dpf.dpf_build_ybus(g)
    nrh = dpf.dpf_nr_create(y, 1)
    bva = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    bvm = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    dpf.dpf_nr_solve(nrh, precision=dpf.FP64, tol=1e-10, max_iter=20, n_case=1, va=bva, vm=bvm)
    nrh.free()
    ws = dpf.dpf_workspace_create(y, K)
    od = _t(outs, torch.int32)
    opts = dpf.SolveOpts(precision=dpf.FP32R, tol=1e-6, max_iter=N1_DC_BUDGET, flat_start=0, **N1_DC, **N1_DC_START,
                         **N1_DC_TEST)
    opts = dpf.dpf_autotune(y, ws, opts, iters=50, n_case=K, outage=od, va_start=bva[0], vm_start=bvm[0])
    r = _solve(y, ws, K, opts, va_start=bva[0], vm_start=bvm[0], outage=od)
    conv = np.nonzero(r["status"] == dpf.CASE_CONVERGED)[0]
    assert conv.size >= 150, conv.size
    assert (r["max_mismatch"][conv] <= 1e-6).all()
    assert (r["iters"][conv] <= N1_DC_BUDGET).all()
    pvpq, pq = oracle.learnable_sets(g.bus_type)
    for k in conv[:: max(1, conv.size // 5)][:5]:
        Yk = _ybus_without(g, int(outs[k]))
        f, _ = oracle.mismatch(Yk, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12, k
        nr = oracle.nr_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set, va_slack=g.va_slack)
        assert nr["converged"], k
        dx = np.concatenate([r["va"][k][pvpq] - nr["va"][pvpq], r["vm"][k][pq] - nr["vm"][pq]])
        lin = spla.spsolve(oracle.jacobian_f(Yk, nr["va"], nr["vm"], g.bus_type), f)
        assert np.abs(dx - lin).max() <= 1e-7, (k, np.abs(dx - lin).max(), np.abs(dx).max())
    rest = np.setdiff1d(np.arange(K), conv)
    for k in rest[:: max(1, rest.size // 3)][:3]:
        f, _ = oracle.mismatch(_ybus_without(g, int(outs[k])), r["va"][k], r["vm"][k], g.p_spec, g.q_spec,
                               g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12 * max(1.0, np.abs(f).max()), k


@pytest.mark.parametrize("outages", [False, True])
def test_pair_kernels_match_single(outages):
    """FP32R batches of >= 64 cases run two cases per thread: the same
    iterates, iteration counts and reported mismatches as one per thread."""
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 100
    kw = {}
    if outages:
        ells = np.concatenate([[-1], np.random.default_rng(8).choice(gridgen.n1_outages(g), K - 1, replace=False)])
        kw["outage"] = _t(ells.astype(np.int32), torch.int32)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    base = dict(precision=dpf.FP32R, max_iter=100, check_every=10, lr=1e-3)
    a = _solve(y, ws, K, dpf.SolveOpts(pair_cases=3, **base), **kw)
    b = _solve(y, ws, K, dpf.SolveOpts(pair_cases=0, **base), **kw)
    assert np.abs(a["va"] - b["va"]).max() < 1e-4 and np.abs(a["vm"] - b["vm"]).max() < 1e-4
    assert np.abs(a["max_mismatch"] - b["max_mismatch"]).max() < 1e-4 * np.abs(b["max_mismatch"]).max()
    assert (a["iters"] == b["iters"]).all()


def test_refined_iterations_repeat_bit_for_bit():
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 130
    ells = np.concatenate([[-1], np.random.default_rng(12).choice(gridgen.n1_outages(g), K - 1, replace=False)])
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    opts = dpf.SolveOpts(precision=dpf.FP32R, max_iter=300, check_every=10, lr=1e-3)
    kw = dict(outage=_t(ells.astype(np.int32), torch.int32))
    a = _solve(y, ws, K, opts, **kw)
    b = _solve(y, ws, K, opts, **kw)
    for key in ("va", "vm", "iters", "status", "max_mismatch"):
        assert np.array_equal(a[key], b[key]), key


def test_refined_tracks_fp64_oracle_trajectory():
    """300-bus grid, 8 cases, constant rate: FP32R iterates stay within the
    FP32 bar (1e-3) of the oracle's FP64 Alg. 1 loop, and the reported FP64
    mismatch is the oracle's of the returned state."""
    g = gridgen.make_grid(300, 5, load_scale=0.1)
    Y = grid_ybus(g)
    K = 8
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    r = _solve(y, ws, K, dpf.SolveOpts(precision=dpf.FP32R, max_iter=200, check_every=10, lr=1e-3,
                                       sched=dpf.SCHED_CONST))
    ref = oracle.dpf_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set,
                           oracle.DPFOptions(lr=1e-3, max_iter=200, check_every=10, sched="const"))
    for k in range(K):
        assert np.abs(r["va"][k] - ref["va"]).max() < 1e-3
        assert np.abs(r["vm"][k] - ref["vm"]).max() < 1e-3
        f, _ = oracle.mismatch(Y, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(r["max_mismatch"][k] - np.abs(f).max()) <= 1e-12 * np.abs(f).max()


def test_shared_start_equals_per_case_starts():
    """va_start/vm_start (one start for every case, device or host) give the
    same solve, bit for bit, as the same state copied into every case's
    va/vm."""
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g)[:70].astype(np.int32)
    K, N = outs.size, g.n_bus
    rng = np.random.default_rng(3)
    va0 = 0.01 * rng.standard_normal(N)
    vm0 = 1.0 + 0.01 * rng.standard_normal(N)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    opts = dpf.SolveOpts(precision=dpf.FP32R, max_iter=200, check_every=25, flat_start=0, lr=1e-4)
    a = _solve(y, ws, K, opts, va0=_t(np.tile(va0, (K, 1))), vm0=_t(np.tile(vm0, (K, 1))), outage=_t(outs, torch.int32))
    b = _solve(y, ws, K, opts, va_start=_t(va0), vm_start=_t(vm0), outage=_t(outs, torch.int32))
    for key in ("va", "vm", "iters", "status", "max_mismatch"):
        assert np.array_equal(a[key], b[key]), key
    h = {k: torch.zeros(v.shape, dtype=v.dtype).pin_memory() for k, v in
         dict(va=torch.zeros((K, N), dtype=torch.float64), vm=torch.zeros((K, N), dtype=torch.float64),
              iters=torch.zeros(K, dtype=torch.int32), status=torch.zeros(K, dtype=torch.int32),
              max_mismatch=torch.zeros(K, dtype=torch.float64)).items()}
    dpf.dpf_solve_batch(y, ws, opts, n_case=K, host_io=True, outage=torch.tensor(outs).pin_memory(),
                        va_start=torch.tensor(va0).pin_memory(), vm_start=torch.tensor(vm0).pin_memory(), **h)
    for key in ("va", "vm", "iters", "status", "max_mismatch"):
        assert np.array_equal(a[key], h[key].numpy()), key
    with pytest.raises(dpf.DPFError):  # va_start without vm_start
        dpf.dpf_solve_batch(y, ws, opts, n_case=K, va_start=_t(va0), va=_t(np.zeros((K, N))), vm=_t(np.zeros((K, N))))


def test_refined_option_checks():
    """FP32R is a solve precision: the evaluation entry points reject it."""
    g = gridgen.config_grid("c1_30bus_fp64")
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, 2)
    va = torch.zeros((2, g.n_bus), dtype=torch.float64, device=DEV)
    with pytest.raises(dpf.DPFError):
        dpf.dpf_power(y, ws, va, va + 1, precision=dpf.FP32R)
    with pytest.raises(dpf.DPFError):
        dpf.dpf_loss_backward(y, ws, va, va + 1, precision=dpf.FP32R)
    with pytest.raises(dpf.DPFError):  # a negative renewal interval
        dpf.dpf_solve_batch(y, ws, dpf.SolveOpts(precision=dpf.FP32R, refresh_every=-1), n_case=2, va=va,
                            vm=va + 1)
    with pytest.raises(dpf.DPFError):  # the DC start needs a positive tolerance and iteration cap
        dpf.dpf_solve_batch(y, ws, dpf.SolveOpts(dc_start=1, dc_tol=0.0), n_case=2, va=va, vm=va + 1)
    with pytest.raises(dpf.DPFError):
        dpf.dpf_solve_batch(y, ws, dpf.SolveOpts(dc_start=1, dc_max_iter=0), n_case=2, va=va, vm=va + 1)


def test_300_bus_n1_converged_cases_within_state_bar():
    """A 300-bus grid (seed 3; ||J^-1||_inf ~130), every N-1 case started from
    the base case (oracle-independent: the library's Newton-Raphson), refined
    FP32 at the tighter tolerance 1e-7 p.u. (which implies the 1e-6 bar), the
    warm-start settings, 10,000 iterations.  Every converged case (at least 3)
    has its reported FP64 mismatch equal to the oracle's recomputation and
    |V| within 1e-5 p.u., theta within 1e-5 rad of the oracle's Newton
    solution of that case: the target's state bars, met here at 1e-7 (at
    1e-6 the residual's first-order image reaches ~7e-5 on this grid)."""
    g = gridgen.make_grid(300, 3, load_scale=0.1)
    outs = gridgen.n1_outages(g).astype(np.int32)
    K, N = outs.size, g.n_bus
    y = dpf.dpf_build_ybus(g)
    nrh = dpf.dpf_nr_create(y, 1)
    bva = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    bvm = torch.zeros((1, N), dtype=torch.float64, device=DEV)
    bst = torch.zeros(1, dtype=torch.int32, device=DEV)
    dpf.dpf_nr_solve(nrh, precision=dpf.FP64, tol=1e-10, max_iter=20, n_case=1, va=bva, vm=bvm, status=bst)
    torch.cuda.synchronize()
    assert int(bst[0]) == dpf.CASE_CONVERGED
    nrh.free()
    ws = dpf.dpf_workspace_create(y, K)
    opts = dpf.SolveOpts(precision=dpf.FP32R, tol=1e-7, max_iter=10000, check_every=25, flat_start=0, **N1_WARM)
    r = _solve(y, ws, K, opts, va_start=bva[0], vm_start=bvm[0], outage=_t(outs, torch.int32))
    conv = np.nonzero(r["status"] == dpf.CASE_CONVERGED)[0]
    assert conv.size >= 3, conv.size
    for k in conv:
        Yk = _ybus_without(g, int(outs[k]))
        f, _ = oracle.mismatch(Yk, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-12 and r["max_mismatch"][k] <= 1e-7, k
        nr = oracle.nr_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set, va_slack=g.va_slack)
        assert nr["converged"], k
        assert np.abs(r["vm"][k] - nr["vm"]).max() < 1e-5, (k, np.abs(r["vm"][k] - nr["vm"]).max())
        assert np.abs(r["va"][k] - nr["va"]).max() < 1e-5, (k, np.abs(r["va"][k] - nr["va"]).max())
