"""GPU parity of the batched Newton-Raphson solver (Alg. 2, dpf_nr_solve)
against the oracle's Newton-Raphson (its own Jacobian, scipy's sparse LU).

Both run Alg. 2 in FP64 from the same start with the same stop test, so
with the FP64 factor they take the same number of Newton steps and land on
the same solution; the bar on the state is 1e-9 (a mismatch below 1e-10
p.u. fixes the state to about cond(J) 1e-10).  The FP32 factor (FP64
mismatch and update) reaches the same solution in at least as many steps.
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
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2603_28203_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    dpf.lib()


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _nr(y, nr, K, precision=dpf.FP64, tol=TOL, max_iter=20, flat=True, va=None, vm=None, lanes=0, fallback=False,
        **kw):
    N = y.n_bus
    out = dict(va=_t(va) if va is not None else torch.zeros((K, N), dtype=torch.float64, device=DEV),
               vm=_t(vm) if vm is not None else torch.ones((K, N), dtype=torch.float64, device=DEV),
               iters=torch.empty(K, dtype=torch.int32, device=DEV),
               status=torch.empty(K, dtype=torch.int32, device=DEV),
               max_mismatch=torch.empty(K, dtype=torch.float64, device=DEV),
               loss=torch.empty(K, dtype=torch.float64, device=DEV))
    dpf.dpf_nr_solve(nr, precision=precision, tol=tol, max_iter=max_iter, flat_start=flat, lanes=lanes,
                     fallback=fallback, n_case=K, **out, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_c1_flat_start_matches_oracle_nr(precision):
    g = gridgen.config_grid("c1_30bus_fp64")
    Y = grid_ybus(g)
    ref = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set, tol=TOL)
    assert ref["converged"]
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, 1)
    r = _nr(y, nr, 1, precision=dpf.FP64 if precision == "fp64" else dpf.FP32)
    assert r["status"][0] == dpf.CASE_CONVERGED and r["max_mismatch"][0] <= TOL
    np.testing.assert_allclose(r["va"][0], ref["va"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["vm"][0], ref["vm"], rtol=0, atol=1e-9)
    f, _ = oracle.mismatch(Y, r["va"][0], r["vm"][0], g.p_spec, g.q_spec, g.bus_type)
    assert abs(np.abs(f).max() - r["max_mismatch"][0]) <= 1e-13
    assert abs(r["loss"][0] - oracle.loss(Y, r["va"][0], r["vm"][0], g.p_spec, g.q_spec, g.bus_type)) <= 1e-20
    if precision == "fp64":
        assert r["iters"][0] == ref["iters"]
    else:
        assert r["iters"][0] >= ref["iters"]


def test_n1_batch_matches_oracle_case_by_case():
    """70 N-1 cases of the 2,000-bus grid (several tiles of cases, a ragged
    last tile) in one call, every sampled case against the oracle's NR on
    Y_bus rebuilt without the branch."""
    g = gridgen.config_grid("c3_n1_2kbus")
    K = 70
    outs = np.random.default_rng(21).choice(gridgen.n1_outages(g), K, replace=False).astype(np.int32)
    outs[5] = -1  # the base case in the middle of the batch
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, K)
    r = _nr(y, nr, K, outage=_t(outs, torch.int32))
    assert (r["status"] == dpf.CASE_CONVERGED).all()
    assert (r["max_mismatch"] <= TOL).all()
    for k in (0, 5, 17, 40, K - 1):
        Yk = grid_ybus(g.without_branch(int(outs[k]))) if outs[k] >= 0 else grid_ybus(g)
        ref = oracle.nr_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set, tol=TOL)
        assert ref["converged"]
        assert r["iters"][k] == ref["iters"], k
        assert np.abs(r["va"][k] - ref["va"]).max() <= 1e-9, k
        assert np.abs(r["vm"][k] - ref["vm"]).max() <= 1e-9, k
        f, _ = oracle.mismatch(Yk, r["va"][k], r["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r["max_mismatch"][k]) <= 1e-13, k


def test_full_n1_batch_fp32_factor_converges_to_the_fp64_solution():
    """All N-1 cases of the 2,000-bus grid (the benchmark's batch).  A few
    outages leave the grid without a solution reachable from the flat start:
    every case the GPU does not converge is one where the oracle's NR fails
    too (infeasible, not counted as a solve), and they are under 1% of the
    batch.  Where both factors converge, the FP32 factor reaches the FP64
    tolerance and the FP64 factor's solution in at least as many steps; its
    reported mismatch equals the oracle's recomputation on sampled cases."""
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g).astype(np.int32)
    K = outs.size
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, K)
    r64 = _nr(y, nr, K, outage=_t(outs, torch.int32))
    r32 = _nr(y, nr, K, precision=dpf.FP32, outage=_t(outs, torch.int32))
    conv = (r64["status"] == dpf.CASE_CONVERGED) & (r32["status"] == dpf.CASE_CONVERGED)
    assert (~conv).sum() <= K // 100
    for k in np.flatnonzero(~conv):
        Yk = grid_ybus(g.without_branch(int(outs[k])))
        ref = oracle.nr_solve(Yk, g.p_spec, g.q_spec, g.bus_type, g.vm_set, tol=TOL, max_iter=20)
        assert not ref["converged"], k
    for r in (r64, r32):
        assert (r["max_mismatch"][conv] <= TOL).all()
    assert (r32["iters"][conv] >= r64["iters"][conv]).all()
    # Both states pass the FP64 test (|f| <= 1e-10), which pins each to the
    # exact solution only up to J^-1 f: their difference is the first-order
    # image of their mismatches, dx = J^-1 (f32 - f64), checked on the case
    # that differs most with the oracle's Jacobian.
    d = np.maximum(np.abs(r32["va"] - r64["va"]), np.abs(r32["vm"] - r64["vm"]))
    d[~conv] = 0
    k = int(np.argmax(d.max(1)))
    assert d[k].max() <= 1e-7
    Yk = grid_ybus(g.without_branch(int(outs[k])))
    f64, _ = oracle.mismatch(Yk, r64["va"][k], r64["vm"][k], g.p_spec, g.q_spec, g.bus_type)
    f32, _ = oracle.mismatch(Yk, r32["va"][k], r32["vm"][k], g.p_spec, g.q_spec, g.bus_type)
    J = oracle.jacobian_f(Yk, r64["va"][k], r64["vm"][k], g.bus_type)
    import scipy.sparse.linalg as spla
    dx = spla.spsolve(J, f32 - f64)
    pvpq, pq = oracle.learnable_sets(g.bus_type)
    act = np.concatenate([r32["va"][k][pvpq] - r64["va"][k][pvpq], r32["vm"][k][pq] - r64["vm"][k][pq]])
    assert np.abs(act - dx).max() <= 1e-3 * np.abs(dx).max() + 1e-13
    for k in np.random.default_rng(3).choice(np.flatnonzero(conv), 4, replace=False):
        Yk = grid_ybus(g.without_branch(int(outs[k])))
        f, _ = oracle.mismatch(Yk, r32["va"][k], r32["vm"][k], g.p_spec, g.q_spec, g.bus_type)
        assert abs(np.abs(f).max() - r32["max_mismatch"][k]) <= 1e-13


def test_per_case_injections_and_warm_start_from_dpf():
    """Per-case P/Q (load levels 0.9..1.1) on the 30-bus grid; the hybrid of
    Sec. 6: Alg. 1 for 300 iterations, then Newton from its state, which
    needs fewer Newton steps than the flat start and lands on the same
    solution as the oracle."""
    g = gridgen.config_grid("c1_30bus_fp64")
    Y = grid_ybus(g)
    K = 40
    sc = np.linspace(0.9, 1.1, K)[:, None]
    P, Q = g.p_spec[None, :] * sc, g.q_spec[None, :] * sc
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, K)
    flat = _nr(y, nr, K, p_spec=_t(P), q_spec=_t(Q))
    ws = dpf.dpf_workspace_create(y, K)
    st = dict(va=torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV),
              vm=torch.ones((K, g.n_bus), dtype=torch.float64, device=DEV),
              iters=torch.empty(K, dtype=torch.int32, device=DEV),
              status=torch.empty(K, dtype=torch.int32, device=DEV),
              max_mismatch=torch.empty(K, dtype=torch.float64, device=DEV))
    dpf.dpf_solve_batch(y, ws, dpf.SolveOpts(precision=dpf.FP64, max_iter=300, tol=1e-12), n_case=K,
                        p_spec=_t(P), q_spec=_t(Q), **st)
    torch.cuda.synchronize()
    warm = _nr(y, nr, K, flat=False, va=st["va"].cpu().numpy(), vm=st["vm"].cpu().numpy(),
               p_spec=_t(P), q_spec=_t(Q))
    for r in (flat, warm):
        assert (r["status"] == dpf.CASE_CONVERGED).all()
    assert (warm["iters"] <= flat["iters"]).all() and warm["iters"].sum() < flat["iters"].sum()
    for k in (0, K // 2, K - 1):
        ref = oracle.nr_solve(Y, P[k], Q[k], g.bus_type, g.vm_set, tol=TOL)
        assert flat["iters"][k] == ref["iters"]
        for r in (flat, warm):
            assert np.abs(r["va"][k] - ref["va"]).max() <= 1e-9
            assert np.abs(r["vm"][k] - ref["vm"]).max() <= 1e-9


def test_edge_cases():
    g = gridgen.config_grid("c3_n1_2kbus")
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, 4)
    # max_iter = 0: the start comes back, with its mismatch
    r = _nr(y, nr, 2, max_iter=0)
    assert (r["status"] == dpf.CASE_MAX_ITER).all() and (r["iters"] == 0).all()
    Y = grid_ybus(g)
    fva, fvm = oracle.flat_start(g.bus_type, g.vm_set, g.va_slack)
    np.testing.assert_array_equal(r["va"][0], fva)
    np.testing.assert_array_equal(r["vm"][0], fvm)
    f, _ = oracle.mismatch(Y, fva, fvm, g.p_spec, g.q_spec, g.bus_type)
    assert abs(np.abs(f).max() - r["max_mismatch"][0]) <= 1e-12 * np.abs(f).max()
    # an outage of a bridge islands the grid; an index out of range; too many cases
    bridge = int(np.flatnonzero(dpf.dpf_ybus_bridges(y))[0])
    with pytest.raises(dpf.DPFError):
        _nr(y, nr, 2, outage=torch.tensor([bridge, -1], dtype=torch.int32, device=DEV))
    with pytest.raises(dpf.DPFError):
        _nr(y, nr, 2, outage=torch.tensor([g.n_branch, -1], dtype=torch.int32, device=DEV))
    with pytest.raises(dpf.DPFError):
        _nr(y, nr, 5)
    # a load far beyond the grid's limit: no solution, reported, no exception
    r = _nr(y, nr, 1, p_spec=_t(8 * g.p_spec[None, :]), q_spec=_t(8 * g.q_spec[None, :]))
    assert r["status"][0] != dpf.CASE_CONVERGED


def test_solve_repeats_bit_for_bit():
    g = gridgen.config_grid("c3_n1_2kbus")
    outs = gridgen.n1_outages(g)[:96].astype(np.int32)
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, outs.size)
    a = _nr(y, nr, outs.size, outage=_t(outs, torch.int32))
    b = _nr(y, nr, outs.size, outage=_t(outs, torch.int32))
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])


@pytest.mark.parametrize("grid", ["c3_n1_2kbus", "c1_30bus_fp64"])
def test_shared_and_global_memory_forms_agree_bit_for_bit(grid):
    """Where one case's factor fits in shared memory (FP32 on the 2,000-bus
    grid; both precisions on the 30-bus grid) the default takes the
    shared-memory form; lanes > 0 forces the global-memory form.  Each
    target's arithmetic is the same in both (same update order), so the
    results agree to the bit."""
    g = gridgen.config_grid(grid)
    outs = gridgen.n1_outages(g)[:40].astype(np.int32)
    K = outs.size
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, K)
    for prec in (dpf.FP32, dpf.FP64):
        a = _nr(y, nr, K, precision=prec, outage=_t(outs, torch.int32))
        b = _nr(y, nr, K, precision=prec, outage=_t(outs, torch.int32), lanes=4)
        for key in a:
            np.testing.assert_array_equal(a[key], b[key])


def test_single_case_on_the_10k_bus_grid():
    """One case of the 10,000-bus grid: too large a factor for shared
    memory, so the global-memory form runs with one case per CTA (256
    slots walking the tree); against the oracle's NR."""
    g = gridgen.config_grid("c2_10kbus")
    Y = grid_ybus(g)
    ref = oracle.nr_solve(Y, g.p_spec, g.q_spec, g.bus_type, g.vm_set, tol=TOL)
    assert ref["converged"]
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, 1)
    r = _nr(y, nr, 1)
    assert r["status"][0] == dpf.CASE_CONVERGED and r["iters"][0] == ref["iters"]
    assert np.abs(r["va"][0] - ref["va"]).max() <= 1e-9
    assert np.abs(r["vm"][0] - ref["vm"]).max() <= 1e-9


def test_fallback_keeps_the_start_where_newton_fails():
    """fallback (warm start): a case Newton cannot solve (8x load) comes back
    as the start that was passed in, with the start's FP64 mismatch; the
    other cases come back as without fallback."""
    g = gridgen.config_grid("c3_n1_2kbus")
    Y = grid_ybus(g)
    K = 3
    sc = np.array([1.0, 8.0, 1.02])[:, None]
    P, Q = g.p_spec[None, :] * sc, g.q_spec[None, :] * sc
    fva, fvm = oracle.flat_start(g.bus_type, g.vm_set, g.va_slack)
    rng = np.random.default_rng(4)
    va0 = np.tile(fva, (K, 1)) + 0.01 * rng.standard_normal((K, g.n_bus)) * (g.bus_type != dpf.SLACK)
    vm0 = np.tile(fvm, (K, 1))
    y = dpf.dpf_build_ybus(g)
    nr = dpf.dpf_nr_create(y, K)
    plain = _nr(y, nr, K, flat=False, va=va0, vm=vm0, p_spec=_t(P), q_spec=_t(Q))
    fb = _nr(y, nr, K, flat=False, va=va0, vm=vm0, p_spec=_t(P), q_spec=_t(Q), fallback=True)
    assert plain["status"][1] != dpf.CASE_CONVERGED and fb["status"][1] == plain["status"][1]
    np.testing.assert_array_equal(fb["va"][1], va0[1])
    np.testing.assert_array_equal(fb["vm"][1], vm0[1])
    f, _ = oracle.mismatch(Y, va0[1], vm0[1], P[1], Q[1], g.bus_type)
    assert abs(np.abs(f).max() - fb["max_mismatch"][1]) <= 1e-12 * np.abs(f).max()
    for k in (0, 2):
        assert fb["status"][k] == dpf.CASE_CONVERGED
        for key in fb:
            np.testing.assert_array_equal(fb[key][k], plain[key][k])


def test_block_diagonal_batch_of_grids():
    """Three grids in one Y_bus (one slack per island): Newton on the whole
    batch against the oracle's NR on the same block-diagonal system, with
    per-case loads (two operating points)."""
    grids = [gridgen.make_grid(n, 100 + i, n_branch=int(1.35 * n), n_pv=max(1, n // 8), load_scale=0.1)
             for i, n in enumerate((40, 120, 75))]
    cat = gridgen.concat_grids(grids)
    Y = grid_ybus(cat)
    sc = np.array([1.0, 0.9])[:, None]
    P, Q = cat.p_spec[None, :] * sc, cat.q_spec[None, :] * sc
    y = dpf.dpf_build_ybus(cat)
    nr = dpf.dpf_nr_create(y, 2)
    r = _nr(y, nr, 2, p_spec=_t(P), q_spec=_t(Q))
    for k in range(2):
        ref = oracle.nr_solve(Y, P[k], Q[k], cat.bus_type, cat.vm_set, tol=TOL)
        assert ref["converged"] and r["status"][k] == dpf.CASE_CONVERGED
        assert r["iters"][k] == ref["iters"]
        assert np.abs(r["va"][k] - ref["va"]).max() <= 1e-9
        assert np.abs(r["vm"][k] - ref["vm"]).max() <= 1e-9
