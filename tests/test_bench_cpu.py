"""CPU checks of bench.py's accounting: the workload it times and the
algorithmic byte counts its roofline divides by (the figures the design
notes quote for the N-1 batch)."""
import numpy as np

import bench


def test_n1_workload_and_algorithmic_bytes():
    g, outages = bench._workload()
    n_pv = int((g.bus_type == 1).sum())
    n_pq = int((g.bus_type == 0).sum())
    nnz = g.n_bus + 2 * g.n_branch
    assert (g.n_bus, n_pv, n_pq, nnz, outages.size) == (2000, 300, 1699, 7400, 2379)
    fwd, adj = bench.algorithmic_bytes(g.n_bus, n_pv, n_pq, nnz, outages.size)
    # per case: forward 16 N + 4 n_pv, adjoint 8 N + 60 n_pv + 80 n_pq; Y and the shared P/Q once per pass
    shared = 16 * nnz + 4 * (g.n_bus + 1) + g.n_bus + 8 * g.n_bus
    assert fwd == outages.size * (16 * g.n_bus + 4 * n_pv) + shared
    assert adj == outages.size * (8 * g.n_bus + 60 * n_pv + 80 * n_pq) + shared
    assert round(fwd / 1e6, 1) == 79.1 and round(adj / 1e6, 1) == 404.4


def test_dc_and_newton_byte_models_scale_with_the_cases():
    b1 = bench.dc_bytes_per_iteration(2000, 7400, 1)
    b2 = bench.dc_bytes_per_iteration(2000, 7400, 2)
    assert b2 - b1 == 2000 * 96                       # 96 B per element and CG iteration
    n1 = bench.nr_bytes_per_step(2000, 10594, 10851, 1)
    n2 = bench.nr_bytes_per_step(2000, 10594, 10851, 2)
    assert n2["fp64"] == 2 * n1["fp64"] and n2["fp32"] == 2 * n1["fp32"]
    assert n1["fp32"] < n1["fp64"]
    assert np.isclose(bench.dc_flops_per_iteration(2000, 7400, 1, 1), 2 * 7400 + 1999 * 15)


def test_refined_byte_model_and_presets():
    g, outages = bench._workload()
    n_pv = int((g.bus_type == 1).sum())
    n_pq = int((g.bus_type == 0).sum())
    nnz = g.n_bus + 2 * g.n_branch
    K = outages.size
    f32, a32 = bench.algorithmic_bytes(g.n_bus, n_pv, n_pq, nnz, K)
    f, a = bench.algorithmic_bytes(g.n_bus, n_pv, n_pq, nnz, K, refined=True)
    # refined FP32: the forward pass reads V_ref (8) and (I_ref, f_ref) (16) per element instead of the
    # shared P/Q; the adjoint moves the same bytes (dV in V's place)
    assert f - f32 == K * 24 * g.n_bus - 8 * g.n_bus
    assert a == a32
    # the warm-started N-1 settings are solve options the binding and the oracle both accept
    import dataclasses
    from paper_2603_28203_gb300.dpf import SolveOpts
    from paper_2603_28203_gb300.presets import N1_DC, N1_DC_START, N1_WARM, TABLE2
    names = {fl.name for fl in dataclasses.fields(SolveOpts)}
    assert set(N1_WARM) <= names and set(TABLE2) <= names and set(N1_DC) <= names and set(N1_DC_START) <= names
    for start, s in (("base", N1_WARM), ("dc", N1_DC)):
        o = bench._oracle_dpf_options(3000, start)
        assert (o.lr, o.beta1, o.beta2, o.eps, o.sched, o.threshold, o.max_iter, o.check_every) == \
            (s["lr"], s["beta1"], s["beta2"], s["eps"], "plateau", s["threshold"], 3000,
             bench.n1_settings(start)[1]["check_every"])
        assert bench.n1_settings(start)[0] is s
    assert bench.n1_settings("dc")[1]["dc_start"] == 1 and "dc_start" not in bench.n1_settings("base")[1]
    for start in ("dc", "base"):
        assert set(bench.n1_settings(start)[1]) <= names


def test_oracle_legs_run_a_shifted_case():
    """The oracle legs (cpu_baseline, --impl reference) run one N-1 case: the
    oracle's DC outage shift of the base case's angles, then Alg. 1 with the
    benchmark's settings; a short budget here.  The shifted start lowers the
    starting mismatch, as on the GPU."""
    import oracle
    from oracle.ybus import grid_ybus
    g, outages = bench._workload()
    ell = int(outages[100])
    it, dt, st = bench._oracle_case((ell, 20, "dc"))
    assert it == 20 and st == 1 and dt > 0.0  # budget spent (not converged in 20 iterations)
    _, base = bench._oracle_base()
    Yk = grid_ybus(g.without_branch(ell))
    f0, _ = oracle.mismatch(Yk, base["va"], base["vm"], g.p_spec, g.q_spec, g.bus_type)
    d = oracle.dc_outage_shift(g.n_bus, g.f_bus, g.t_bus, g.x, g.tap, g.bus_type, base["va"], ell)
    f1, _ = oracle.mismatch(Yk, base["va"] + d, base["vm"], g.p_spec, g.q_spec, g.bus_type)
    assert np.abs(f1).max() < np.abs(f0).max()
