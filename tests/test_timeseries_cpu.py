"""Host-side checks of the time-series driver and of its workload: option
validation and checkpoint fingerprints (no device), and that the 10,000-bus
time-series load model has a power-flow solution at its heaviest hour (the
oracle's Newton-Raphson, Alg. 2)."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.ybus import grid_ybus

torch = pytest.importorskip("torch")

from paper_2603_28203_gb300 import _abi  # noqa: E402
from paper_2603_28203_gb300.timeseries import TABLE3_T1, _fingerprint, solve_time_series  # noqa: E402


def test_newton_from_is_validated_before_any_device_work():
    P = np.zeros((2, 3))
    with pytest.raises(ValueError, match="newton_from"):
        solve_time_series(None, None, P, P, window=2, newton_from="newton")
    with pytest.raises(ValueError, match="warm_from"):
        solve_time_series(None, None, P, P, window=2, warm_from="previous")


def test_fingerprint_tells_the_first_window_starts_apart():
    p = torch.arange(6, dtype=torch.float64).reshape(2, 3)
    base = (p, p, _abi.FP32R, 1e-6, 50, dict(TABLE3_T1))
    marker = object()  # any NewtonSolver stand-in: only its presence counts
    plain = _fingerprint(*base, None, 0, 96)
    via_dpf = _fingerprint(*base, marker, 0, 96, "dpf")
    via_flat = _fingerprint(*base, marker, 0, 96, "flat")
    assert len({plain, via_dpf, via_flat}) == 3
    # later windows start from the previous window whatever solved the first,
    # but the two warm-start readings differ
    assert _fingerprint(*base, marker, 96, 96, "dpf") == _fingerprint(*base, marker, 96, 96, "flat")
    assert _fingerprint(*base, None, 96, 96, "dpf", "same_hour") != _fingerprint(*base, None, 96, 96, "dpf", "last")
    assert _fingerprint(*base, None, 0, 96, "dpf", "same_hour") == _fingerprint(*base, None, 0, 96, "dpf", "last")


def test_time_series_grid_solves_at_its_peak_hour():
    """Winter noon (t = 12: daily x seasonal factor 1.25 x 1.15, plus the
    per-bus noise) is the heaviest hour of the load model; Newton-Raphson
    from the flat start reaches 1e-10 p.u. there in a handful of steps with
    |V| above 0.9."""
    g = gridgen.config_grid("c4_timeseries_10kbus")
    P, Q = gridgen.time_series(g, 1, seed=4, t0=12)
    r = oracle.nr_solve(grid_ybus(g), P[0], Q[0], g.bus_type, g.vm_set, tol=1e-10, max_iter=12)
    assert r["converged"] and r["iters"] <= 10
    assert r["vm"].min() > 0.9
