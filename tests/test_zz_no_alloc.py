"""The allocation-free forward evaluation (dpf_power_noalloc).

It serves callers that cannot allocate device memory (an application that
owns the device memory budget, or a loop that cannot afford cudaMalloc's
synchronisation).  Its output must equal the workspace-based dpf_power
(FP64) within the FP64 parity tolerance, on two calls in a row that share the
library's fixed scratch array.  This file is collected last on purpose.
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


def _state(K, N, seed):
    rng = np.random.default_rng(seed)
    va = torch.tensor(0.2 * rng.standard_normal((K, N)), dtype=torch.float64, device=DEV)
    vm = torch.tensor(1.0 + 0.05 * rng.standard_normal((K, N)), dtype=torch.float64, device=DEV)
    return va, vm


@pytest.mark.parametrize("name,K", [("c1_30bus_fp64", 7), ("c3_n1_2kbus", 100)])
def test_noalloc_matches_dpf_power_twice(name, K):
    g = gridgen.config_grid(name)
    y = dpf.dpf_build_ybus(g)
    ws = dpf.dpf_workspace_create(y, K)
    for call in range(2):  # the second call reuses the scratch left by the first
        va, vm = _state(K, g.n_bus, 10 * call + K)
        p_ref, q_ref = dpf.dpf_power(y, ws, va, vm, precision=dpf.FP64)
        p = torch.full_like(va, float("nan"))
        q = torch.full_like(va, float("nan"))
        dpf.dpf_power_noalloc(y, va, vm, p, q)
        torch.cuda.synchronize()
        scale = max(p_ref.abs().max().item(), q_ref.abs().max().item())
        assert (p - p_ref).abs().max().item() <= 1e-10 * scale
        assert (q - q_ref).abs().max().item() <= 1e-10 * scale
        # and one case straight against the oracle's S = V (Y V)^*
        k = K - 1
        S = oracle.s_calc(grid_ybus(g), vm[k].cpu().numpy() * np.exp(1j * va[k].cpu().numpy()))
        assert np.abs(p[k].cpu().numpy() - S.real).max() <= 1e-10 * scale
        assert np.abs(q[k].cpu().numpy() - S.imag).max() <= 1e-10 * scale


def test_noalloc_rejects_oversized_batch():
    g = gridgen.config_grid("c3_n1_2kbus")
    y = dpf.dpf_build_ybus(g)
    K = dpf._abi.NOALLOC_MAX_ELEMS // g.n_bus + 1
    va = torch.zeros((K, g.n_bus), dtype=torch.float64, device=DEV)
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_power_noalloc(y, va, va, va.clone(), va.clone())
    assert e.value.code == -1 and "scratch" in str(e.value)
    # outputs that do not match the inputs' shape or precision are refused before the call
    small = torch.zeros((2, g.n_bus), dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        dpf.dpf_power_noalloc(y, small, small, torch.zeros((1, g.n_bus), dtype=torch.float64, device=DEV), small.clone())
    with pytest.raises(ValueError):
        dpf.dpf_power_noalloc(y, small, small, small.float(), small.clone())
