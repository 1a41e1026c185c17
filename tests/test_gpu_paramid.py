"""Parameter identification on an uneven block-diagonal batch (reduced size).

Three synthetic grids of different sizes form one block-diagonal system (one
slack per island, Sec. 4.2); 8 operating points per grid come from the FP64
oracle's Newton-Raphson at the true branch parameters; branch r and x are
perturbed by U(-10%, +10%).  Adam on the series admittances (g, b) with the
branch adjoint:
  * FP64: step for step equal to the same loop written with the oracle's
    parameter gradient and Adam (1e-9 relative);
  * FP32: the loss falls and the parameter error shrinks.
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
from paper_2603_28203_gb300.paramid import identify_branches  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2603_28203_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    dpf.lib()


@pytest.fixture(scope="module")
def case():
    grids = [gridgen.make_grid(n, 100 + i, load_scale=0.3) for i, n in enumerate([40, 80, 120])]
    cat = gridgen.concat_grids(grids)
    Y = grid_ybus(cat)
    K = 8
    P, Q = gridgen.time_series(cat, K, seed=5)
    va, vm = [], []
    for k in range(K):
        r = oracle.nr_solve(Y, P[k], Q[k], cat.bus_type, cat.vm_set)
        assert r["converged"]
        va.append(r["va"])
        vm.append(r["vm"])
    pert = gridgen.perturb_branches(cat, 5)
    return cat, np.array(va), np.array(vm), P, Q, 1 / (cat.r + 1j * cat.x), 1 / (pert.r + 1j * pert.x)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def test_paramid_fp64_matches_oracle_loop(case):
    cat, va, vm, P, Q, ys_true, ys0 = case
    y = dpf.dpf_build_ybus(cat)
    ws = dpf.dpf_workspace_create(y, va.shape[0])
    iters, lr = 30, 3e-3
    g, b, _ = identify_branches(y, ws, _t(va), _t(vm), _t(P), _t(Q), _t(ys0.real), _t(ys0.imag), iters, lr,
                                precision=dpf.FP64)
    # the same loop on the oracle
    og, ob = ys0.real.copy(), ys0.imag.copy()
    sg, sb = np.abs(og), np.abs(ob)
    ag, ab = oracle.Adam(og.size, lr, (0.9, 0.999)), oracle.Adam(ob.size, lr, (0.9, 0.999))
    for _ in range(iters):
        z = 1 / (og + 1j * ob)
        Yp = oracle.build_ybus(cat.n_bus, cat.f_bus, cat.t_bus, z.real, z.imag, cat.b_ch, cat.tap)
        dg = np.zeros_like(og)
        db = np.zeros_like(ob)
        for k in range(va.shape[0]):
            out = oracle.param_grad(Yp, va[k], vm[k], P[k], Q[k], cat.bus_type, cat.f_bus, cat.t_bus, cat.tap)
            dg += out[0]
            db += out[1]
        og = ag.step(og, dg, sg)
        ob = ab.step(ob, db, sb)
    assert np.abs(g.cpu().numpy() - og).max() <= 1e-9 * np.abs(og).max()
    assert np.abs(b.cpu().numpy() - ob).max() <= 1e-9 * np.abs(ob).max()


def test_paramid_fp32_reduces_error(case):
    cat, va, vm, P, Q, ys_true, ys0 = case
    y = dpf.dpf_build_ybus(cat)
    ws = dpf.dpf_workspace_create(y, va.shape[0])
    g, b, hist = identify_branches(y, ws, _t(va), _t(vm), _t(P), _t(Q), _t(ys0.real), _t(ys0.imag), 400, 3e-3,
                                   precision=dpf.FP32, record_every=100)
    e0 = np.median(np.abs(ys0.imag - ys_true.imag) / np.abs(ys_true.imag))
    e1 = np.median(np.abs(b.cpu().numpy() - ys_true.imag) / np.abs(ys_true.imag))
    assert hist[-1][1] < 0.05 * hist[0][1] or hist[-1][1] < 1e-6
    assert e1 < 0.5 * e0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paramid_step_matches_loss_backward(case, precision):
    """The staged step gives dpf_loss_backward's branch gradients and loss for the
    same inputs, on every step (the loss pass does not disturb the staged points)."""
    cat, va, vm, P, Q, ys_true, ys0 = case
    prec = dict(fp64=dpf.FP64, fp32=dpf.FP32)[precision]
    y = dpf.dpf_build_ybus(cat)
    ws = dpf.dpf_workspace_create(y, va.shape[0])
    g, b = _t(ys0.real), _t(ys0.imag)
    ref = dpf.dpf_loss_backward(y, ws, _t(va), _t(vm), _t(P), _t(Q), g_series=g, b_series=b, precision=prec,
                                want=("loss", "d_g", "d_b"))
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    dpf.dpf_paramid_begin(y, ws, _t(va), _t(vm), _t(P), _t(Q), precision=prec)
    for _ in range(3):
        out = dpf.dpf_paramid_step(y, ws, g, b, want=("d_g", "d_b", "loss"))
        out = {k: v.cpu().numpy() for k, v in out.items()}
        for k in ("d_g", "d_b", "loss"):
            assert np.allclose(out[k], ref[k], rtol=1e-12, atol=1e-14 * np.abs(ref[k]).max()), k


def test_paramid_step_needs_staged_points(case):
    cat, va, vm, P, Q, ys_true, ys0 = case
    y = dpf.dpf_build_ybus(cat)
    ws = dpf.dpf_workspace_create(y, va.shape[0])
    g, b = _t(ys0.real), _t(ys0.imag)
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_paramid_step(y, ws, g, b)
    assert e.value.code == -6  # DPF_E_STATE
    dpf.dpf_paramid_begin(y, ws, _t(va), _t(vm), _t(P), _t(Q))
    dpf.dpf_paramid_step(y, ws, g, b)
    dpf.dpf_power(y, ws, _t(va), _t(vm))  # another use of the workspace drops the staged points
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_paramid_step(y, ws, g, b)
    assert e.value.code == -6
