"""CPU FP64 oracle for Differentiable Power-Flow (DPF).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline legs of `bench.py` may import
it.  It shares no code with the CUDA library (`paper_2603_28203_gb300`), and
the library never imports it.

Every routine works in float64 with numpy/scipy and follows the paper's
statement of the problem:

  ybus.build_ybus      branch pi-model -> Y_bus (Sec. 2.1, Eq. powerbalance,
                       whose footnote defers to the MATPOWER branch model)
  power.*              S_calc = V (Y V)^*, mismatch f, MSE loss
                       (Eq. powerbalance, Eq. pf_equation_full, Alg. 1)
  jacobian.*           dS/d|V|, dS/dtheta and J_f (Alg. 2)
  gradient.*           dL/dx = (2/m) J_f^T f (Sec. 4.1 with the MSE of Alg. 1),
                       parameter gradients dL/d(g, b, b_ch), dL/dP, dL/dQ
  optim.*              Adam (Kingma & Ba), ReduceLROnPlateau, StepLR
                       (Sec. 5.3, Tables 2-3)
  dpf.dpf_solve        the DPF loop (Alg. 1)
  nr.nr_solve          Newton-Raphson (Alg. 2), the ground-truth solver
  dc.dc_solve          DC approximation B theta = P (Sec. 2 comparison model,
                       Alg. 2's optional initialisation)
  dc.dc_outage_shift   DC angle change of an outage, B' dtheta = (B - B') theta
                       (a start for warm-started N-1 cases)

Pins (tests/test_oracle_*.py) tie each of these to something other than the
oracle itself: closed forms (two-bus line, Y_bus hand values), the
power-balance invariant, central finite differences, scipy's fsolve and
torch.optim on the same gradient sequence.  Iteration counts of the DPF loop
have no published value to compare against: parity unpinned.
"""
from .ybus import build_ybus, branch_blocks
from .power import s_calc, mismatch, loss, learnable_sets
from .jacobian import dS_dVm_dVa, jacobian_f
from .gradient import loss_grad, param_grad
from .optim import SGD, Adam, ReduceLROnPlateau, RMSprop, StepLR
from .dpf import DPFOptions, dpf_solve, flat_start
from .nr import nr_solve
from .dc import dc_branch_flows, dc_matrix, dc_outage_shift, dc_solve, dc_susceptance

__all__ = [
    "build_ybus", "branch_blocks", "s_calc", "mismatch", "loss", "learnable_sets",
    "dS_dVm_dVa", "jacobian_f", "loss_grad", "param_grad", "Adam", "SGD", "RMSprop",
    "ReduceLROnPlateau", "StepLR", "DPFOptions", "dpf_solve", "flat_start",
    "nr_solve", "dc_solve", "dc_matrix", "dc_susceptance", "dc_branch_flows", "dc_outage_shift",
]
