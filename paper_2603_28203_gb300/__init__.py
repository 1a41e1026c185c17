"""GB300-native Differentiable Power-Flow (DPF) hot path.

The CUDA library (csrc/, C ABI in include/dpf.h) runs batched DPF iterations
(Alg. 1): complex CSR SpMV I = Y V with the mismatch and loss fused in its
epilogue, the hand-written adjoint (Y applied to the mismatch-weighted
voltages), a fused Adam step with per-case schedulers, N-1 outages as a
per-case correction of one shared Y_bus, and an FP64 convergence test.
`dpf` is the ctypes binding (same names as the C functions), `autograd` the
torch.autograd.Function over the adjoint.
"""
from . import _abi
from ._abi import (CASE_CONVERGED, CASE_DIVERGED, CASE_MAX_ITER, FP32, FP32R, FP64, MIXED, OPT_ADAM, OPT_RMSPROP, OPT_SGD,
                   PQ, PV, SCHED_CONST,
                   SCHED_PLATEAU, SCHED_STEP, SLACK)
from .dpf import (DPFError, SolveOpts, Workspace, Ybus, dpf_active_count, dpf_adam_update, dpf_autotune, dpf_build_ybus,
                  dpf_build_ybus_host, dpf_default_opts, dpf_iterations_done, dpf_kernel_launches, dpf_kernel_times,
                  dpf_last_error, dpf_profile_enable, dpf_read_bandwidth, dpf_grid_barrier_cost,
                  dpf_dc_solve, dpf_loss_backward, NewtonSolver, dpf_nr_analyze, dpf_nr_create, dpf_nr_pattern,
                  dpf_nr_solve, dpf_paramid_begin, dpf_paramid_step, dpf_power,
                  dpf_power_noalloc,
                  dpf_solve_batch, dpf_solve_begin, dpf_solve_end,
                  dpf_solve_iterate, dpf_status_str, dpf_workspace_create, dpf_ybus_bridges,
                  dpf_ybus_export, dpf_ybus_upload, lib)
