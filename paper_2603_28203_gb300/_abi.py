"""ctypes declarations mirroring include/dpf.h."""
from __future__ import annotations

import ctypes as C

DPF_OK = 0
DPF_E_INVALID, DPF_E_ISLANDED, DPF_E_CUDA, DPF_E_OOM, DPF_E_UNSUPPORTED, DPF_E_STATE = -1, -2, -3, -4, -5, -6
CASE_CONVERGED, CASE_MAX_ITER, CASE_DIVERGED = 0, 1, 2
PQ, PV, SLACK = 0, 1, 2
FP32, FP64, MIXED, FP32R = 0, 1, 2, 3
SCHED_CONST, SCHED_PLATEAU, SCHED_STEP = 0, 1, 2
OPT_ADAM, OPT_SGD, OPT_RMSPROP = 0, 1, 2
NOALLOC_MAX_ELEMS = 1 << 18

p_i32 = C.POINTER(C.c_int32)
p_u8 = C.POINTER(C.c_uint8)
p_f64 = C.POINTER(C.c_double)


class DpfGrid(C.Structure):
    _fields_ = [
        ("n_bus", C.c_int32), ("n_branch", C.c_int32),
        ("bus_type", C.c_void_p), ("p_spec", C.c_void_p), ("q_spec", C.c_void_p),
        ("vm_set", C.c_void_p), ("va_slack", C.c_double),
        ("f_bus", C.c_void_p), ("t_bus", C.c_void_p),
        ("r", C.c_void_p), ("x", C.c_void_p), ("b_ch", C.c_void_p), ("tap", C.c_void_p),
        ("shift", C.c_void_p),
    ]


class DpfBatch(C.Structure):
    _fields_ = [
        ("n_case", C.c_int32), ("host_io", C.c_int32),
        ("p_spec", C.c_void_p), ("q_spec", C.c_void_p), ("vm_set", C.c_void_p),
        ("outage", C.c_void_p), ("va", C.c_void_p), ("vm", C.c_void_p),
        ("iters", C.c_void_p), ("status", C.c_void_p), ("max_mismatch", C.c_void_p),
        ("loss", C.c_void_p), ("va_start", C.c_void_p), ("vm_start", C.c_void_p),
    ]


class DpfSolveOpts(C.Structure):
    _fields_ = [
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("optimizer", C.c_int32), ("momentum", C.c_double), ("alpha", C.c_double),
        ("sched", C.c_int32),
        ("factor", C.c_double), ("threshold", C.c_double), ("min_lr", C.c_double),
        ("patience", C.c_int32), ("cooldown", C.c_int32),
        ("step_size", C.c_int32), ("gamma", C.c_double),
        ("max_iter", C.c_int32), ("check_every", C.c_int32), ("tol", C.c_double), ("gate", C.c_double),
        ("flat_start", C.c_int32), ("precision", C.c_int32),
        ("lanes", C.c_int32), ("warps", C.c_int32), ("row_blocks", C.c_int32),
        ("use_graph", C.c_int32), ("pair_cases", C.c_int32), ("pdl", C.c_int32), ("stage_v", C.c_int32),
        ("plain", C.c_int32),
        ("dc_start", C.c_int32), ("stage_y", C.c_int32),
        ("dc_tol", C.c_double), ("dc_max_iter", C.c_int32), ("refresh_every", C.c_int32),
    ]


class DpfNrOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("flat_start", C.c_int32), ("lanes", C.c_int32), ("fallback", C.c_int32)]


VP = C.c_void_p
I32 = C.c_int32

# name -> (restype, argtypes)
SIGNATURES = {
    "dpf_build_ybus_host": (C.c_int, [C.POINTER(DpfGrid), C.POINTER(VP)]),
    "dpf_ybus_upload": (C.c_int, [VP, VP]),
    "dpf_build_ybus": (C.c_int, [C.POINTER(DpfGrid), VP, C.POINTER(VP)]),
    "dpf_ybus_free": (C.c_int, [VP]),
    "dpf_ybus_info": (C.c_int, [VP, p_i32, p_i32, p_i32]),
    "dpf_ybus_export": (C.c_int, [VP, VP, VP, VP, VP]),
    "dpf_ybus_bridges": (C.c_int, [VP, VP]),
    "dpf_default_opts": (None, [C.POINTER(DpfSolveOpts)]),
    "dpf_workspace_create": (C.c_int, [VP, I32, C.POINTER(VP)]),
    "dpf_workspace_free": (C.c_int, [VP]),
    "dpf_solve_batch": (C.c_int, [VP, VP, C.POINTER(DpfBatch), C.POINTER(DpfSolveOpts), VP]),
    "dpf_solve_begin": (C.c_int, [VP, VP, C.POINTER(DpfBatch), C.POINTER(DpfSolveOpts), VP]),
    "dpf_solve_iterate": (C.c_int, [VP, I32, VP]),
    "dpf_solve_end": (C.c_int, [VP, C.POINTER(DpfBatch), VP]),
    "dpf_active_count": (C.c_int, [VP, p_i32, VP]),
    "dpf_autotune": (C.c_int, [VP, VP, C.POINTER(DpfBatch), C.POINTER(DpfSolveOpts), I32, VP]),
    "dpf_iterations_done": (C.c_int, [VP, p_i32]),
    "dpf_power": (C.c_int, [VP, VP, I32, VP, VP, VP, I32, VP, VP, VP]),
    "dpf_loss_backward": (C.c_int, [VP, VP, I32, VP, VP, VP, VP, VP, VP, VP, I32,
                                    VP, VP, VP, VP, VP, VP, VP, VP, VP]),
    "dpf_power_noalloc": (C.c_int, [VP, I32, VP, VP, VP, VP, VP]),
    "dpf_paramid_begin": (C.c_int, [VP, VP, I32, VP, VP, VP, VP, I32, VP]),
    "dpf_dc_solve": (C.c_int, [VP, VP, I32, VP, VP, C.c_double, I32, VP, VP, VP, VP]),
    "dpf_nr_create": (C.c_int, [VP, I32, C.POINTER(VP)]),
    "dpf_nr_free": (C.c_int, [VP]),
    "dpf_nr_default_opts": (None, [C.POINTER(DpfNrOpts)]),
    "dpf_nr_solve": (C.c_int, [VP, C.POINTER(DpfBatch), C.POINTER(DpfNrOpts), VP]),
    "dpf_nr_stats": (C.c_int, [VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64), p_i32, C.POINTER(C.c_int64)]),
    "dpf_nr_analyze": (C.c_int, [VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64), p_i32]),
    "dpf_nr_pattern": (C.c_int, [VP, VP, VP, VP, VP]),
    "dpf_paramid_step": (C.c_int, [VP, VP, VP, VP, VP, VP, VP, VP, VP]),
    "dpf_profile_enable": (C.c_int, [VP, I32]),
    "dpf_kernel_times": (C.c_int, [VP, p_f64, p_f64, p_i32, p_i32, VP]),
    "dpf_kernel_launches": (C.c_int, [VP, C.POINTER(C.c_int64)]),
    "dpf_read_bandwidth": (C.c_int, [VP, C.c_int64, C.c_int32, C.POINTER(C.c_double), VP]),
    "dpf_grid_barrier_cost": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), VP]),
    "dpf_adam_update": (C.c_int, [I32, VP, VP, VP, VP, VP, I32, C.c_double, C.c_double, C.c_double, C.c_double,
                                  VP]),
    "dpf_last_error": (C.c_char_p, []),
    "dpf_status_str": (C.c_char_p, [C.c_int]),
}
