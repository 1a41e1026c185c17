"""Python binding of libdpf (include/dpf.h): argument marshalling only.

Every function keeps the C name.  Device arrays are torch CUDA tensors
(float64 / int32, contiguous); their data pointers and the current torch
stream are passed straight to the library, which does all the work in its own
CUDA kernels.  There is no fallback: if libdpf.so is missing or a call fails,
an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import _abi
from .build import LIB

_lib = None


class DPFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdpf error {code}: {msg}")
        self.code = code


def lib():
    """Load libdpf.so (built in-tree by `build.build()`); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libdpf.so not found at {LIB}; build it with paper_2603_28203_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, (res, args) in _abi.SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != _abi.DPF_OK:
        raise DPFError(rc, lib().dpf_last_error().decode())


def _ptr(t):
    """Data pointer of a contiguous tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to libdpf must be contiguous"
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---- grid / Y_bus -----------------------------------------------------------
class Ybus:
    """Owner of a dpf_ybus handle."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep
        n, m, z = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().dpf_ybus_info(handle, C.byref(n), C.byref(m), C.byref(z)))
        self.n_bus, self.n_branch, self.nnz = n.value, m.value, z.value

    def free(self):
        if self.handle:
            lib().dpf_ybus_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _grid_struct(grid):
    arrs = dict(
        bus_type=np.ascontiguousarray(grid.bus_type, np.uint8),
        p_spec=np.ascontiguousarray(grid.p_spec, np.float64),
        q_spec=np.ascontiguousarray(grid.q_spec, np.float64),
        vm_set=np.ascontiguousarray(grid.vm_set, np.float64),
        f_bus=np.ascontiguousarray(grid.f_bus, np.int32),
        t_bus=np.ascontiguousarray(grid.t_bus, np.int32),
        r=np.ascontiguousarray(grid.r, np.float64),
        x=np.ascontiguousarray(grid.x, np.float64),
        b_ch=np.ascontiguousarray(grid.b_ch, np.float64),
        tap=np.ascontiguousarray(grid.tap, np.float64),
    )
    shift = getattr(grid, "shift", None)
    if shift is not None:
        arrs["shift"] = np.ascontiguousarray(shift, np.float64)
    g = _abi.DpfGrid()
    g.n_bus = arrs["bus_type"].size
    g.n_branch = arrs["f_bus"].size
    for k, v in arrs.items():
        setattr(g, k, v.ctypes.data)
    g.va_slack = float(getattr(grid, "va_slack", 0.0))
    return g, arrs


def dpf_build_ybus_host(grid) -> Ybus:
    g, keep = _grid_struct(grid)
    h = C.c_void_p()
    _check(lib().dpf_build_ybus_host(C.byref(g), C.byref(h)))
    return Ybus(h, keep)


def dpf_ybus_upload(y: Ybus, stream=None):
    _check(lib().dpf_ybus_upload(y.handle, _stream(stream)))


def dpf_build_ybus(grid, stream=None) -> Ybus:
    g, keep = _grid_struct(grid)
    h = C.c_void_p()
    _check(lib().dpf_build_ybus(C.byref(g), _stream(stream), C.byref(h)))
    return Ybus(h, keep)


def dpf_ybus_export(y: Ybus):
    """(row_ptr, col, val) of the FP64 CSR in user bus order (numpy)."""
    rp = np.empty(y.n_bus + 1, np.int32)
    col = np.empty(y.nnz, np.int32)
    re = np.empty(y.nnz, np.float64)
    im = np.empty(y.nnz, np.float64)
    _check(lib().dpf_ybus_export(y.handle, rp.ctypes.data, col.ctypes.data, re.ctypes.data, im.ctypes.data))
    return rp, col, re + 1j * im


def dpf_ybus_bridges(y: Ybus) -> np.ndarray:
    out = np.empty(max(y.n_branch, 1), np.uint8)
    _check(lib().dpf_ybus_bridges(y.handle, out.ctypes.data))
    return out[: y.n_branch].astype(bool)


# ---- options / workspace ----------------------------------------------------
@dataclasses.dataclass
class SolveOpts:
    """Mirror of dpf_solve_opts; None keeps the library default (Table 2 etc.)."""
    lr: float | None = None
    optimizer: int | None = None
    momentum: float | None = None
    alpha: float | None = None
    beta1: float | None = None
    beta2: float | None = None
    eps: float | None = None
    sched: int | None = None
    factor: float | None = None
    threshold: float | None = None
    min_lr: float | None = None
    patience: int | None = None
    cooldown: int | None = None
    step_size: int | None = None
    gamma: float | None = None
    max_iter: int | None = None
    check_every: int | None = None
    tol: float | None = None
    gate: float | None = None
    flat_start: int | None = None
    precision: int | None = None
    lanes: int | None = None
    warps: int | None = None
    row_blocks: int | None = None
    use_graph: int | None = None
    pair_cases: int | None = None
    pdl: int | None = None
    stage_v: int | None = None
    plain: int | None = None
    dc_start: int | None = None
    stage_y: int | None = None
    dc_tol: float | None = None
    dc_max_iter: int | None = None
    refresh_every: int | None = None

    def to_c(self) -> _abi.DpfSolveOpts:
        o = _abi.DpfSolveOpts()
        lib().dpf_default_opts(C.byref(o))
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if v is not None:
                setattr(o, f.name, v)
        return o


def dpf_default_opts() -> _abi.DpfSolveOpts:
    o = _abi.DpfSolveOpts()
    lib().dpf_default_opts(C.byref(o))
    return o


class Workspace:
    def __init__(self, y: Ybus, max_case: int):
        self.ybus = y
        h = C.c_void_p()
        _check(lib().dpf_workspace_create(y.handle, int(max_case), C.byref(h)))
        self.handle = h

    def free(self):
        if self.handle:
            lib().dpf_workspace_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dpf_workspace_create(y: Ybus, max_case: int) -> Workspace:
    return Workspace(y, max_case)


# ---- batched solve -----------------------------------------------------------
def _batch_struct(n_case, host_io=False, p_spec=None, q_spec=None, vm_set=None, outage=None, va=None,
                  vm=None, iters=None, status=None, max_mismatch=None, loss=None, va_start=None, vm_start=None):
    b = _abi.DpfBatch()
    b.n_case = int(n_case)
    b.host_io = 1 if host_io else 0
    for name, t in dict(p_spec=p_spec, q_spec=q_spec, vm_set=vm_set, outage=outage, va=va, vm=vm,
                        iters=iters, status=status, max_mismatch=max_mismatch, loss=loss,
                        va_start=va_start, vm_start=vm_start).items():
        setattr(b, name, _ptr(t))
    return b


def _opts(opts):
    if opts is None:
        return dpf_default_opts()
    if isinstance(opts, SolveOpts):
        return opts.to_c()
    return opts


def dpf_solve_batch(y: Ybus, ws: Workspace | None, opts=None, stream=None, **batch):
    """Solve every case; `batch` holds the dpf_batch fields as tensors."""
    b = _batch_struct(**batch)
    o = _opts(opts)
    _check(lib().dpf_solve_batch(y.handle, ws.handle if ws else None, C.byref(b), C.byref(o), _stream(stream)))


def dpf_solve_begin(y: Ybus, ws: Workspace, opts=None, stream=None, **batch):
    b = _batch_struct(**batch)
    o = _opts(opts)
    _check(lib().dpf_solve_begin(y.handle, ws.handle, C.byref(b), C.byref(o), _stream(stream)))


def dpf_autotune(y: Ybus, ws: Workspace, opts=None, iters: int = 25, stream=None, **batch) -> SolveOpts:
    """Launch shape picked by the library's autotuner for this batch (returned as SolveOpts)."""
    b = _batch_struct(**batch)
    o = _opts(opts)
    _check(lib().dpf_autotune(y.handle, ws.handle, C.byref(b), C.byref(o), int(iters), _stream(stream)))
    out = SolveOpts(**{f.name: getattr(opts, f.name) for f in dataclasses.fields(SolveOpts)}) \
        if isinstance(opts, SolveOpts) else SolveOpts()
    out.lanes, out.warps, out.row_blocks, out.pair_cases, out.stage_v, out.stage_y = (
        o.lanes, o.warps, o.row_blocks, o.pair_cases, o.stage_v, o.stage_y)
    return out


def dpf_solve_iterate(ws: Workspace, n_iter: int, stream=None):
    _check(lib().dpf_solve_iterate(ws.handle, int(n_iter), _stream(stream)))


def dpf_solve_end(ws: Workspace, stream=None, **batch):
    b = _batch_struct(**batch)
    _check(lib().dpf_solve_end(ws.handle, C.byref(b), _stream(stream)))


def dpf_active_count(ws: Workspace, stream=None) -> int:
    n = C.c_int32()
    _check(lib().dpf_active_count(ws.handle, C.byref(n), _stream(stream)))
    return n.value


def dpf_profile_enable(ws: Workspace, on: bool = True):
    _check(lib().dpf_profile_enable(ws.handle, 1 if on else 0))


def dpf_kernel_times(ws: Workspace, stream=None):
    """(fwd_ms_total, adj_ms_total, n_fwd, n_adj) of the bracketed launches."""
    f, a = C.c_double(), C.c_double()
    nf, na = C.c_int32(), C.c_int32()
    _check(lib().dpf_kernel_times(ws.handle, C.byref(f), C.byref(a), C.byref(nf), C.byref(na), _stream(stream)))
    return f.value, a.value, nf.value, na.value


def dpf_kernel_launches(ws: Workspace) -> int:
    n = C.c_int64()
    _check(lib().dpf_kernel_launches(ws.handle, C.byref(n)))
    return n.value


def dpf_read_bandwidth(buf, reps: int = 20, stream=None) -> float:
    """GB/s of the library's read probe over a device tensor (see include/dpf.h)."""
    g = C.c_double()
    _check(lib().dpf_read_bandwidth(_ptr(buf), int(buf.numel() * buf.element_size()), int(reps), C.byref(g),
                                    _stream(stream)))
    return g.value


def dpf_grid_barrier_cost(ctas_per_sm: int = 4, reps: int = 1000, stream=None) -> float:
    """Microseconds per grid-wide barrier of a cooperative launch (see include/dpf.h)."""
    us = C.c_double()
    _check(lib().dpf_grid_barrier_cost(int(ctas_per_sm), int(reps), C.byref(us), _stream(stream)))
    return us.value


def dpf_iterations_done(ws: Workspace) -> int:
    n = C.c_int32()
    _check(lib().dpf_iterations_done(ws.handle, C.byref(n)))
    return n.value


# ---- evaluation ----------------------------------------------------------------
def _check_states(y: Ybus, *tensors):
    """The per-case arrays of an evaluation call: float64 CUDA tensors of one
    shape (K, n_bus) on one device, contiguous (the C ABI sees only K)."""
    import torch
    ref = tensors[0]
    if ref.dim() != 2 or ref.shape[1] != y.n_bus or ref.shape[0] < 1:
        raise ValueError(f"expected a (n_case, {y.n_bus}) array, got {tuple(ref.shape)}")
    for t in tensors:
        if t is None:
            continue
        if not torch.is_tensor(t) or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError("per-case arrays must be float64 CUDA tensors")
        if tuple(t.shape) != tuple(ref.shape) or t.device != ref.device or not t.is_contiguous():
            raise ValueError("per-case arrays must share one contiguous (n_case, n_bus) shape and device")


def dpf_power(y: Ybus, ws: Workspace, va, vm, outage=None, precision=_abi.FP32, stream=None):
    """(P_calc, Q_calc) [K][N] float64 CUDA tensors."""
    import torch
    _check_states(y, va, vm)
    p = torch.empty_like(va)
    q = torch.empty_like(va)
    _check(lib().dpf_power(y.handle, ws.handle, int(va.shape[0]), _ptr(va), _ptr(vm), _ptr(outage),
                           int(precision), _ptr(p), _ptr(q), _stream(stream)))
    return p, q


def dpf_power_noalloc(y: Ybus, va, vm, p_calc, q_calc, stream=None):
    """FP64 S_calc into caller-provided tensors without any device allocation.

    For callers that cannot allocate device memory (see include/dpf.h); the
    library's fixed scratch limits n_case * n_bus to NOALLOC_MAX_ELEMS.
    """
    _check_states(y, va, vm, p_calc, q_calc)
    _check(lib().dpf_power_noalloc(y.handle, int(va.shape[0]), _ptr(va), _ptr(vm), _ptr(p_calc), _ptr(q_calc),
                                   _stream(stream)))


def dpf_loss_backward(y: Ybus, ws: Workspace, va, vm, p_spec=None, q_spec=None, outage=None,
                      g_series=None, b_series=None, precision=_abi.FP32, want=("loss", "d_va", "d_vm"),
                      stream=None):
    """Loss per case and the requested gradients, as float64 CUDA tensors (dict)."""
    import torch
    K, N = va.shape
    M = y.n_branch
    out = {}
    shapes = dict(loss=(K,), d_va=(K, N), d_vm=(K, N), d_p=(K, N), d_q=(K, N), d_g=(M,), d_b=(M,), d_bch=(M,))
    for name in want:
        out[name] = torch.empty(shapes[name], dtype=torch.float64, device=va.device)
    g = [out.get(n) for n in ("loss", "d_va", "d_vm", "d_p", "d_q", "d_g", "d_b", "d_bch")]
    _check(lib().dpf_loss_backward(y.handle, ws.handle, int(K), _ptr(va), _ptr(vm), _ptr(p_spec), _ptr(q_spec),
                                   _ptr(outage), _ptr(g_series), _ptr(b_series), int(precision),
                                   *[_ptr(t) for t in g], _stream(stream)))
    return out


def dpf_dc_solve(y: Ybus, ws: Workspace, n_case: int, p_spec=None, outage=None, tol: float = 1e-10,
                 max_iter: int = 10000, stream=None):
    """DC angles [n_case][N] (float64 CUDA), CG iterations and relative residual per case."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    va = torch.empty((n_case, y.n_bus), dtype=torch.float64, device=dev)
    it = torch.empty(n_case, dtype=torch.int32, device=dev)
    res = torch.empty(n_case, dtype=torch.float64, device=dev)
    _check(lib().dpf_dc_solve(y.handle, ws.handle, int(n_case), _ptr(p_spec), _ptr(outage), float(tol), int(max_iter),
                              _ptr(va), _ptr(it), _ptr(res), _stream(stream)))
    return dict(va=va, iters=it, rel_residual=res)


# ---- Newton-Raphson (Alg. 2) ---------------------------------------------------
def dpf_nr_analyze(y: Ybus) -> dict:
    """Sizes of the host analysis of the Newton solver (no CUDA call)."""
    npos, npairs, nl = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().dpf_nr_analyze(y.handle, C.byref(npos), C.byref(npairs), C.byref(nl)))
    return dict(n_pos=npos.value, n_pairs=npairs.value, n_levels=nl.value)


def dpf_nr_pattern(y: Ybus) -> dict:
    """Elimination order (user bus indices), filled pattern in that order and
    tree levels of the Newton solver's host analysis (no CUDA call)."""
    sz = dpf_nr_analyze(y)
    n = y.n_bus
    order = np.empty(n, np.int32)
    row_ptr = np.empty(n + 1, np.int32)
    col = np.empty(sz["n_pos"], np.int32)
    level = np.empty(n, np.int32)
    _check(lib().dpf_nr_pattern(y.handle, order.ctypes.data, row_ptr.ctypes.data, col.ctypes.data,
                                level.ctypes.data))
    return dict(order=order, row_ptr=row_ptr, col=col, level=level, **sz)


class NewtonSolver:
    """dpf_nr handle: host analysis + device buffers for up to max_case cases."""

    def __init__(self, y: Ybus, max_case: int):
        self.ybus = y
        h = C.c_void_p()
        _check(lib().dpf_nr_create(y.handle, int(max_case), C.byref(h)))
        self.handle = h

    def free(self):
        if self.handle:
            lib().dpf_nr_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        npos, npairs, nl, nlaunch = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64()
        _check(lib().dpf_nr_stats(self.handle, C.byref(npos), C.byref(npairs), C.byref(nl), C.byref(nlaunch)))
        return dict(n_pos=npos.value, n_pairs=npairs.value, n_levels=nl.value, launches=nlaunch.value)


def dpf_nr_create(y: Ybus, max_case: int) -> NewtonSolver:
    return NewtonSolver(y, max_case)


def dpf_nr_solve(nr: NewtonSolver, precision=_abi.FP64, tol: float = 1e-10, max_iter: int = 20, flat_start=True,
                 lanes: int = 0, fallback=False, stream=None, **batch):
    """Newton-Raphson for every case; `batch` holds the dpf_batch fields as CUDA tensors (va, vm required).
    fallback (with flat_start False): unconverged cases keep their start."""
    b = _batch_struct(**batch)
    o = _abi.DpfNrOpts()
    lib().dpf_nr_default_opts(C.byref(o))
    o.precision, o.tol, o.max_iter = int(precision), float(tol), int(max_iter)
    o.flat_start, o.lanes, o.fallback = (1 if flat_start else 0), int(lanes), (1 if fallback else 0)
    _check(lib().dpf_nr_solve(nr.handle, C.byref(b), C.byref(o), _stream(stream)))


def dpf_paramid_begin(y: Ybus, ws: Workspace, va, vm, p_spec=None, q_spec=None, precision=_abi.FP32, stream=None):
    """Stage K measured operating points ([K][N] float64 CUDA tensors) for dpf_paramid_step."""
    _check(lib().dpf_paramid_begin(y.handle, ws.handle, int(va.shape[0]), _ptr(va), _ptr(vm), _ptr(p_spec),
                                   _ptr(q_spec), int(precision), _stream(stream)))
    ws.pid_cases = int(va.shape[0])


def dpf_paramid_step(y: Ybus, ws: Workspace, g_series, b_series, want=("d_g", "d_b"), out=None, stream=None):
    """Branch gradients (and optionally the loss) at the staged operating points.

    `out` may hold preallocated float64 CUDA tensors by name (reused across
    steps); missing ones are allocated.  Returns the dict of requested outputs.
    """
    import torch
    M = y.n_branch
    out = dict(out or {})
    for name in want:
        if name not in out:
            n = getattr(ws, "pid_cases", 0) if name == "loss" else M
            out[name] = torch.empty(n, dtype=torch.float64, device=g_series.device)
    g = [out.get(n) if n in want else None for n in ("d_g", "d_b", "d_bch", "loss")]
    _check(lib().dpf_paramid_step(y.handle, ws.handle, _ptr(g_series), _ptr(b_series),
                                  *[_ptr(t) for t in g], _stream(stream)))
    return {k: out[k] for k in want}


def dpf_adam_update(x, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, lr_scale=None, stream=None):
    """One Adam step on device float64 vectors (in place on x, m, v)."""
    _check(lib().dpf_adam_update(int(x.numel()), _ptr(x), _ptr(grad), _ptr(m), _ptr(v), _ptr(lr_scale), int(t),
                                 float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))


def dpf_last_error() -> str:
    return lib().dpf_last_error().decode()


def dpf_status_str(code: int) -> str:
    return lib().dpf_status_str(int(code)).decode()
