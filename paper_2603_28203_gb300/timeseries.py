"""Time-series power flows with warm starts (Sec. 5.4.2, Table 3).

Snapshots are solved in windows of `window` cases per batched call.  The
first window starts flat with the t = 0 settings of Table 3 (Adam lr 0.03564,
betas (0.9802, 0.9440), StepLR step 100 / gamma 0.773, <= 1,000 iterations);
every later window starts from the solutions of the previous window,
snapshot by snapshot (snapshot t from snapshot t - window, the same hour of
day for a 96-hour window), with the t > 0 settings (Adam lr 0.00027, betas
(0.7847, 0.6624), ReduceLROnPlateau 0.8 / 2 / 0.0388 / 4, <= 300 iterations).
With `warm_from="last"` (the other reading of Sec. 5.4.2's warm start) every
snapshot of a window starts from the solution of the previous window's last
snapshot instead (one shared start, dpf_batch.va_start).  The solutions stay
on the device between windows; only the window's injections are copied in.
All arithmetic runs in the library's kernels.

With `first_newton`, the first window's Alg. 1 solutions are handed to
Newton-Raphson on the GPU (dpf_nr_solve, FP32 factor, to 1e-10 p.u.) as
start and fallback: a snapshot Newton solves leaves the window exact, one it
cannot keeps Alg. 1's state.  (The caption of Fig. 4 notes the first full fit
could be replaced by Newton-Raphson; Sec. 6 names gradient methods as the
initialisers of Newton solves.)  With `newton_from="flat"` the first window
skips the Alg. 1 fit: Newton-Raphson solves it from the flat start, and
Alg. 1 runs only on the warm-started windows after it.

With `checkpoint` (a directory), every solved window is saved as
window_<first snapshot>.npz (its solutions, iterations, statuses, mismatches
and losses, and a fingerprint of what it was solved from: the window's
injections, the precision, tolerance, test interval and optimiser settings,
and whether its start was flat or the previous window's); with `resume`,
saved windows are loaded instead of solved -- a file whose fingerprint
differs from the one this call would solve is rejected (ValueError) -- and
the last loaded window's solutions warm-start the next one, so an
interrupted series continues where it stopped.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import _abi
from .dpf import NewtonSolver, SolveOpts, Workspace, Ybus, dpf_nr_solve, dpf_solve_batch

TABLE3_T0 = dict(lr=0.03564, beta1=0.9802, beta2=0.9440, sched=_abi.SCHED_STEP, step_size=100, gamma=0.773,
                 max_iter=1000)
TABLE3_T1 = dict(lr=0.00027, beta1=0.7847, beta2=0.6624, sched=_abi.SCHED_PLATEAU, factor=0.8, patience=2,
                 threshold=0.0388, cooldown=4, max_iter=300)


def _fingerprint(p, q, precision, tol, check_every, settings, first_newton, w0, window, newton_from="dpf",
                 warm_from="same_hour"):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(p.cpu().numpy()).tobytes())
    h.update(np.ascontiguousarray(q.cpu().numpy()).tobytes())
    h.update(json.dumps(dict(precision=int(precision), tol=float(tol), check_every=int(check_every),
                             settings={k: settings[k] for k in sorted(settings)},
                             newton=(newton_from if first_newton is not None and w0 == 0 else False),
                             warm=(warm_from if w0 > 0 else False),
                             window=int(window)), sort_keys=True).encode())
    return h.hexdigest()


def solve_time_series(y: Ybus, ws: Workspace, p_series, q_series, window: int = 96, precision=_abi.FP32,
                      first=None, later=None, check_every: int = 25, tol: float = 1e-6, stream=None,
                      first_newton: NewtonSolver | None = None, newton_from: str = "dpf",
                      checkpoint: str | None = None, resume: bool = False, warm_from: str = "same_hour"):
    """Solve T snapshots ([T][N] injections, numpy or torch); returns numpy arrays.

    `first` / `later` override the Table 3 settings (dicts of SolveOpts fields).
    `first_newton`: a NewtonSolver for `window` cases of this Y_bus; the first
    window's Alg. 1 solutions then go through Newton-Raphson (start and
    fallback; its `iters` and `status` are then Newton's); with
    `newton_from="flat"` Newton-Raphson alone solves the first window from
    the flat start.
    `checkpoint` / `resume`: per-window save and restart (module docstring).
    `warm_from`: "same_hour" (snapshot t from snapshot t - window) or "last"
    (a window's every snapshot from the previous window's last snapshot).
    """
    if newton_from not in ("dpf", "flat"):
        raise ValueError(f"newton_from must be 'dpf' or 'flat', not {newton_from!r}")
    if warm_from not in ("same_hour", "last"):
        raise ValueError(f"warm_from must be 'same_hour' or 'last', not {warm_from!r}")
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    P = torch.as_tensor(np.asarray(p_series, np.float64) if not torch.is_tensor(p_series) else p_series,
                        dtype=torch.float64)
    Q = torch.as_tensor(np.asarray(q_series, np.float64) if not torch.is_tensor(q_series) else q_series,
                        dtype=torch.float64)
    T, N = P.shape
    out = {k: np.empty((T, N)) for k in ("va", "vm")}
    out.update(iters=np.empty(T, np.int32), status=np.empty(T, np.int32), max_mismatch=np.empty(T),
               loss=np.empty(T))
    va = torch.zeros((window, N), dtype=torch.float64, device=dev)
    vm = torch.zeros((window, N), dtype=torch.float64, device=dev)
    res = dict(iters=torch.zeros(window, dtype=torch.int32, device=dev),
               status=torch.zeros(window, dtype=torch.int32, device=dev),
               max_mismatch=torch.zeros(window, dtype=torch.float64, device=dev),
               loss=torch.zeros(window, dtype=torch.float64, device=dev))
    if checkpoint:
        os.makedirs(checkpoint, exist_ok=True)
    for w0 in range(0, T, window):
        K = min(window, T - w0)
        path = os.path.join(checkpoint, f"window_{w0:06d}.npz") if checkpoint else None
        settings = dict(TABLE3_T0 if w0 == 0 else TABLE3_T1)
        settings.update((first if w0 == 0 else later) or {})
        fp = _fingerprint(P[w0:w0 + K], Q[w0:w0 + K], precision, tol, check_every, settings, first_newton, w0,
                          window, newton_from, warm_from) if path else None
        if resume and path and os.path.exists(path):
            with np.load(path) as z:
                if z["va"].shape != (K, N):
                    raise ValueError(f"{path}: saved window has shape {z['va'].shape}, expected {(K, N)}")
                if "fingerprint" not in z.files or str(z["fingerprint"]) != fp:
                    raise ValueError(f"{path}: saved window was solved from other inputs or settings")
                for k in out:
                    out[k][w0:w0 + K] = z[k]
            va[:K] = torch.as_tensor(out["va"][w0:w0 + K], device=dev)
            vm[:K] = torch.as_tensor(out["vm"][w0:w0 + K], device=dev)
            last = K
            continue
        p = P[w0:w0 + K].to(dev).contiguous()
        q = Q[w0:w0 + K].to(dev).contiguous()
        opts = SolveOpts(precision=precision, check_every=check_every, tol=tol, flat_start=1 if w0 == 0 else 0,
                         **settings)
        newton_only = w0 == 0 and first_newton is not None and newton_from == "flat"
        shared = {}
        if w0 > 0 and warm_from == "last":  # the previous window's last solution, for every snapshot
            shared = dict(va_start=va[last - 1].clone(), vm_start=vm[last - 1].clone())
        if not newton_only:
            dpf_solve_batch(y, ws, opts, stream=stream, n_case=K, p_spec=p, q_spec=q, va=va[:K], vm=vm[:K],
                            **shared, **{k: v[:K] for k, v in res.items()})
        if w0 == 0 and first_newton is not None:
            dpf_nr_solve(first_newton, precision=_abi.FP32, tol=1e-10, max_iter=20, flat_start=newton_only,
                         fallback=not newton_only, stream=stream, n_case=K, p_spec=p, q_spec=q, va=va[:K],
                         vm=vm[:K], **{k: v[:K] for k, v in res.items()})
        out["va"][w0:w0 + K] = va[:K].cpu().numpy()
        out["vm"][w0:w0 + K] = vm[:K].cpu().numpy()
        last = K
        for k, v in res.items():
            out[k][w0:w0 + K] = v[:K].cpu().numpy()
        if path:
            tmp = path + ".tmp.npz"
            np.savez(tmp, fingerprint=np.array(fp), **{k: out[k][w0:w0 + K] for k in out})
            os.replace(tmp, path)  # a window file is complete or absent
    return out
