"""Bus admittance matrix from the branch table (oracle; test infrastructure).

The paper takes Y_bus as given (Sec. 2.1) and points to the MATPOWER manual,
sections 3.6 and 4.1, for the model behind Eq. powerbalance.  That model is
the branch pi-equivalent: a series admittance y_s = 1/(r + j x), total line
charging b_ch split half to each end, and an ideal transformer of ratio tau at
the from-bus.  Its 2x2 contribution to Y_bus, in (from, to) order, is

    [ (y_s + j b_ch/2) / tau^2     -y_s / tau      ]
    [ -y_s / tau                   y_s + j b_ch/2  ]

(no phase shift, so the block is symmetric).  Bus shunts are zero in every
synthetic grid.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def branch_blocks(r, x, b_ch, tap):
    """Per-branch (Y_ff, Y_ft, Y_tf, Y_tt) of the pi-model, complex float64."""
    r = np.asarray(r, np.float64)
    x = np.asarray(x, np.float64)
    b_ch = np.asarray(b_ch, np.float64)
    tau = np.asarray(tap, np.float64)
    tau = np.where(tau == 0.0, 1.0, tau)  # MATPOWER convention: 0 means "no tap"
    y_s = 1.0 / (r + 1j * x)
    y_sh = 0.5j * b_ch
    y_ff = (y_s + y_sh) / tau ** 2
    y_ft = -y_s / tau
    y_tf = -y_s / tau
    y_tt = y_s + y_sh
    return y_ff, y_ft, y_tf, y_tt


def build_ybus(n_bus, f_bus, t_bus, r, x, b_ch, tap, shift=None):
    """Y_bus (scipy CSR, complex128, n_bus x n_bus), summing branch blocks.

    A plain loop over branches adds each 2x2 block at (f, f), (f, t), (t, f),
    (t, t); duplicate positions (parallel branches) are summed.
    """
    if shift is not None and np.any(np.asarray(shift) != 0.0):
        raise ValueError("phase-shifting transformers are not modelled")
    y_ff, y_ft, y_tf, y_tt = branch_blocks(r, x, b_ch, tap)
    acc: dict[tuple[int, int], complex] = {}

    def add(i, j, v):
        acc[(i, j)] = acc.get((i, j), 0.0) + v

    for ell in range(len(f_bus)):
        f, t = int(f_bus[ell]), int(t_bus[ell])
        add(f, f, y_ff[ell])
        add(f, t, y_ft[ell])
        add(t, f, y_tf[ell])
        add(t, t, y_tt[ell])
    for i in range(n_bus):  # every bus has a diagonal entry, even if isolated
        add(i, i, 0.0)
    keys = sorted(acc)
    rows = np.array([k[0] for k in keys], np.int64)
    cols = np.array([k[1] for k in keys], np.int64)
    vals = np.array([acc[k] for k in keys], np.complex128)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_bus, n_bus))


def grid_ybus(grid):
    """Y_bus of a `gridgen.Grid`."""
    return build_ybus(grid.n_bus, grid.f_bus, grid.t_bus, grid.r, grid.x,
                      grid.b_ch, grid.tap, grid.shift)
