"""DC approximation of the power flow (oracle; test infrastructure).

The paper lists the DC approximation as the linearised comparison model and
as an optional initialisation (Sec. 2, Table 1, Alg. 2).  Its textbook form:
with |V| = 1, no resistance, no charging and small angle differences, the
active flow of branch l = (f, t) is b_l (theta_f - theta_t) with
b_l = 1 / (x_l tau_l) (the series reactance seen through the tap, tau at the
from-bus; tau 0 read as 1), and the injections satisfy

    B theta = P,   B = sum_l b_l (e_f - e_t)(e_f - e_t)^T,

over the pv and pq buses, the slack angles being fixed (one slack per
island).  An outaged branch is left out of B.  scipy's sparse solve is the
linear-algebra step.

Outage shift (a start for the N-1 cases of a warm-started batch, built on the
DC model above; the paper's warm starts of Sec. 5.4.2 and its DC
initialisation combined): for angles theta and an outaged branch l, the
angle change that removing l causes in the DC model,

    B' dtheta = (B - B') theta   on the pv and pq rows,  dtheta = 0 at slacks,

with B' the matrix without l, so that B' (theta + dtheta) = B theta there:
the injections theta implies stay, carried by the remaining branches.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .power import SLACK


def dc_susceptance(x, tap):
    """b_l = 1 / (x_l tau_l)."""
    tau = np.where(np.asarray(tap, np.float64) == 0.0, 1.0, np.asarray(tap, np.float64))
    return 1.0 / (np.asarray(x, np.float64) * tau)


def dc_matrix(n_bus, f_bus, t_bus, x, tap, outage=-1):
    """B (CSR, n x n) of the branches except `outage`."""
    b = dc_susceptance(x, tap)
    keep = np.ones(b.size, bool)
    if outage is not None and outage >= 0:
        keep[outage] = False
    f, t, b = np.asarray(f_bus)[keep], np.asarray(t_bus)[keep], b[keep]
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([b, b, -b, -b])
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_bus, n_bus)).tocsr()


def dc_solve(n_bus, f_bus, t_bus, x, tap, bus_type, p_spec, va_slack=0.0, outage=-1):
    """Angles theta [n_bus] of the DC power flow (slack angles = va_slack)."""
    bus_type = np.asarray(bus_type)
    B = dc_matrix(n_bus, f_bus, t_bus, x, tap, outage)
    s = np.where(bus_type == SLACK)[0]
    u = np.where(bus_type != SLACK)[0]
    theta = np.zeros(n_bus)
    theta[s] = va_slack
    rhs = np.asarray(p_spec, np.float64)[u] - B[u][:, s] @ theta[s]
    theta[u] = spl.spsolve(B[u][:, u].tocsc(), rhs)
    return theta


def dc_branch_flows(f_bus, t_bus, x, tap, theta):
    """Active flow of every branch from its from-bus, b_l (theta_f - theta_t)."""
    b = dc_susceptance(x, tap)
    theta = np.asarray(theta, np.float64)
    return b * (theta[np.asarray(f_bus)] - theta[np.asarray(t_bus)])


def dc_outage_shift(n_bus, f_bus, t_bus, x, tap, bus_type, theta, outage):
    """dtheta [n_bus] with B' dtheta = (B - B') theta on the non-slack rows and
    dtheta = 0 at the slack buses (B' without branch `outage`; zero for -1)."""
    theta = np.asarray(theta, np.float64)
    if outage is None or outage < 0:
        return np.zeros(n_bus)
    bus_type = np.asarray(bus_type)
    B = dc_matrix(n_bus, f_bus, t_bus, x, tap)
    Bo = dc_matrix(n_bus, f_bus, t_bus, x, tap, outage)
    u = np.where(bus_type != SLACK)[0]
    rhs = ((B - Bo) @ theta)[u]
    d = np.zeros(n_bus)
    d[u] = spl.spsolve(Bo[u][:, u].tocsc(), rhs)
    return d
