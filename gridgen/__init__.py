"""Seeded synthetic power-grid generator.

This module produces INPUTS only: bus positions, branch tables, bus types and
specified injections.  It holds none of the power-flow arithmetic (no
admittance matrix, no power, no mismatch); both the CPU oracle and the CUDA
path consume what it returns.

The paper measures on IEEE-118, case9241pegase and the LIPS time series
(Sec. 5.1), none of which are available here.  These generators stand in for
them with grids of matching shape: 10,000-bus meshed grids with ~37k Y_bus
nonzeros, close to case9241pegase's 37,655 (Sec. 5.4.3, Fig. node_and_edge_scaling).

Recipe (one grid):
  * buses uniform in the unit square;
  * a spanning tree = Euclidean minimum spanning tree of the 8-nearest-neighbour
    graph, plus extra edges drawn without replacement from 4-nearest-neighbour
    pairs not in the tree, until the branch count is reached
    (default round(1.35 N));
  * series r ~ U(0.002, 0.02) p.u., x = r * U(5, 15), total charging
    b ~ U(0, 0.05); 10% of branches are transformers with an off-nominal tap
    U(0.95, 1.05) at the from-bus; no phase shifters;
  * slack = highest-degree bus (lowest index on ties), |V| = 1, angle 0;
  * PV buses chosen uniformly among the rest (round(0.15 N) by default) with
    |V| set-points U(0.98, 1.05);
  * PQ buses carry loads P ~ lognormal(mean 0.3 p.u., sigma_log 0.5) at power
    factor 0.95 (lagging);
  * PV dispatch sums to `dispatch` x total load, split in proportion to
    U(0.5, 1.5) weights;
  * loads are multiplied by `load_scale`.  With the stated load level
    (mean 0.3 p.u.) a Newton-Raphson continuation solves the 2,000-bus grid
    only up to ~20% and the 10,000-bus grid up to ~12% of it (long pendant
    chains of PQ buses behind single branches collapse in voltage), so the
    large workloads use load_scale = 0.1; the 30-bus grid solves at full load.
    The 10,000-bus time-series grid uses 0.05: its load model peaks at 1.44x
    the base load (winter noon), and at 0.1 Newton-Raphson from a flat or
    base-case start fails on the peak hours (42% of the year) while at 0.05
    it solves every hour.

Specified injections are net (generation - load) in p.u.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
from scipy.spatial import cKDTree

PQ, PV, SLACK = 0, 1, 2


@dataclasses.dataclass
class Grid:
    """One synthetic grid.  Arrays are numpy, bus-indexed or branch-indexed."""

    bus_type: np.ndarray  # uint8 [N]: 0 PQ, 1 PV, 2 slack
    p_spec: np.ndarray  # float64 [N] net active injection (p.u.)
    q_spec: np.ndarray  # float64 [N] net reactive injection (p.u.; used at PQ)
    vm_set: np.ndarray  # float64 [N] |V| set-point (PV, slack); 1.0 at PQ
    va_slack: float  # slack angle (rad)
    f_bus: np.ndarray  # int32 [M]
    t_bus: np.ndarray  # int32 [M]
    r: np.ndarray  # float64 [M]
    x: np.ndarray  # float64 [M]
    b_ch: np.ndarray  # float64 [M] total line charging
    tap: np.ndarray  # float64 [M] off-nominal ratio at the from-bus (1 = none)
    shift: np.ndarray  # float64 [M] phase shift (always 0 here)
    pos: np.ndarray  # float64 [N,2] bus coordinates
    p_load: np.ndarray  # float64 [N] base active load (PQ buses)
    q_load: np.ndarray  # float64 [N] base reactive load
    gen_w: np.ndarray  # float64 [N] PV dispatch weights (0 elsewhere)
    dispatch: float

    @property
    def n_bus(self) -> int:
        return int(self.bus_type.shape[0])

    @property
    def n_branch(self) -> int:
        return int(self.f_bus.shape[0])

    @property
    def slack(self) -> int:
        return int(np.flatnonzero(self.bus_type == SLACK)[0])

    @property
    def pv(self) -> np.ndarray:
        return np.flatnonzero(self.bus_type == PV)

    @property
    def pq(self) -> np.ndarray:
        return np.flatnonzero(self.bus_type == PQ)

    def copy(self) -> "Grid":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy()
                              if isinstance(getattr(self, f.name), np.ndarray)
                              else getattr(self, f.name))
                     for f in dataclasses.fields(self)})

    def without_branch(self, ell: int) -> "Grid":
        """The same grid with branch `ell` removed (N-1 outage)."""
        keep = np.ones(self.n_branch, bool)
        keep[ell] = False
        g = self.copy()
        for name in ("f_bus", "t_bus", "r", "x", "b_ch", "tap", "shift"):
            setattr(g, name, getattr(g, name)[keep])
        return g


def _connect_components(pos, edges):
    """Join the components of an edge set with nearest cross-component pairs."""
    n = pos.shape[0]
    while True:
        e = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
        a = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
        ncomp, lab = connected_components(a, directed=False)
        if ncomp == 1:
            return edges
        # nearest pair between component 0 and any other component
        in0 = np.flatnonzero(lab == 0)
        out = np.flatnonzero(lab != 0)
        tree = cKDTree(pos[out])
        d, j = tree.query(pos[in0])
        k = int(np.argmin(d))
        u, v = int(in0[k]), int(out[j[k]])
        edges.add((min(u, v), max(u, v)))


def _topology(pos, n_branch, rng):
    n = pos.shape[0]
    kt = cKDTree(pos)
    k8 = min(8, n - 1)
    d, nb = kt.query(pos, k=k8 + 1)
    rows = np.repeat(np.arange(n), k8)
    cols = nb[:, 1:].reshape(-1)
    w = d[:, 1:].reshape(-1)
    a = coo_matrix((w, (rows, cols)), shape=(n, n)).tocsr()
    a = a.maximum(a.T)
    mst = minimum_spanning_tree(a).tocoo()
    tree = {(min(int(u), int(v)), max(int(u), int(v))) for u, v in zip(mst.row, mst.col)}
    tree = _connect_components(pos, tree)
    n_extra = n_branch - len(tree)
    if n_extra < 0:
        raise ValueError("n_branch smaller than a spanning tree")
    k4 = min(4, n - 1)
    _, nb4 = kt.query(pos, k=k4 + 1)
    cand = set()
    for i in range(n):
        for j in nb4[i, 1:]:
            e = (min(i, int(j)), max(i, int(j)))
            if e not in tree:
                cand.add(e)
    cand = sorted(cand)
    if n_extra > len(cand):
        raise ValueError("not enough nearest-neighbour pairs for the branch count")
    pick = rng.choice(len(cand), size=n_extra, replace=False)
    edges = sorted(tree) + [cand[i] for i in sorted(pick)]
    return np.array(edges, dtype=np.int64)


def make_grid(n_bus: int, seed: int, n_branch: int | None = None,
              n_pv: int | None = None, tf_frac: float = 0.10,
              load_mean: float = 0.3, load_sigma: float = 0.5, pf: float = 0.95,
              dispatch: float = 1.03, load_scale: float = 1.0) -> Grid:
    """Synthetic meshed grid per the recipe in the module docstring.

    `load_scale` multiplies every drawn load (and hence the dispatch) after the
    draw, so the random stream and topology do not depend on it.
    """
    if n_bus < 2:
        raise ValueError("need at least 2 buses")
    rng = np.random.default_rng(seed)
    if n_branch is None:
        n_branch = max(n_bus - 1, int(round(1.35 * n_bus)))
    if n_pv is None:
        n_pv = int(round(0.15 * n_bus))
    n_pv = min(n_pv, n_bus - 1)
    pos = rng.random((n_bus, 2))
    edges = _topology(pos, n_branch, rng)
    m = edges.shape[0]
    # random orientation: the tap sits at the from-bus
    flip = rng.random(m) < 0.5
    f = np.where(flip, edges[:, 1], edges[:, 0]).astype(np.int32)
    t = np.where(flip, edges[:, 0], edges[:, 1]).astype(np.int32)
    r = rng.uniform(0.002, 0.02, m)
    x = r * rng.uniform(5.0, 15.0, m)
    b_ch = rng.uniform(0.0, 0.05, m)
    tap = np.ones(m)
    n_tf = int(round(tf_frac * m))
    tf = rng.choice(m, size=n_tf, replace=False)
    tap[tf] = rng.uniform(0.95, 1.05, n_tf)
    shift = np.zeros(m)

    deg = np.bincount(np.concatenate([f, t]), minlength=n_bus)
    slack = int(np.argmax(deg))
    others = np.setdiff1d(np.arange(n_bus), [slack])
    pv = np.sort(rng.choice(others, size=n_pv, replace=False))
    bus_type = np.zeros(n_bus, np.uint8)
    bus_type[pv] = PV
    bus_type[slack] = SLACK
    pq = np.flatnonzero(bus_type == PQ)

    vm_set = np.ones(n_bus)
    vm_set[pv] = rng.uniform(0.98, 1.05, n_pv)
    mu = math.log(load_mean) - 0.5 * load_sigma ** 2
    p_load = np.zeros(n_bus)
    p_load[pq] = rng.lognormal(mu, load_sigma, pq.size)
    p_load *= load_scale
    q_load = p_load * math.tan(math.acos(pf))
    gen_w = np.zeros(n_bus)
    gen_w[pv] = rng.uniform(0.5, 1.5, n_pv)
    p_spec, q_spec = _injections(p_load, q_load, gen_w, dispatch)
    return Grid(bus_type=bus_type, p_spec=p_spec, q_spec=q_spec, vm_set=vm_set,
                va_slack=0.0, f_bus=f, t_bus=t, r=r, x=x, b_ch=b_ch, tap=tap,
                shift=shift, pos=pos, p_load=p_load, q_load=q_load, gen_w=gen_w,
                dispatch=dispatch)


def _injections(p_load, q_load, gen_w, dispatch):
    """Net injections: PV generation = dispatch x total load (weights gen_w)."""
    total = p_load.sum(axis=-1, keepdims=True)
    wsum = gen_w.sum()
    p_gen = (dispatch * total * gen_w / wsum) if wsum > 0 else np.zeros_like(p_load)
    return p_gen - p_load, -q_load


def bridges(n_bus: int, f_bus: np.ndarray, t_bus: np.ndarray) -> np.ndarray:
    """Boolean [M]: True where removing the branch disconnects the grid.

    Iterative Tarjan low-link over the (multi)graph; parallel branches are
    never bridges.
    """
    m = len(f_bus)
    adj = [[] for _ in range(n_bus)]
    for e in range(m):
        u, v = int(f_bus[e]), int(t_bus[e])
        adj[u].append((v, e))
        adj[v].append((u, e))
    disc = [-1] * n_bus
    low = [0] * n_bus
    is_bridge = np.zeros(m, bool)
    timer = 0
    for root in range(n_bus):
        if disc[root] != -1:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            u, pe, it = stack[-1]
            advanced = False
            for v, e in it:
                if e == pe:
                    continue
                if disc[v] == -1:
                    disc[v] = low[v] = timer
                    timer += 1
                    stack.append((v, e, iter(adj[v])))
                    advanced = True
                    break
                low[u] = min(low[u], disc[v])
            if not advanced:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[u])
                    if low[u] > disc[p]:
                        is_bridge[pe] = True
    return is_bridge


def n1_outages(grid: Grid) -> np.ndarray:
    """Branches whose single outage leaves the grid connected (int32)."""
    br = bridges(grid.n_bus, grid.f_bus, grid.t_bus)
    return np.flatnonzero(~br).astype(np.int32)


def time_series(grid: Grid, n_snap: int, seed: int, t0: int = 0):
    """Hourly net injections [T][N] for snapshots t0 .. t0+n_snap-1.

    load_i(t) = P0_i (1 + 0.25 sin(2 pi t/24 - pi/2)) (1 + 0.15 cos(2 pi t/8760))
                (1 + eps_it),  eps ~ N(0, 0.05) drawn per bus per snapshot;
    Q scales with P; PV dispatch is rescaled to `dispatch` x that hour's load.
    The noise of snapshot t depends only on (seed, t), so any window can be
    generated on its own.
    """
    t = np.arange(t0, t0 + n_snap, dtype=np.float64)
    daily = 1.0 + 0.25 * np.sin(2 * np.pi * t / 24.0 - np.pi / 2)
    season = 1.0 + 0.15 * np.cos(2 * np.pi * t / 8760.0)
    noise = np.empty((n_snap, grid.n_bus))
    for k in range(n_snap):
        rk = np.random.default_rng([seed, int(t[k])])
        noise[k] = 1.0 + rk.normal(0.0, 0.05, grid.n_bus)
    scale = (daily * season)[:, None] * noise
    p_load = grid.p_load[None, :] * scale
    q_load = grid.q_load[None, :] * scale
    p, q = _injections(p_load, q_load, grid.gen_w[None, :], grid.dispatch)
    return p, q


def perturb_branches(grid: Grid, seed: int, rel: float = 0.10) -> Grid:
    """Copy of `grid` with r and x scaled by (1 + U(-rel, rel)) per branch."""
    rng = np.random.default_rng(seed)
    g = grid.copy()
    g.r = g.r * (1.0 + rng.uniform(-rel, rel, g.n_branch))
    g.x = g.x * (1.0 + rng.uniform(-rel, rel, g.n_branch))
    return g


def add_random_branches(grid: Grid, n_extra: int, seed: int) -> Grid:
    """Copy of `grid` with `n_extra` branches between random bus pairs (no
    duplicates, no self-loops), drawn from the same r / x / b_ch
    distributions; the edge-scaling experiment (Sec. 5.4.3) adds random
    connections the same way."""
    rng = np.random.default_rng(seed)
    g = grid.copy()
    have = set(zip(np.minimum(g.f_bus, g.t_bus).tolist(), np.maximum(g.f_bus, g.t_bus).tolist()))
    f, t = [], []
    while len(f) < n_extra:
        a, b = (int(v) for v in rng.integers(0, g.n_bus, 2))
        key = (min(a, b), max(a, b))
        if a == b or key in have:
            continue
        have.add(key)
        f.append(a)
        t.append(b)
    r = rng.uniform(0.002, 0.02, n_extra)
    x = r * rng.uniform(5.0, 15.0, n_extra)
    g.f_bus = np.concatenate([g.f_bus, np.array(f, np.int32)])
    g.t_bus = np.concatenate([g.t_bus, np.array(t, np.int32)])
    g.r = np.concatenate([g.r, r])
    g.x = np.concatenate([g.x, x])
    g.b_ch = np.concatenate([g.b_ch, rng.uniform(0.0, 0.05, n_extra)])
    g.tap = np.concatenate([g.tap, np.ones(n_extra)])
    g.shift = np.concatenate([g.shift, np.zeros(n_extra)])
    return g


def concat_grids(grids) -> Grid:
    """Block-diagonal batch of grids (one island each), bus indices offset."""
    off = np.cumsum([0] + [g.n_bus for g in grids])
    cat = lambda name: np.concatenate([getattr(g, name) for g in grids])
    return Grid(bus_type=cat("bus_type"), p_spec=cat("p_spec"), q_spec=cat("q_spec"), vm_set=cat("vm_set"),
                va_slack=0.0,
                f_bus=np.concatenate([g.f_bus + o for g, o in zip(grids, off)]).astype(np.int32),
                t_bus=np.concatenate([g.t_bus + o for g, o in zip(grids, off)]).astype(np.int32),
                r=cat("r"), x=cat("x"), b_ch=cat("b_ch"), tap=cat("tap"), shift=cat("shift"),
                pos=cat("pos"), p_load=cat("p_load"), q_load=cat("q_load"), gen_w=cat("gen_w"),
                dispatch=grids[0].dispatch)


def uneven_sizes(n_grids: int, seed: int, lo: int = 300, hi: int = 80_000) -> np.ndarray:
    """Grid sizes log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_grids))).astype(int)


def two_bus(p_load: float, q_load: float, r: float, x: float, e: float = 1.0) -> Grid:
    """Slack (|V|=e, angle 0) feeding one PQ load through z = r + jx, no charging."""
    z = np.zeros(2)
    return Grid(bus_type=np.array([SLACK, PQ], np.uint8),
                p_spec=np.array([0.0, -p_load]), q_spec=np.array([0.0, -q_load]),
                vm_set=np.array([e, 1.0]), va_slack=0.0,
                f_bus=np.array([0], np.int32), t_bus=np.array([1], np.int32),
                r=np.array([r]), x=np.array([x]), b_ch=np.zeros(1), tap=np.ones(1),
                shift=np.zeros(1), pos=np.zeros((2, 2)), p_load=np.array([0.0, p_load]),
                q_load=np.array([0.0, q_load]), gen_w=z.copy(), dispatch=1.0)


# Named workloads (sizes and seeds of the five configurations).
CONFIGS = {
    "c1_30bus_fp64": dict(n_bus=30, seed=0, n_branch=41, n_pv=5),
    "c2_10kbus": dict(n_bus=10_000, seed=1, load_scale=0.1),
    "c3_n1_2kbus": dict(n_bus=2_000, seed=2, load_scale=0.1),
    "c4_timeseries_10kbus": dict(n_bus=10_000, seed=3, load_scale=0.05),
}


def config_grid(name: str) -> Grid:
    """The grid of a named workload."""
    return make_grid(**CONFIGS[name])
