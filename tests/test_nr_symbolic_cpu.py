"""CPU checks of the Newton solver's host analysis (dpf_nr_analyze /
dpf_nr_pattern): the elimination order, the filled block pattern and the
elimination-tree levels.  No GPU call is made.

The pin is independent of the library's bookkeeping: Gaussian elimination
without pivoting of a dense matrix with random values on Y_bus's pattern,
in the reported order, must produce nonzeros exactly on the reported
filled pattern (generic values leave no accidental zeros, so the numerical
and the symbolic fill coincide)."""
import os

import numpy as np
import pytest

import gridgen
from conftest import small_grid


@pytest.fixture(scope="module")
def dpf():
    from paper_2603_28203_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    import paper_2603_28203_gb300 as m
    m.lib()
    return m


def _dense_fill(g, order, seed):
    """Nonzero pattern of L + U from dense elimination (no pivoting) of a
    diagonally dominant random matrix on the graph of the grid, rows and
    columns in `order`."""
    n = g.n_bus
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    for f, t in zip(g.f_bus, g.t_bus):
        A[f, t] = rng.uniform(0.5, 1.5)
        A[t, f] = rng.uniform(0.5, 1.5)
    A[np.arange(n), np.arange(n)] = np.abs(A).sum(1) + 1.0
    A = A[np.ix_(order, order)]
    for k in range(n - 1):
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return np.abs(A) > 1e-13


def _structural_fill(g, order):
    """Filled pattern of elimination in `order`, by the graph rule: eliminating
    a vertex joins all its not yet eliminated neighbours (no arithmetic)."""
    n = g.n_bus
    rank = np.empty(n, int)
    rank[order] = np.arange(n)
    adj = [set() for _ in range(n)]
    for f, t in zip(g.f_bus, g.t_bus):
        adj[rank[f]].add(rank[t])
        adj[rank[t]].add(rank[f])
    pat = np.eye(n, dtype=bool)
    for k in range(n):
        later = sorted(j for j in adj[k] if j > k)
        for a in later:
            pat[k, a] = pat[a, k] = True
            adj[a].update(b for b in later if b != a)
    return pat


@pytest.mark.parametrize("n,seed", [(30, 0), (200, 5), (600, 9)])
def test_filled_pattern_equals_elimination_fill(dpf, n, seed):
    g = small_grid(n, seed)
    y = dpf.dpf_build_ybus_host(g)
    p = dpf.dpf_nr_pattern(y)
    order = p["order"]
    assert np.array_equal(np.sort(order), np.arange(n))          # a permutation
    rp, col = p["row_ptr"], p["col"]
    assert rp[0] == 0 and rp[-1] == p["n_pos"] == col.size
    pat = np.zeros((n, n), bool)
    for r in range(n):
        c = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0)                            # sorted, no duplicates
        assert r in c                                            # diagonal present
        pat[r, c] = True
    assert np.array_equal(pat, pat.T)                            # symmetric pattern
    np.testing.assert_array_equal(pat, _dense_fill(g, order, seed + 1))
    np.testing.assert_array_equal(pat, _structural_fill(g, order))


@pytest.mark.parametrize("n,seed", [(30, 0), (300, 2)])
def test_levels_follow_the_elimination_tree(dpf, n, seed):
    g = small_grid(n, seed)
    y = dpf.dpf_build_ybus_host(g)
    p = dpf.dpf_nr_pattern(y)
    rp, col, level = p["row_ptr"], p["col"], p["level"]
    height = np.zeros(n, int)
    for r in range(n):                                           # parent = first U column
        up = col[rp[r]:rp[r + 1]]
        up = up[up > r]
        if up.size:
            height[up[0]] = max(height[up[0]], height[r] + 1)
    np.testing.assert_array_equal(level, height)
    assert p["n_levels"] == level.max() + 1
    # every L column of a row sits on a strictly lower level (its updates are final first)
    for r in range(n):
        lo = col[rp[r]:rp[r + 1]]
        lo = lo[lo < r]
        assert np.all(level[lo] < level[r])


def test_update_count_is_the_sum_of_squared_u_rows(dpf):
    g = small_grid(200, 5)
    y = dpf.dpf_build_ybus_host(g)
    p = dpf.dpf_nr_pattern(y)
    rp, col = p["row_ptr"], p["col"]
    nu = np.array([(col[rp[r]:rp[r + 1]] > r).sum() for r in range(g.n_bus)])
    assert p["n_pairs"] == int((nu.astype(np.int64) ** 2).sum())


def test_fill_of_the_contingency_grid_is_moderate(dpf):
    """Minimum degree on the 2,000-bus grid: the factor stays within a small
    multiple of Y_bus (nnz = N + 2M)."""
    g = gridgen.config_grid("c3_n1_2kbus")
    y = dpf.dpf_build_ybus_host(g)
    s = dpf.dpf_nr_analyze(y)
    nnz = g.n_bus + 2 * g.n_branch
    assert nnz <= s["n_pos"] <= 6 * nnz
    assert s["n_levels"] < g.n_bus


def test_block_diagonal_batch_keeps_its_islands_apart(dpf):
    """Several grids in one Y_bus (one slack per island, the uneven batch):
    the elimination fills only within an island, and the filled pattern is
    exactly the fill of graph elimination in the reported order.  (Dense
    numeric elimination is not used here: along the long elimination chains
    of this batch some fill values decay below any fixed zero threshold.)"""
    grids = [gridgen.make_grid(n, 100 + i, n_branch=int(1.35 * n), n_pv=max(1, n // 8))
             for i, n in enumerate((40, 120, 75))]
    cat = gridgen.concat_grids(grids)
    y = dpf.dpf_build_ybus_host(cat)
    p = dpf.dpf_nr_pattern(y)
    n = cat.n_bus
    island = np.repeat(np.arange(len(grids)), [g.n_bus for g in grids])
    order, rp, col = p["order"], p["row_ptr"], p["col"]
    pat = np.zeros((n, n), bool)
    for r in range(n):
        c = col[rp[r]:rp[r + 1]]
        assert np.all(island[order[c]] == island[order[r]])
        pat[r, c] = True
    np.testing.assert_array_equal(pat, _structural_fill(cat, order))


@pytest.mark.parametrize("seed", range(12))
def test_random_grids_fill_and_levels(dpf, seed):
    """Random small grids (sizes 4..90, branch ratios 1.0..1.8): the filled
    pattern equals graph-elimination fill in the reported order, every
    position's pivot sits on a level no higher than either of its rows, and
    the L columns of a row are on strictly lower levels."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 91))
    m = max(n - 1, int(round(n * rng.uniform(1.0, 1.8))))
    g = gridgen.make_grid(n, 500 + seed, n_branch=m, n_pv=max(1, n // 6))
    y = dpf.dpf_build_ybus_host(g)
    p = dpf.dpf_nr_pattern(y)
    order, rp, col, level = p["order"], p["row_ptr"], p["col"], p["level"]
    assert np.array_equal(np.sort(order), np.arange(n))
    pat = np.zeros((n, n), bool)
    for r in range(n):
        c = col[rp[r]:rp[r + 1]]
        pat[r, c] = True
        lo = c[c < r]
        assert np.all(level[lo] < level[r])
    np.testing.assert_array_equal(pat, _structural_fill(g, order))
