"""CPU checks of the C ABI library: it loads, exports every declared symbol,
and its host-side logic (Y_bus assembly, validation, bridges, defaults) is
right.  No GPU call is made."""
import json
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import gridgen
import oracle
from oracle.ybus import grid_ybus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dpf():
    from paper_2603_28203_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    import paper_2603_28203_gb300 as m
    m.lib()
    return m


def test_exports_every_declared_symbol(dpf):
    src = open(os.path.join(ROOT, "include", "dpf.h")).read()
    names = set(re.findall(r"\b(dpf_[a-z0-9_]+)\s*\(", src))
    assert len(names) >= 15
    L = dpf.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


@pytest.mark.parametrize("name", ["c1_30bus_fp64", "c3_n1_2kbus"])
def test_host_ybus_matches_oracle(dpf, name):
    g = gridgen.config_grid(name)
    y = dpf.dpf_build_ybus_host(g)
    rp, col, val = dpf.dpf_ybus_export(y)
    Y = grid_ybus(g)
    Y.sort_indices()
    np.testing.assert_array_equal(rp, Y.indptr)       # index work: bit-exact
    np.testing.assert_array_equal(col, Y.indices)
    assert np.abs(val - Y.data).max() <= 1e-15 * np.abs(Y.data).max()


def _bridges_brute(g):
    out = np.zeros(g.n_branch, bool)
    for e in range(g.n_branch):
        keep = np.arange(g.n_branch) != e
        a = sp.coo_matrix((np.ones(keep.sum()), (g.f_bus[keep], g.t_bus[keep])), shape=(g.n_bus, g.n_bus))
        out[e] = connected_components(a, directed=False)[0] > 1
    return out


@pytest.mark.parametrize("n,seed", [(30, 0), (120, 3)])
def test_bridges_brute_force(dpf, n, seed):
    g = gridgen.make_grid(n, seed, n_branch=int(1.2 * n))
    y = dpf.dpf_build_ybus_host(g)
    np.testing.assert_array_equal(dpf.dpf_ybus_bridges(y), _bridges_brute(g))


def _bad(g, **changes):
    h = g.copy()
    for k, v in changes.items():
        setattr(h, k, v)
    return h


def test_validation_errors(dpf):
    g = gridgen.config_grid("c1_30bus_fp64")
    cases = {
        -1: [
            _bad(g, bus_type=np.where(np.arange(g.n_bus) < 2, 2, g.bus_type).astype(np.uint8)),  # two slacks
            _bad(g, bus_type=np.where(g.bus_type == 2, 0, g.bus_type).astype(np.uint8)),          # none
            _bad(g, f_bus=np.where(np.arange(g.n_branch) == 3, g.n_bus, g.f_bus).astype(np.int32)),
            _bad(g, t_bus=np.where(np.arange(g.n_branch) == 3, g.f_bus, g.t_bus).astype(np.int32)),
            _bad(g, r=np.where(np.arange(g.n_branch) == 0, 0.0, g.r), x=np.where(np.arange(g.n_branch) == 0, 0.0, g.x)),
            _bad(g, p_spec=np.where(np.arange(g.n_bus) == 1, np.nan, g.p_spec)),
            _bad(g, tap=np.where(np.arange(g.n_branch) == 0, -1.0, g.tap)),
        ],
        -5: [
            _bad(g, shift=np.where(np.arange(g.n_branch) == 0, 0.1, 0.0)),
            _bad(g, f_bus=np.concatenate([g.f_bus, g.f_bus[:1]]), t_bus=np.concatenate([g.t_bus, g.t_bus[:1]]),
                 r=np.concatenate([g.r, g.r[:1]]), x=np.concatenate([g.x, g.x[:1]]),
                 b_ch=np.concatenate([g.b_ch, g.b_ch[:1]]), tap=np.concatenate([g.tap, g.tap[:1]]),
                 shift=np.zeros(g.n_branch + 1)),
        ],
    }
    for code, grids in cases.items():
        for h in grids:
            with pytest.raises(dpf.DPFError) as e:
                dpf.dpf_build_ybus_host(h)
            assert e.value.code == code, dpf.dpf_last_error()


def test_islands_need_one_slack_each(dpf):
    a = gridgen.make_grid(30, 1, load_scale=0.5)
    b = gridgen.make_grid(40, 2, load_scale=0.5)
    cat = gridgen.concat_grids([a, b])
    y = dpf.dpf_build_ybus_host(cat)  # two islands, one slack each
    assert y.n_bus == 70 and y.nnz == 70 + 2 * (a.n_branch + b.n_branch)
    bad = _bad(cat, bus_type=np.where(np.arange(70) == b.slack + 30, 0, cat.bus_type).astype(np.uint8))
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_build_ybus_host(bad)
    assert e.value.code == -1 and "island" in dpf.dpf_last_error()


def test_tap_zero_means_none(dpf):
    g = gridgen.config_grid("c1_30bus_fp64")
    h = _bad(g, tap=np.where(g.tap == 1.0, 0.0, g.tap))
    a = dpf.dpf_ybus_export(dpf.dpf_build_ybus_host(g))[2]
    b = dpf.dpf_ybus_export(dpf.dpf_build_ybus_host(h))[2]
    np.testing.assert_array_equal(a, b)


def test_default_opts_are_table2(dpf):
    t2 = json.load(open(os.path.join(ROOT, "tests", "golden", "hyperparameters.json")))["table2_static"]
    o = dpf.dpf_default_opts()
    assert (o.beta1, o.beta2) == tuple(t2["betas"])
    assert (o.factor, o.patience, o.threshold, o.cooldown) == (t2["factor"], t2["patience"], t2["threshold"], t2["cooldown"])
    assert o.max_iter == t2["max_iter"] and o.sched == dpf.SCHED_PLATEAU


def test_status_strings(dpf):
    for c in (0, -1, -2, -3, -4, -5, -6):
        assert dpf.dpf_status_str(c) and dpf.dpf_status_str(c) != "unknown status"


def test_c_program_builds_and_calls_the_library(dpf, tmp_path):
    """The header is plain C99: a C program compiles against it, links
    libdpf.so and calls host-only entry points (Y_bus build and validation,
    the Newton analysis, defaults, error reporting; no CUDA call)."""
    import shutil
    import subprocess
    from paper_2603_28203_gb300.build import LIB
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_dpf.c"
    src.write_text(r'''
#include <stdio.h>
#include "dpf.h"
int main(void) {
  /* two buses, one line: slack 0 feeding a PQ load at bus 1 */
  const uint8_t type[2] = {DPF_SLACK, DPF_PQ};
  const double p[2] = {0.0, -0.5}, q[2] = {0.0, -0.1}, vm[2] = {1.0, 1.0};
  const int32_t f[1] = {0}, t[1] = {1};
  const double r[1] = {0.01}, x[1] = {0.1}, bch[1] = {0.0}, tap[1] = {0.0};
  dpf_grid g = {2, 1, type, p, q, vm, 0.0, f, t, r, x, bch, tap, NULL};
  dpf_ybus* y = NULL;
  if (dpf_build_ybus_host(&g, &y) != DPF_OK) { printf("build: %s\n", dpf_last_error()); return 1; }
  int32_t n = 0, m = 0, nnz = 0;
  dpf_ybus_info(y, &n, &m, &nnz);
  int64_t npos = 0, npairs = 0;
  int32_t nl = 0;
  if (dpf_nr_analyze(y, &npos, &npairs, &nl) != DPF_OK) return 2;
  dpf_nr_opts o;
  dpf_nr_default_opts(&o);
  dpf_solve_opts so;
  dpf_default_opts(&so);
  g.n_branch = -1; /* invalid: must be rejected with a message, not a crash */
  dpf_ybus* bad = NULL;
  const int rc = dpf_build_ybus_host(&g, &bad);
  printf("%d %d %d %lld %lld %d %d %d %d\n", n, m, nnz, (long long)npos, (long long)npairs, nl, o.max_iter,
         so.max_iter, rc == DPF_E_INVALID);
  dpf_ybus_free(y);
  return 0;
}
''')
    exe = tmp_path / "use_dpf"
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I" + inc, str(src), "-o", str(exe), "-L" + libdir,
                    "-ldpf", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, m, nnz, npos, npairs, nl, nr_iter, dpf_iter, rejected = map(int, out)
    assert (n, m, nnz) == (2, 1, 4)
    assert (npos, npairs, nl) == (4, 1, 2)     # one elimination: the 2x2 pattern, one product, two levels
    assert nr_iter == 20 and dpf_iter == 1000 and rejected == 1


def test_newton_handle_needs_an_uploaded_ybus(dpf):
    """dpf_nr_create on a host-only Y_bus is refused (DPF_E_STATE) before any
    CUDA call; bad arguments are DPF_E_INVALID."""
    g = gridgen.config_grid("c1_30bus_fp64")
    y = dpf.dpf_build_ybus_host(g)
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_nr_create(y, 4)
    assert e.value.code == dpf._abi.DPF_E_STATE
    with pytest.raises(dpf.DPFError) as e:
        dpf.dpf_nr_create(y, 0)
    assert e.value.code == dpf._abi.DPF_E_INVALID


def test_binding_structs_match_the_header_layout(dpf, tmp_path):
    """The ctypes mirrors of the ABI structs (dpf_grid, dpf_batch,
    dpf_solve_opts, dpf_nr_opts) have the C compiler's size and the offset
    of every field, so a field added to the header without the binding (or
    in another order) fails here rather than shifting every later field."""
    import ctypes
    import shutil
    import subprocess
    from paper_2603_28203_gb300 import _abi
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"dpf_grid": _abi.DpfGrid, "dpf_batch": _abi.DpfBatch, "dpf_solve_opts": _abi.DpfSolveOpts,
               "dpf_nr_opts": _abi.DpfNrOpts}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dpf.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I" + inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, fname, v = line.split()
        got[(cname, fname)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
