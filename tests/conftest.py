import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libdpf")


def small_grid(n, seed, **kw):
    """A tiny synthetic grid for brute-force checks."""
    import gridgen
    n_branch = kw.pop("n_branch", n + 1 if n > 3 else n - 1)
    n_pv = kw.pop("n_pv", 1)
    return gridgen.make_grid(n, seed, n_branch=n_branch, n_pv=n_pv, **kw)
