"""Build libdpf.so in-tree for sm_103a (nvcc + g++, translation units compiled in parallel)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libdpf.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH") or "/usr/local/cuda"
    return home


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile the CUDA library; returns the path of libdpf.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    objs, cmds = [], []
    for src in ("dpf_api.cu", "dpf_noalloc.cu", "dpf_nr.cu"):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cu = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + INCLUDE, *os.environ.get("DPF_NVCC_FLAGS", "").split(), "-c", os.path.join(CSRC, src),
              "-o", obj]
        if ptxas_info:
            cu.insert(1, "-Xptxas=-v")
        objs.append(obj)
        cmds.append(cu)
    for src in ("dpf_host.cpp", "dpf_nr_symbolic.cpp"):
        host_o = os.path.join(OUT_DIR, src.replace(".cpp", ".o"))
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + INCLUDE,
                     "-I" + os.path.join(cuda, "include"), "-c", os.path.join(CSRC, src), "-o", host_o])
        objs.append(host_o)
    with ThreadPoolExecutor(len(cmds)) as ex:
        outs = list(ex.map(_run, cmds))
    tmp = LIB + ".tmp"
    outs.append(_run([nvcc, *ARCH, "-shared", *objs, "-o", tmp]))
    os.replace(tmp, LIB)
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
