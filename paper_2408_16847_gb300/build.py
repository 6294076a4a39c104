"""Build libtpcf.so (the C-ABI CUDA library) in-tree for sm_103a.

Every .cu file under csrc/ is compiled with nvcc for ``-gencode
arch=compute_103a,code=sm_103a``; map_inst.cu is compiled once per multipole
limit M = 0..TPCF_MAX_M.  Objects go to csrc/_build/, the library to the package
directory.  Translation units are compiled in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libtpcf.so")
BUILD = os.path.join(CSRC, "_build")
MAX_M = 16
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _units():
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.splitext(os.path.basename(src))[0]
        if base == "map_inst":
            for m in range(MAX_M + 1):
                units.append((src, os.path.join(BUILD, "%s_m%d.o" % (base, m)), ["-DTPCF_M=%d" % m]))
        else:
            units.append((src, os.path.join(BUILD, base + ".o"), []))
    return units


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link; returns the library path.  Skips work that is up to date."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= newest:
        return OUT
    nvcc = _nvcc()
    todo = []
    for src, obj, extra in _units():
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < newest:
            todo.append([nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        list(ex.map(run, todo))
    objs = [obj for _, obj, _ in _units()]
    tmp = OUT + ".%d.tmp" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
