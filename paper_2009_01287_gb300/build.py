"""Build the C-ABI library libdgsc.so in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel, then linked
against the shared CUDA runtime.  No PyTorch headers are involved: the
library's interface is include/dg.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libdgsc.so")
INSPECT_LIB = os.path.join(OUT_DIR, "libdgsc_inspect.so")
# host-only translation units that also make up the inspection library
HOST_ONLY = ("basis.cpp", "mesh.cpp", "mesh3.cpp", "mesh_map.cpp", "load.cpp", "sparse.cpp", "host_operator.cpp",
             "precond_setup.cpp", "work_units.cpp",
             "precond3.cpp")
INSPECT_ONLY = ("inspect.cpp",)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _obj(src: str) -> str:
    return os.path.join(OUT_DIR, os.path.basename(src) + ".o")


def build(verbose: bool = False, extra=()) -> str:
    """Compile every source, link libdgsc.so and libdgsc_inspect.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    cmds = [[nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", _obj(src)] for src in sources()]
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
    for c, r in zip(cmds, res):
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(c) + "\n" + r.stdout + r.stderr)
    main = [_obj(s) for s in sources() if os.path.basename(s) not in INSPECT_ONLY]
    insp = [_obj(os.path.join(CSRC, f)) for f in HOST_ONLY + INSPECT_ONLY]
    for out, objs in ((LIB, main), (INSPECT_LIB, insp)):
        link = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", out, *objs]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: " + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=[a for a in sys.argv[1:] if a != "-v"]))
