"""Build the qmcfi CUDA library in-tree for sm_103a (GB300).

    python -m paper_1508_02512_gb300.build

compiles csrc/qmc_kernels.cu and csrc/qmc_host.cpp in parallel with nvcc and links
paper_1508_02512_gb300/_build/libqmcfi.so against the shared CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libqmcfi.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["qmc_kernels.cu", "qmc_host.cpp", "qmc_noalloc.cu"] + [f"qmc_kern_d{d}.cu" for d in range(1, 7)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the qmcfi library")


def _cuda_lib_dir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + ["qmc_internal.h", "qmc_device.cuh", "lattice_table.h"]]
    files.append(os.path.join(ROOT, "include", "qmcfi.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC,
                     "-I", os.path.join(ROOT, "include")] + list(extra)
    tag = f"{os.getpid()}"
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.rsplit(".", 1)[0] + f".{tag}.o")
        objs.append(obj)
        cmds.append([nv, "-c", os.path.join(CSRC, src), "-o", obj] + common)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {cmd[2]}")
        return p.stdout + p.stderr

    with ThreadPoolExecutor(len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + f".{tag}.tmp"
    libdir = _cuda_lib_dir(nv)
    run([nv, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-L", libdir,
                                                     "-Xlinker", f"-rpath={libdir}"])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
