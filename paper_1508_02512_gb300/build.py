"""Build the qmcfi CUDA library in-tree for sm_103a (GB300).

    python -m paper_1508_02512_gb300.build

compiles the csrc/ translation units in parallel with nvcc and links paper_1508_02512_gb300/_build/libqmcfi.so
against the shared CUDA runtime and NVRTC.  The device headers are also embedded into the library as string
literals (_build/qmc_jit_sources.h), because the generated evaluators (qmc_jit.cpp) are compiled at run time
together with them.
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
SOURCES = ["qmc_kernels.cu", "qmc_prepare.cpp", "qmc_pass.cpp", "qmc_context.cpp", "qmc_precision.cpp", "qmc_noalloc.cu", "qmc_jit.cpp"]
# the ahead-of-time kernels, one translation unit per sector dimension (built in parallel)
DIM_SOURCE = "qmc_kern_dim.cu"
DIMS = range(1, 7)
# device headers compiled again at run time with the generated evaluators: (C identifier, file)
EMBEDDED = [("qmc_src_qmcfi_h", os.path.join(ROOT, "include", "qmcfi.h")),
            ("qmc_src_qmc_internal_h", os.path.join(CSRC, "qmc_internal.h")),
            ("qmc_src_qmc_dev_cuh", os.path.join(CSRC, "qmc_dev.cuh"))]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the qmcfi library")


def _cuda_lib_dir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + [DIM_SOURCE, "qmc_internal.h", "qmc_host_internal.h", "qmc_device.cuh", "qmc_dev.cuh", "lattice_table.h"]]
    files.append(os.path.join(ROOT, "include", "qmcfi.h"))
    return files


def write_embedded(path: str) -> None:
    """C++ header holding each file of EMBEDDED as a raw string literal."""
    out = ["/* generated by paper_1508_02512_gb300/build.py: device headers for run-time compilation */", "#pragma once"]
    for name, f in EMBEDDED:
        text = open(f).read()
        if ')QMCSRC"' in text:
            raise RuntimeError(f"{f} contains the raw-string delimiter")
        out.append(f'static const char {name}[] = R"QMCSRC({text})QMCSRC";')
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        fh.write("\n".join(out) + "\n")
    os.replace(tmp, path)


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
    write_embedded(os.path.join(OUT, "qmc_jit_sources.h"))
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", OUT,
                     "-I", os.path.join(ROOT, "include")] + list(extra)
    tag = f"{os.getpid()}"
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.rsplit(".", 1)[0] + f".{tag}.o")
        objs.append(obj)
        cmds.append([nv, "-c", os.path.join(CSRC, src), "-o", obj] + common)
    for d in DIMS:
        obj = os.path.join(OUT, f"qmc_kern_d{d}.{tag}.o")
        objs.append(obj)
        cmds.append([nv, "-c", os.path.join(CSRC, DIM_SOURCE), "-o", obj, f"-DQMC_S={d}"] + common)

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
    run([nv, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-L", libdir, "-lnvrtc",
                                                     "-Xlinker", f"-rpath={libdir}"])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
