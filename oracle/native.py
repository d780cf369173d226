"""Build and load the oracle's plain-C integrand (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libqmc_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile qmc_oracle.c with gcc (-O2, OpenMP); returns the path of the shared library."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sector_args = [i, i, P(i), P(i), d, P(i), i, P(d), P(i), i, P(d), P(i), d, i, i]
        _lib.oracle_point.argtypes = sector_args + [P(d), P(d), i]
        _lib.oracle_point.restype = i
        _lib.oracle_lattice_sums.argtypes = sector_args + [i, ll, P(ll), P(d), i, i, P(d), P(d), P(d), P(ll)]
        _lib.oracle_lattice_sums.restype = i
        _lib.oracle_cbc_component.argtypes = [ll, P(d), P(ll), ll, i, P(d), P(d)]
        _lib.oracle_cbc_component.restype = i
    return _lib
