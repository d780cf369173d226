"""The FP64 kernels' table-driven logarithm and arctangent (`qlog`, `qatan2` in csrc/qmc_dev.cuh), checked on the
host without a GPU.

Their source is cut out of qmc_dev.cuh as written and compiled with g++ through a shim for the few CUDA
intrinsics it uses (bit casts, the correctly rounded reciprocal, the FP32 division estimate, round-to-nearest
conversion); the shared-memory tables become a host struct filled by the same `logtab_init`.  Both functions
must stay within a few ulp of the C library's log and atan2 over arguments spanning the normal range, near 1,
across all four quadrants and on the axes, and must hand zero, negative, subnormal and non-finite arguments to
the library."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_gen_build")
SRC = os.path.join(ROOT, "paper_1508_02512_gb300", "csrc", "qmc_dev.cuh")

SHIM = r"""
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
using std::atan; using std::atan2; using std::copysign; using std::fabs; using std::fma; using std::log;
using std::max; using std::min;
#define DEV static inline
#define __shared__
#define QMC_PI 3.141592653589793
static struct { int x; } threadIdx = {0}, blockDim = {1};
static inline long long __double_as_longlong(double d) { long long b; std::memcpy(&b, &d, 8); return b; }
static inline double __longlong_as_double(long long b) { double d; std::memcpy(&d, &b, 8); return d; }
static inline double __drcp_rn(double x) { return 1.0 / x; }
static inline float __fdividef(float a, float b) { return a / b; }
static inline int __float2int_rn(float f) { return (int)std::nearbyint(f); }
"""

TAIL = r"""
extern "C" void h_init() { logtab_init(); }
extern "C" void h_qlog(const double *x, double *y, long n) { for (long i = 0; i < n; ++i) y[i] = qlog(x[i]); }
extern "C" void h_qatan2(const double *y, const double *x, double *r, long n) {
    for (long i = 0; i < n; ++i) r[i] = qatan2(y[i], x[i]);
}
"""


@pytest.fixture(scope="module")
def lib():
    text = open(SRC).read()
    m = re.search(r"/\* -+ table-driven FP64 log and atan2 \*/(.*?)/\* principal log \*/", text, re.S)
    assert m, "table-driven log/atan2 block not found in qmc_dev.cuh"
    os.makedirs(WORK, exist_ok=True)
    cpp = os.path.join(WORK, "device_math_host.cpp")
    so = os.path.join(WORK, "device_math_host.so")
    with open(cpp, "w") as f:
        f.write(SHIM + m.group(1) + TAIL)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", cpp, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.h_init()
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def qlog(L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    L.h_qlog(_ptr(x), _ptr(y), ctypes.c_long(len(x)))
    return y


def qatan2(L, y, x):
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty_like(x)
    L.h_qatan2(_ptr(y), _ptr(x), _ptr(r), ctypes.c_long(len(x)))
    return r


def test_qlog_matches_the_library_to_a_few_ulp(lib):
    rng = np.random.default_rng(5)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 300000),      # the normal range
                        1.0 + rng.uniform(-0.02, 0.02, 200000),       # near 1, both sides
                        1.0 + rng.uniform(-1e-9, 1e-9, 100000),
                        2.0 ** rng.integers(-60, 60, 100000) * (1.0 + rng.uniform(-1e-3, 1e-3, 100000)),
                        rng.uniform(0.5, 2.0, 200000)])
    got, ref = qlog(lib, x), np.log(x)
    nz = ref != 0.0
    rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
    assert rel.max() < 2e-15, (rel.max(), x[nz][np.argmax(rel)])
    assert np.all(got[~nz] == 0.0)
    assert qlog(lib, [1.0])[0] == 0.0


def test_qlog_special_arguments_follow_the_library(lib):
    x = np.array([0.0, -0.0, -1.0, 5e-324, 1e-310, np.inf, np.nan])
    with np.errstate(divide="ignore", invalid="ignore"):
        got, ref = qlog(lib, x), np.log(np.where(x < 0, np.nan, x))
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), (got, ref)


def test_qatan2_matches_the_library_in_every_quadrant(lib):
    rng = np.random.default_rng(6)
    n = 400000
    mag = 10.0 ** rng.uniform(-20, 20, (2, n))
    sgn = rng.choice([-1.0, 1.0], (2, n))
    y, x = sgn[0] * mag[0], sgn[1] * mag[1]
    # ratios near the grid points and the octant boundary |y| = |x|
    k = rng.integers(0, 129, 100000) / 128.0
    xs = rng.uniform(0.1, 10.0, 100000)
    y = np.concatenate([y, xs * (k + rng.uniform(-1e-6, 1e-6, 100000)), xs, -xs])
    x = np.concatenate([x, xs, xs * (1 + 1e-12), -xs * (1 - 1e-12)])
    got, ref = qatan2(lib, y, x), np.arctan2(y, x)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    assert rel.max() < 2e-15, (rel.max(), y[np.argmax(rel)], x[np.argmax(rel)])


def test_qatan2_axes_and_special_arguments_follow_the_library(lib):
    y = np.array([0.0, -0.0, 0.0, -0.0, 1.0, -1.0, 0.0, 1e-40, 1e40, np.inf, np.nan, 1.0, 3.0])
    x = np.array([1.0, 1.0, -1.0, -1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0, np.nan, -3.0])
    got, ref = qatan2(lib, y, x), np.arctan2(y, x)
    same = (np.abs(got - ref) <= 2e-16 * np.abs(ref)) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), (got, ref)
    assert math.copysign(1.0, qatan2(lib, [-0.0], [-1.0])[0]) == -1.0   # -pi for y = -0, x < 0
