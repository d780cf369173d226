"""The island criterion of a mixed pass on the host, without a GPU: the device functions (`shift_floor`,
`shifted_index`, `island_key`, `island_bin` of csrc/qmc_dev.cuh) are cut out as written and compiled with g++
through a shim that maps the correctly rounded intrinsics to IEEE operations (-ffp-contract=off).  Their decisions
must equal, bit for bit, the criterion restated from its definition in numpy (tests/islands_ref.py), at random
lattice points and at the edges (k_j = 0, k_j = n - 1, shifts near 0 and 1, keys at the thresholds), and the key
must be the product of (k_j + 1) / n to FP32 rounding."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import islands_ref as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_gen_build")
CSRC = os.path.join(ROOT, "paper_1508_02512_gb300", "csrc")

SHIM = r"""
#include <cmath>
#include <cstdint>
#define DEV static inline
#define QMC_ISLAND_LEVELS 6
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __frcp_rn(float a) { return 1.0f / a; }
static inline float __uint2float_rn(uint32_t u) { return (float)u; }
using std::floor;
using std::fmaxf;
"""

TAIL = r"""
extern "C" void h_island(const uint32_t *r, const double *delta, int dim, uint32_t n, unsigned mask, int npts,
                         uint32_t *k_out, float *key_out, int *bin_out) {
    const float rn = island_rn(n);
    for (int p = 0; p < npts; ++p) {
        uint32_t k[6] = {0, 0, 0, 0, 0, 0};
        for (int j = 0; j < dim; ++j) k[j] = shifted_index(r[p * dim + j], shift_floor(delta[j], n), n);
        const float key = island_key<6>(k, mask, rn);
        for (int j = 0; j < dim; ++j) k_out[p * dim + j] = k[j];
        key_out[p] = key;
        bin_out[p] = island_bin(key);
    }
}
extern "C" int h_level(int code) { return island_level(code); }
"""


def cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def lib():
    text = open(os.path.join(CSRC, "qmc_dev.cuh")).read()
    part = cut(text, "DEV uint32_t shift_floor(double delta, uint32_t n) {", "DEV void kahan_add(")
    os.makedirs(WORK, exist_ok=True)
    cpp = os.path.join(WORK, "islands_host.cpp")
    so = os.path.join(WORK, "islands_host.so")
    with open(cpp, "w") as f:
        f.write(SHIM + part + TAIL)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", cpp, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.h_island.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint,
                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.h_level.argtypes = [ctypes.c_int]
    return L


def run(lib, idx, n, z, delta, mask):
    dim = len(z)
    r = np.stack([(np.asarray(idx, dtype=np.uint64) * np.uint64(zj)) % np.uint64(n) for zj in z], axis=1)
    r = np.ascontiguousarray(r.astype(np.uint32))
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
    npts = len(idx)
    k = np.zeros((npts, dim), dtype=np.uint32)
    key = np.zeros(npts, dtype=np.float32)
    b = np.zeros(npts, dtype=np.int32)
    lib.h_island(r.ctypes.data, d.ctypes.data, dim, n, mask, npts, k.ctypes.data, key.ctypes.data, b.ctypes.data)
    return k, key, b


@pytest.mark.parametrize("n,dim", [(1021, 4), (65521, 6), (1048573, 3), (16777213, 2)])
def test_device_criterion_equals_its_definition(lib, n, dim):
    rng = np.random.default_rng(n)
    z = rng.integers(1, n, dim)
    idx = np.concatenate([rng.integers(0, n, 20000), [0, 1, n - 1]])
    for trial in range(4):
        delta = rng.uniform(0.0, 1.0, dim)
        if trial == 1:
            delta[:] = 0.0
        if trial == 2:
            delta[:] = np.nextafter(1.0, 0.0)
        mask = int(rng.integers(1, 1 << dim))
        k, key, b = run(lib, idx, n, z, delta, mask)
        k_ref = R.shifted_indices(idx, n, z, delta)
        key_ref = R.keys(k_ref, mask, n)
        assert np.array_equal(k.astype(np.uint64), k_ref)
        assert np.array_equal(key, key_ref)
        assert np.array_equal(b, R.bins(key_ref))
        # the key is the product of (k_j + 1) / n to FP32 rounding (a few ulps), or the floor
        exact = np.ones(len(idx))
        for j in range(dim):
            if (mask >> j) & 1:
                exact *= (k_ref[:, j].astype(np.float64) + 1.0) / n
        big = exact > 1e-29
        assert np.all(np.abs(key[big] - exact[big]) <= 1e-6 * exact[big])
        assert np.all(key[~big] <= 1.1e-30)
        # k_j is floor(n x_j) of the shifted coordinate x_j = {i z_j / n + delta_j}
        x = np.mod(idx[:, None].astype(np.float64) * z[None, :] / n + delta[None, :], 1.0)
        off = np.abs(k_ref.astype(np.float64) - np.floor(n * x))
        assert np.all((off == 0) | (off == 1) | (off == n - 1))  # only where n x sits at an integer in FP64


def test_bins_at_the_thresholds(lib):
    """keys just below, at and above each level's threshold: a key below 10^-(L+1) (in FP32) is an island at
    level L; the bin counts the levels"""
    n = 1000
    for L in range(R.LEVELS):
        xi = R.XI[L]
        for key in (np.nextafter(xi, np.float32(0)), xi, np.nextafter(xi, np.float32(1))):
            b = int(R.bins(np.array([key], dtype=np.float32))[0])
            assert (b > L) == bool(key < xi)
    # one singular variable: k + 1 = 100 of n = 1000 gives the key 0.1f rounded as the device rounds it
    k, key, b = run(lib, np.array([0]), n, [1], [0.0999], 1)
    assert int(k[0, 0]) == 99 and key[0] == np.float32(np.float32(100) * (np.float32(1) / np.float32(1000)))
    assert int(b[0]) == int(R.bins(key)[0])


def test_precision_codes(lib):
    assert [lib.h_level(c) for c in range(-1, 10)] == [-1, -1, -1, 0, 1, 2, 3, 4, 5, -1, -1]
