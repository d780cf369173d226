"""The GPU's Taylor subtraction for endpoint exponents alpha <= -2 (class-2 sectors, Sec. II Eq. 11 with p > 0),
checked on the host without a GPU.

The device functions (`point_integrand_taylor` with its series and jet helpers, the periodising transform and the
integer power) are cut out of csrc/qmc_dev.cuh as written and compiled with g++ through a shim (the table-driven
logarithm becomes the C library's).  Evaluated on packed sectors from qmc_prepare, they must give, point by point,
the weighted integrand of the oracle (oracle/taylor.py, written from Eq. 11 independently: truncated power series
by binomial expansion, where the kernel uses the power recurrence of a series).  Cases: massless bubbles with raised
propagator powers (alpha = -2 and -3, one expanded variable) and the massless box with one squared propagator
(alpha = -2 beside alpha = -1: jets in two variables), at random points and at points near the faces t_j = 0, where
the kernel takes remainders from their series.  The tolerance is the rounding of the subtracted form near the
switch to series, u / 0.02^(p+1) ~ 1e-11 for p = 2, with margin."""
import ctypes
import dataclasses
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import integrate as OI
from oracle import sectors as OS
from oracle import taylor as TT
from paper_1508_02512_gb300 import api
from paper_1508_02512_gb300 import tables as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_gen_build")
CSRC = os.path.join(ROOT, "paper_1508_02512_gb300", "csrc")

SHIM = r"""
#include <cmath>
#include <cstdint>
#include <cstring>
#include "qmc_internal.h"
using std::fma;
#define DEV static inline
#define __device__
#define __noinline__
static inline double __drcp_rn(double x) { return 1.0 / x; }
static inline double qlog(double x) { return std::log(x); }
struct Exps {
    int eU0, eU1, eF0, eF1;
};
"""

TAIL = r"""
template <int S>
static void run(const PackedSector *s, const PackedTerm *T, const double *x, int r, Exps ex, int maxm, double *out) {
    if (maxm == 0) point_integrand_taylor<S, 0>(*s, T, x, r, ex, out);
    else if (maxm == 2) point_integrand_taylor<S, 2>(*s, T, x, r, ex, out);
    else point_integrand_taylor<S, 4>(*s, T, x, r, ex, out);
}
extern "C" void h_taylor(const void *sec, const void *terms, int dim, const double *x, int r, int eU0, int eU1,
                         int eF0, int eF1, int maxm, double *out) {
    const PackedSector *s = static_cast<const PackedSector *>(sec);
    const PackedTerm *T = static_cast<const PackedTerm *>(terms);
    const Exps ex{eU0, eU1, eF0, eF1};
    switch (dim) {
        case 1: run<1>(s, T, x, r, ex, maxm, out); break;
        case 2: run<2>(s, T, x, r, ex, maxm, out); break;
        case 3: run<3>(s, T, x, r, ex, maxm, out); break;
        default: break;
    }
}
"""


def cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def lib():
    text = open(os.path.join(CSRC, "qmc_dev.cuh")).read()
    parts = [
        cut(text, "DEV double ipow(double v, int e) {", "/* ----"),
        cut(text, "/* ------------------------------------------------------------------ periodising transform",
            "/* ------------------------------------------------------------------ polynomials from shared memory"),
        cut(text, "/* ================================================================== endpoint exponents alpha <= -2",
            "template <int S, int MAXM>\n__global__"),
    ]
    os.makedirs(WORK, exist_ok=True)
    cpp = os.path.join(WORK, "taylor_host.cpp")
    so = os.path.join(WORK, "taylor_host.so")
    with open(cpp, "w") as f:
        f.write(SHIM + "\n".join(parts) + TAIL)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), cpp, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.h_taylor.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return L


def with_nu(topo, nus):
    return dataclasses.replace(topo, props=tuple(dataclasses.replace(p, nu=n) for p, n in zip(topo.props, nus)))


SECTOR_BYTES = 208
TERM = np.dtype([("c", "<f8"), ("e", "u1", (8,))])


def packed_sectors(prep):
    """(header fields, [(sector bytes, terms array)]) of a packed image, in table order"""
    buf = bytes(prep.packed)
    hdr = np.frombuffer(buf, dtype=np.int32, count=16)
    eU0, eU1, eF0, eF1 = (int(v) for v in hdr[6:10])
    sectors_off, terms_off = np.frombuffer(buf, dtype=np.int64, count=2, offset=_off_sectors(buf))
    out = {}
    for k in range(prep.info.n_sectors):
        rec = buf[sectors_off + k * SECTOR_BYTES: sectors_off + (k + 1) * SECTOR_BYTES]
        ints = np.frombuffer(rec, dtype=np.int32)
        term0, n_terms, orig = int(ints[24]), int(ints[25]), int(ints[26])
        terms = np.frombuffer(buf, dtype=TERM, count=n_terms, offset=terms_off + 16 * term0).copy()
        out[orig] = (rec, terms)
    return (eU0, eU1, eF0, eF1), [out[k] for k in range(prep.info.n_sectors)]


def _off_sectors(buf):
    # PackedHeader: 16 int32, pre[QMC_MAX_ORDERS + 4] doubles, 3 x 3 int32 class ranges, max_terms, n_terms_total,
    # then (8-byte aligned) sectors_off, terms_off
    off = 16 * 4 + 12 * 8 + 9 * 4 + 2 * 4
    return (off + 7) // 8 * 8


def points(dim, n, rng, near_face):
    x = rng.uniform(0.0, 1.0, (n, dim))
    if near_face:  # t = phi_3(x) < 0.02 needs x below ~0.15
        x[:, 0] = rng.uniform(1e-4, 0.15, n)
        if dim > 1:
            x[: n // 2, 1] = rng.uniform(1e-4, 0.15, n // 2)
    return x


def check(lib, topo, point, omin, omax, strategy, zero, seed):
    blob = T.compile_integral(topo, zero, strategy=strategy, allow_higher_poles=True)
    prep = api.prepare(blob, W.kinematics(topo, **point), omin, omax)
    secs = OS.decompose(topo, zero, strategy, allow_higher_poles=True)
    prob = OI.make_problem(topo, point, omin, omax, sectors=secs)
    e4, packed = packed_sectors(prep)
    assert len(packed) == len(prob.sectors) and tuple(e4) == tuple(prob.e4)
    maxm = 4 if prep.info.n_slots > 3 else (2 if prep.info.n_slots > 1 else 0)
    rng = np.random.default_rng(seed)
    worst, n_taylor = 0.0, 0
    for (rec, terms), sec in zip(packed, prob.sectors):
        if int(sec.A.min()) > -2:
            continue
        n_taylor += 1
        assert np.frombuffer(rec, dtype=np.int32)[27] == 1  # class-2 flag of the packed sector
        for near in (False, True):
            x = points(sec.dim, 200, rng, near)
            t, _, w = TT.transform(3, x)
            ref = np.prod(w, axis=1)[:, None] * TT.point_series(sec, e4, t, prob.kmax)
            got = np.zeros((len(x), 5))
            for i in range(len(x)):
                xi = np.ascontiguousarray(x[i])
                lib.h_taylor(rec, terms.ctypes.data, sec.dim, xi.ctypes.data, 3, *e4, maxm, got[i].ctypes.data)
            k = ref.shape[1]
            assert np.mean(np.abs(ref)) > 0  # (a slot may vanish identically: no pole of that order)
            scale = np.maximum(np.abs(ref), np.mean(np.abs(ref)))
            err = float(np.max(np.abs(got[:, :k] - ref) / scale))
            worst = max(worst, err)
    assert n_taylor > 0
    return worst


@pytest.mark.parametrize("nus", [(3, 1), (4, 1), (3, 2), (3, 3)])
def test_raised_power_bubble_points_match_the_oracle(lib, nus):
    worst = check(lib, with_nu(W.bubble(False), nus), dict(pp1=-2.0), -2, 2, "iterated", (), 3)
    print(f"bubble {nus}: worst |kernel - oracle| / |value| = {worst:.2e}")
    assert worst < 1e-9


@pytest.mark.parametrize("strategy", ["iterated", "geometric"])
def test_squared_propagator_box_points_match_the_oracle(lib, strategy):
    topo = W.box(False)
    dotted = with_nu(topo, (2, 1, 1, 1))
    pt = dict(s=-3.0, t=-2.0, pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)
    worst = check(lib, dotted, pt, -2, 0, strategy, ("pp1", "pp2", "pp3", "pp4"), 5)
    print(f"box with nu1 = 2 ({strategy}): worst |kernel - oracle| / |value| = {worst:.2e}")
    assert worst < 1e-9
