"""Generated polynomial evaluators, checked on the host without a GPU.

The library writes, per family of sector tables, straight-line code for every sector's U~, F~ (at real t or at
the complex deformed point z of Eq. 14) and the gradient and Hessian polynomials of F~ (Eq. 14 and its
Jacobian).  Here that code is compiled for the host with a small shim and evaluated at random points against
the packed table's own terms (coefficient hi + lo, exponents) summed in FP64: every term must enter its own
polynomial exactly once with its exponents.  NVRTC compiles the same source for sm_103a without a device.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from paper_1508_02512_gb300 import _native as N
from paper_1508_02512_gb300 import api
from paper_1508_02512_gb300 import tables as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_gen_build")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1508_02512_gb300 import build
    build.build()
    N.lib()


# host mirrors of the packed image records (csrc/qmc_internal.h)
class PackedHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("n_sectors", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("loops", ctypes.c_int32), ("n_nu", ctypes.c_int32), ("n_props", ctypes.c_int32),
                ("eU0", ctypes.c_int32), ("eU1", ctypes.c_int32), ("eF0", ctypes.c_int32), ("eF1", ctypes.c_int32),
                ("order_min", ctypes.c_int32), ("order_max", ctypes.c_int32), ("kmax", ctypes.c_int32),
                ("n_slots", ctypes.c_int32), ("pre_low", ctypes.c_int32), ("n_pre", ctypes.c_int32),
                ("pre", ctypes.c_double * (N.QMC_MAX_ORDERS + 4)), ("class_begin", ctypes.c_int32 * 3),
                ("class_end", ctypes.c_int32 * 3), ("class_maxm", ctypes.c_int32 * 3), ("max_terms", ctypes.c_int32),
                ("n_terms_total", ctypes.c_int32), ("sectors_off", ctypes.c_int64), ("terms_off", ctypes.c_int64),
                ("total_bytes", ctypes.c_int64), ("flops_per_eval", ctypes.c_double),
                ("transc_per_eval", ctypes.c_double), ("n_deformed", ctypes.c_int32), ("n_negative", ctypes.c_int32),
                ("max_sigma", ctypes.c_int32), ("reserved", ctypes.c_int32), ("termsf_off", ctypes.c_int64),
                ("family", ctypes.c_uint64), ("reserved2", ctypes.c_int64)]


class PackedSector(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sigma", ctypes.c_int32), ("sing_mask", ctypes.c_int32),
                ("M", ctypes.c_int32), ("A", ctypes.c_int32 * 8), ("B", ctypes.c_int32 * 8), ("nU", ctypes.c_int32),
                ("nF", ctypes.c_int32), ("nG", ctypes.c_int32), ("nH", ctypes.c_int32), ("term0", ctypes.c_int32),
                ("n_terms", ctypes.c_int32), ("orig_index", ctypes.c_int32), ("taylor", ctypes.c_int32),
                ("gstart", ctypes.c_int16 * 8), ("hstart", ctypes.c_int16 * 24), ("D", ctypes.c_double),
                ("flops", ctypes.c_double), ("transc", ctypes.c_double), ("Df", ctypes.c_float),
                ("pad", ctypes.c_float)]


TERM_F = np.dtype([("hi", "<f4"), ("lo", "<f4"), ("e", "u1", (8,))])


def prepared(cfg, **point):
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    kin = W.kinematics(cfg.topology, **{**cfg.point, **point}) if point else cfg.kin
    return api.prepare(blob, kin, cfg.order_min, cfg.order_max)


def image(prep):
    buf = bytes(prep.packed)
    h = PackedHeader.from_buffer_copy(buf, 0)
    assert h.magic == 0x31504D51
    secs = [PackedSector.from_buffer_copy(buf, h.sectors_off + k * ctypes.sizeof(PackedSector))
            for k in range(h.n_sectors)]
    terms = np.frombuffer(buf, dtype=TERM_F, count=h.n_terms_total, offset=h.termsf_off)
    return h, secs, terms


def blocks(h, s):
    """term index ranges (within the sector) of U, F, every gradient and every Hessian polynomial"""
    S = h.dim
    bG = s.nU + s.nF
    bH = bG + s.nG
    g = [(bG + s.gstart[j], bG + s.gstart[j + 1]) for j in range(S)]
    hh = [(bH + s.hstart[p], bH + s.hstart[p + 1]) for p in range(S * (S + 1) // 2)]
    return (0, s.nU), (s.nU, s.nU + s.nF), g, hh


def test_family_source_depends_on_structure_only():
    pa, pb, pc = prepared(W.CONFIG1), prepared(W.CONFIG1, s=7.5, t=-2.5), prepared(W.CONFIG0)
    a, b, c = api.gen_source(pa), api.gen_source(pb), api.gen_source(pc)
    assert a == b and a != c
    assert api.gen_source(prepared(W.CONFIG1)) == a  # deterministic
    fa, fb, fc = (image(p)[0].family for p in (pa, pb, pc))
    assert fa == fb and fa != fc and fa != 0


def subsets(mask):
    """every subset Y of the singular variables (bit mask), the zeroed coordinates of the endpoint subtraction"""
    out, Y = [], 0
    while True:
        out.append(Y)
        Y = (Y - mask) & mask
        if Y == 0:
            return out


def own_subset(pre, h, k, Y):
    """the zeroed subset whose function serves Y: every subset has its own, except in the FP32 code of undeformed
    sectors (one function, Y = 0, evaluated with the zeroed coordinates)"""
    return 0 if (pre == "qg" and h.class_begin[0] <= k < h.class_end[0]) else Y


def vanishes(e, Y):
    """a term with a positive power of a zeroed coordinate is zero on that face"""
    return any(((Y >> j) & 1) and e[j] for j in range(len(e)))


@pytest.mark.parametrize("cfg", W.CONFIGS, ids=lambda c: c.name)
def test_every_term_enters_its_polynomial_once(cfg):
    """Per sector and zeroed subset Y: every term that does not vanish at t_Y = 0 enters its own polynomial exactly
    once, and no other term appears, in both precisions."""
    prep = prepared(cfg)
    h, secs, terms = image(prep)
    for pre, precision, head in (("qg", N.QMC_PREC_MIXED, "const float4"), ("qd", N.QMC_PREC_FP64, "const PackedTerm")):
        src = api.gen_source(prep, precision)
        funcs = {}
        for m in re.finditer(rf"\b({pre}_(?:ufr|gh|ufc)_(\d+)_(\d+))\({head}[^{{]*\{{(.*?)\n\}}", src, flags=re.S):
            funcs[m.group(1)] = m.group(4)
        check_terms(cfg, h, secs, terms, funcs, pre)


def check_terms(cfg, h, secs, terms, funcs, pre):
    for k, s in enumerate(secs):
        U, F, G, H = blocks(h, s)
        e = terms[s.term0: s.term0 + s.n_terms]["e"]
        for Y in sorted({own_subset(pre, h, k, Y) for Y in subsets(s.sing_mask)}):
            if h.class_begin[0] <= k < h.class_end[0]:
                groups = {f"{pre}_ufr_{k}_{Y}": [U, F]}
            else:
                groups = {f"{pre}_gh_{k}_{Y}": G + H, f"{pre}_ufc_{k}_{Y}": [U, F]}
            for name, ranges in groups.items():
                body = funcs[name]
                # (accumulator, term) of every statement that adds a term; a complex term is one statement (FP32,
                # packed over both lanes) or a statement on .x followed by one on .y (FP64)
                pairs = re.findall(r"a(\d+)(?:\.x|\.re)? (?:=|\+=) (?:fmaf?\(|cfma2c\(|rfma2[ch]\(|add2\(a\d+(?:\.re)?, "
                                   r"bc2\()?C\[(\d+)\]", body)
                got = {}
                for acc, term in pairs:
                    got.setdefault(int(term), set()).add(int(acc))
                want = {i: {a} for a, (lo, hi) in enumerate(ranges) for i in range(lo, hi) if not vanishes(e[i], Y)}
                assert got == want, (cfg.name, name)
                assert len(pairs) == len(want), (cfg.name, name)


SHIM = r"""
#include <math.h>
#define DEV static inline
#define __device__
#define __noinline__ static
#define __restrict__
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
struct c2 { float2 re, im; };
static inline float2 mk2(float x, float y) { float2 r; r.x = x; r.y = y; return r; }
static inline float2 bc2(float v) { return mk2(v, v); }
static inline float2 add2(float2 a, float2 b) { return mk2(a.x + b.x, a.y + b.y); }
static inline float2 mul2(float2 a, float2 b) { return mk2(a.x * b.x, a.y * b.y); }
static inline float2 fma2(float2 a, float2 b, float2 c) { return mk2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
static inline float2 neg2(float2 a) { return mk2(-a.x, -a.y); }
static inline c2 mkc2(float2 re, float2 im) { c2 r; r.re = re; r.im = im; return r; }
static inline c2 zero_c2() { return mkc2(bc2(0.f), bc2(0.f)); }
static inline c2 cmul2(c2 a, c2 b) { return mkc2(fma2(a.re, b.re, neg2(mul2(a.im, b.im))), fma2(a.re, b.im, mul2(a.im, b.re))); }
static inline float2 rfma2h(const float4 &c, float2 m, float2 a) { return fma2(mk2(c.x, c.y), m, a); }
static inline float2 rfma2c(const float4 &c, float2 m, float2 a) { return fma2(mk2(c.x, c.y), m, fma2(mk2(c.z, c.w), m, a)); }
static inline c2 cfma2c(const float4 &c, c2 m, c2 a) {
    return mkc2(fma2(mk2(c.x, c.y), m.re, fma2(mk2(c.z, c.w), m.re, a.re)), fma2(mk2(c.x, c.y), m.im, fma2(mk2(c.z, c.w), m.im, a.im)));
}
"""


def dispatch(h, secs, pre, R, Cx, term, ool):
    """extern "C" entry points h_ufr / h_gh / h_ufc(sector, Y, C, ...) switching over (sector, zeroed subset); ool:
    the source holds out-of-line functions with by-value results (large families), else inlined void functions."""
    S = h.dim
    NP = S * (S + 1) // 2
    ta = ", ".join(f"t[{j}]" for j in range(S))
    re_, im_ = ("re", "im") if pre == "qg" else ("x", "y")
    za = ", ".join(f"z[{j}].{re_}, z[{j}].{im_}" for j in range(S))
    Rr, GH, Cc = ("QgR", "QgGH", "QgC") if pre == "qg" else ("QdR", "QdGH", "QdC")
    ufr, gh, ufc = [], [], []
    for k in range(h.n_sectors):
        for Y in subsets(secs[k].sing_mask):
            n, lab = f"{k}_{own_subset(pre, h, k, Y)}", k * 64 + Y
            if h.class_begin[0] <= k < h.class_end[0]:
                ufr.append(f"case {lab}: {{ {Rr} r = {pre}_ufr_{n}(C, {ta}); U[0] = r.U; U[1] = r.F; return; }}"
                           if ool else f"case {lab}: {pre}_ufr_{n}(C, t, U[0], U[1]); return;")
            else:
                gh.append(f"case {lab}: {{ {GH} r = {pre}_gh_{n}(C, {ta}); for (int j = 0; j < {S}; ++j) g[j] = "
                          f"r.g[j]; for (int q = 0; q < {NP}; ++q) hh[q] = r.h[q]; return; }}"
                          if ool else f"case {lab}: {pre}_gh_{n}(C, t, g, hh); return;")
                ufc.append(f"case {lab}: {{ {Cc} r = {pre}_ufc_{n}(C, {za}); UF[0] = r.U; UF[1] = r.F; return; }}"
                           if ool else f"case {lab}: {pre}_ufc_{n}(C, z, UF[0], UF[1]); return;")
    return [f'extern "C" void h_ufr(int s, int Y, const {term} *C, const {R} *t, {R} *U) {{ switch (s * 64 + Y) {{ '
            + " ".join(ufr) + " } }",
            f'extern "C" void h_gh(int s, int Y, const {term} *C, const {R} *t, {R} *g, {R} *hh) {{ '
            f'switch (s * 64 + Y) {{ ' + " ".join(gh) + " } }",
            f'extern "C" void h_ufc(int s, int Y, const {term} *C, const {Cx} *z, {Cx} *UF) {{ switch (s * 64 + Y) {{ '
            + " ".join(ufc) + " } }"]


def generated_body(src, pol):
    """the generated per-sector functions (everything between the include and the evaluator struct)"""
    i0 = src.index('#include "qmc_dev.cuh"') + len('#include "qmc_dev.cuh"')
    return src[i0:src.index(f"struct {pol}")]


def host_harness(src, h, secs):
    """C++ source: the generated per-sector functions plus extern "C" entry points taking arrays"""
    body = generated_body(src, "QgPol")
    return "\n".join([SHIM, body] + dispatch(h, secs, "qg", "float2", "c2", "float4", "struct QgGH" in body))


def poly_value(terms, lo, hi, x):
    """FP64 sum over terms[lo:hi] of (hi + lo) * prod_j x_j^e_j (x real or complex)"""
    v = 0.0
    mag = 0.0
    for t in terms[lo:hi]:
        c = float(t["hi"]) + float(t["lo"])
        m = 1.0 + 0.0j if np.iscomplexobj(x) else 1.0
        for j in range(len(x)):
            m = m * x[j] ** int(t["e"][j])
        v += c * m
        mag += abs(c * m)
    return v, mag


@pytest.mark.parametrize("cfg", [W.CONFIG0, W.CONFIG1, W.CONFIG2], ids=lambda c: c.name)
def test_generated_functions_evaluate_the_table_polynomials(cfg):
    """Each generated FP32 function (per sector and zeroed subset; two points per call, one per lane) against the
    table's terms summed in FP64 at random points with the subset's coordinates zero.  The gradient and Hessian
    terms take the coefficient's FP32 part only, U and F the hi + lo pair: both agree with FP64 to FP32 rounding."""
    prep = prepared(cfg)
    h, secs, terms = image(prep)
    src = api.gen_source(prep)
    os.makedirs(WORK, exist_ok=True)
    cpp = os.path.join(WORK, f"gen_{cfg.name}.cpp")
    so = os.path.join(WORK, f"gen_{cfg.name}.so")
    open(cpp, "w").write(host_harness(src, h, secs))
    subprocess.check_call(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, cpp])
    L = ctypes.CDLL(so)
    S = h.dim
    NP = S * (S + 1) // 2
    rng = np.random.Generator(np.random.PCG64(11))
    fptr = ctypes.POINTER(ctypes.c_float)
    worst = 0.0
    for k, s in enumerate(secs):
        T_s = np.ascontiguousarray(terms[s.term0: s.term0 + s.n_terms])
        # coefficient slots as staged for the two-point path: (hi, hi, lo, lo)
        C4 = np.ascontiguousarray(np.stack([T_s["hi"], T_s["hi"], T_s["lo"], T_s["lo"]], -1).astype(np.float32))
        Cp = C4.ctypes.data_as(ctypes.c_void_p)
        U, F, G, H = blocks(h, s)
        for Y in subsets(s.sing_mask):
            t = rng.uniform(0.0, 1.0, (2, S)).astype(np.float32)   # lane a, lane b
            t[:, [j for j in range(S) if (Y >> j) & 1]] = 0.0
            t2 = np.ascontiguousarray(t.T)                          # float2 per variable
            tp = t2.ctypes.data_as(fptr)
            refs, got = [], []
            if h.class_begin[0] <= k < h.class_end[0]:
                outv = np.zeros((2, 2), np.float32)                 # U, F as float2
                L.h_ufr(k, Y, Cp, tp, outv.ctypes.data_as(fptr))
                for ln in range(2):
                    refs += [poly_value(T_s, *U, t[ln].astype(np.float64)), poly_value(T_s, *F, t[ln].astype(np.float64))]
                    got += [outv[0, ln], outv[1, ln]]
            else:
                g = np.zeros((S, 2), np.float32)
                hh = np.zeros((NP, 2), np.float32)
                L.h_gh(k, Y, Cp, tp, g.ctypes.data_as(fptr), hh.ctypes.data_as(fptr))
                zc = (t * (1 - 0.3j * rng.uniform(0, 1, (2, S)))).astype(np.complex64)
                # c2 per variable: (re lane a, re lane b, im lane a, im lane b)
                zf = np.ascontiguousarray(np.stack([zc.real.T, zc.imag.T], 1).reshape(S, 4).astype(np.float32))
                uf = np.zeros((2, 4), np.float32)
                L.h_ufc(k, Y, Cp, zf.ctypes.data_as(fptr), uf.ctypes.data_as(fptr))
                for ln in range(2):
                    tl = t[ln].astype(np.float64)
                    refs += [poly_value(T_s, lo, hi, tl) for lo, hi in G + H]
                    got += list(g[:, ln]) + list(hh[:, ln])
                    z64 = zc[ln].astype(np.complex128)
                    refs += [poly_value(T_s, *U, z64), poly_value(T_s, *F, z64)]
                    got += [complex(uf[0, ln], uf[0, 2 + ln]), complex(uf[1, ln], uf[1, 2 + ln])]
            for (rv, mag), gv in zip(refs, got):
                if mag == 0.0:
                    assert gv == 0, (k, Y)  # every term vanishes on this face
                    continue
                err = abs(complex(gv) - rv) / mag
                worst = max(worst, err)
    print(f"{cfg.name}: worst |generated FP32 - table FP64| / sum|terms| = {worst:.2e}")
    assert worst < 2e-6


SHIM64 = r"""
#include <math.h>
#define DEV static inline
#define __device__
#define __noinline__ static
#define __restrict__
struct cd { double x, y; };
static inline cd mk(double x, double y) { return cd{x, y}; }
static inline cd cmul(cd a, cd b) { return cd{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)}; }
struct PackedTerm { double c; unsigned char e[8]; };
"""


def host_harness64(src, h, secs):
    body = generated_body(src, "QdPol")
    return "\n".join([SHIM64, body] + dispatch(h, secs, "qd", "double", "cd", "PackedTerm", "struct QdGH" in body))


TERM_D = np.dtype([("c", "<f8"), ("e", "u1", (8,))])


@pytest.mark.parametrize("cfg", [W.CONFIG1, W.CONFIG2], ids=lambda c: c.name)
def test_generated_fp64_functions_evaluate_the_table_polynomials(cfg):
    prep = prepared(cfg)
    h, secs, _ = image(prep)
    terms = np.frombuffer(bytes(prep.packed), dtype=TERM_D, count=h.n_terms_total, offset=h.terms_off)
    src = api.gen_source(prep, N.QMC_PREC_FP64)
    os.makedirs(WORK, exist_ok=True)
    cpp = os.path.join(WORK, f"gen64_{cfg.name}.cpp")
    so = os.path.join(WORK, f"gen64_{cfg.name}.so")
    open(cpp, "w").write(host_harness64(src, h, secs))
    subprocess.check_call(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, cpp])
    L = ctypes.CDLL(so)
    S = h.dim
    NP = S * (S + 1) // 2
    rng = np.random.Generator(np.random.PCG64(12))
    dptr = ctypes.POINTER(ctypes.c_double)
    worst = 0.0

    def ref(T_s, lo, hi, x):
        v, mag = 0.0, 0.0
        for tt in T_s[lo:hi]:
            m = 1.0 + 0.0j if np.iscomplexobj(x) else 1.0
            for j in range(len(x)):
                m = m * x[j] ** int(tt["e"][j])
            v += tt["c"] * m
            mag += abs(tt["c"] * m)
        return v, mag

    for k, s in enumerate(secs):
        T_s = np.ascontiguousarray(terms[s.term0: s.term0 + s.n_terms])
        Cp = T_s.ctypes.data_as(ctypes.c_void_p)
        U, F, G, H = blocks(h, s)
        for Y in subsets(s.sing_mask):
            t = rng.uniform(0.0, 1.0, S)
            t[[j for j in range(S) if (Y >> j) & 1]] = 0.0
            tp = t.ctypes.data_as(dptr)
            if h.class_begin[0] <= k < h.class_end[0]:
                outv = np.zeros(2)
                L.h_ufr(k, Y, Cp, tp, outv.ctypes.data_as(dptr))
                refs, got = [ref(T_s, *U, t), ref(T_s, *F, t)], list(outv)
            else:
                g = np.zeros(S)
                hh = np.zeros(NP)
                L.h_gh(k, Y, Cp, tp, g.ctypes.data_as(dptr), hh.ctypes.data_as(dptr))
                refs = [ref(T_s, lo, hi, t) for lo, hi in G + H]
                got = list(g) + list(hh)
                zc = t * (1 - 0.3j * rng.uniform(0, 1, S))
                zf = np.ascontiguousarray(np.stack([zc.real, zc.imag], -1))
                uf = np.zeros(4)
                L.h_ufc(k, Y, Cp, zf.ctypes.data_as(dptr), uf.ctypes.data_as(dptr))
                refs += [ref(T_s, *U, zc), ref(T_s, *F, zc)]
                got += [complex(uf[0], uf[1]), complex(uf[2], uf[3])]
            for (rv, mag), gv in zip(refs, got):
                if mag == 0.0:
                    assert gv == 0, (k, Y)
                    continue
                worst = max(worst, abs(complex(gv) - rv) / mag)
    print(f"{cfg.name}: worst |generated FP64 - table| / sum|terms| = {worst:.2e}")
    assert worst < 1e-14


def test_nvrtc_compiles_generated_source_without_a_device():
    for precision in (N.QMC_PREC_MIXED, N.QMC_PREC_FP64):
        info = api.gen_compile(prepared(W.CONFIG1), load=False, precision=precision)
        assert info.cubin_bytes > 0 and info.source_bytes > 0 and info.compile_ms > 0


def test_disk_cache_of_compiled_modules(tmp_path, monkeypatch):
    """QMC_GEN_CACHE_DIR: the first compilation writes the cubin, the next one (another family member, another
    kinematic point) reads it instead of running NVRTC; other precisions and families get their own files."""
    monkeypatch.setenv("QMC_GEN_CACHE_DIR", str(tmp_path))
    a = api.gen_compile(prepared(W.CONFIG1), load=False)
    files = sorted(os.listdir(tmp_path))
    assert a.cached == 0 and len(files) == 1 and files[0].endswith(".cubin")
    b = api.gen_compile(prepared(W.CONFIG1, s=7.0, t=-2.5), load=False)
    assert b.cached == 2 and b.cubin_bytes == a.cubin_bytes and b.compile_ms < a.compile_ms
    c = api.gen_compile(prepared(W.CONFIG1), load=False, precision=N.QMC_PREC_FP64)
    assert c.cached == 0 and len(os.listdir(tmp_path)) == 2
    monkeypatch.delenv("QMC_GEN_CACHE_DIR")
    d = api.gen_compile(prepared(W.CONFIG1), load=False)
    assert d.cached == 0
