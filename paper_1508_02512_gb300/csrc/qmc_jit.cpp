/*
 * Generated polynomial evaluators for the FP32 pass (run-time code generation with NVRTC).
 *
 * The sector integrand of Eqs. 7-9 and 14 is dominated by polynomial evaluation: U~, F~ and, for deformed
 * sectors, the S gradient and S(S+1)/2 Hessian polynomials of F~ (Eq. 14 and its Jacobian), at real t or at
 * the complex point z.  The table evaluator of the kernels walks the staged terms and decodes each term's
 * exponent bytes on every point, which costs far more integer instructions than the FP32 arithmetic itself.
 * The exponents of a sector table depend only on the topology and on the kinematic class (which invariants
 * vanish); the coefficients depend on the kinematic point.  So, once per family of tables, this file writes
 * every sector's monomials as straight-line CUDA: each distinct monomial is formed once, as its parent
 * monomial times one variable (the parent drops one power of the highest-index variable, so the factors are
 * multiplied in the same order as in the table evaluator), and every term adds coefficient x monomial to its
 * polynomial with the same two FMAs (coefficient hi + lo) as the table evaluator.  Coefficients are still read
 * from the sector's staged term table, so a new kinematic point of the same family reuses the compiled code.
 *
 * The generated source includes the kernel templates of qmc_dev.cuh (embedded into this library at build
 * time) and instantiates, for each sector class of the family, the persistent evaluation kernel with the
 * generated evaluator: FP32 (coefficients hi + lo, two FMAs per term) or FP64 (one FMA per term; the table
 * evaluator's repeated monomial products are what the FP64 pipe spends much of its time on).  The FP32/FP64
 * probe keeps the table evaluators: it only samples a few thousand points.  NVRTC compiles it for sm_103a; the cubin is loaded with the
 * runtime's library API and launched through its kernel handles.  Modules are cached per family for the life
 * of the process.
 */
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qmc_internal.h"
#include "qmc_jit_sources.h" /* generated at build time: the device headers as string literals */

namespace {

#define QMC_JIT_GENERATOR_VERSION 8u
#define QMC_GEN_INLINE_TERMS 2048 /* families with more terms get out-of-line sector functions */

const PackedHeader *hdr(const void *p) {
    const PackedHeader *h = static_cast<const PackedHeader *>(p);
    return (h && h->magic == QMC_PACK_MAGIC) ? h : nullptr;
}

int maxm_of(const PackedHeader *h, int c) { return h->class_maxm[c] == 0 ? 0 : (h->class_maxm[c] <= 2 ? 2 : 4); }

const PackedSector *sectors(const PackedHeader *h) {
    return reinterpret_cast<const PackedSector *>(reinterpret_cast<const unsigned char *>(h) + h->sectors_off);
}
const PackedTermF *terms_f(const PackedHeader *h) {
    return reinterpret_cast<const PackedTermF *>(reinterpret_cast<const unsigned char *>(h) + h->termsf_off);
}

/* ---------------------------------------------------------------- family key (what the generated code depends on) */
struct Fnv {
    uint64_t v = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            v ^= b[i];
            v *= 1099511628211ull;
        }
    }
    void add_i(int64_t x) { add(&x, sizeof(x)); }
};

uint64_t family_key(const PackedHeader *h) {
    Fnv f;
    f.add_i(QMC_JIT_GENERATOR_VERSION);
    f.add_i(h->dim);
    f.add_i(h->n_sectors);
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        f.add_i(h->class_begin[c]);
        f.add_i(h->class_end[c]);
        f.add_i(maxm_of(h, c));
    }
    const PackedSector *ps = sectors(h);
    const PackedTermF *tf = terms_f(h);
    for (int s = 0; s < h->n_sectors; ++s) {
        const PackedSector &p = ps[s];
        f.add_i(p.sing_mask);
        f.add_i(p.nU);
        f.add_i(p.nF);
        f.add_i(p.nG);
        f.add_i(p.nH);
        f.add(p.gstart, sizeof(p.gstart));
        f.add(p.hstart, sizeof(p.hstart));
        for (int k = 0; k < p.n_terms; ++k) f.add(tf[p.term0 + k].e, 8);
    }
    return f.v;
}

/* ---------------------------------------------------------------- code generation */
struct Entry {
    int acc;   /* accumulator (polynomial) */
    int term;  /* term index within the sector */
};

using Key = uint64_t; /* exponents packed 4 bits per variable */

Key key_of(const uint8_t *e, int S) {
    Key k = 0;
    for (int j = 0; j < S; ++j) k |= (Key)(e[j] & 15u) << (4 * j);
    return k;
}
int exp_of(Key k, int j) { return (int)((k >> (4 * j)) & 15u); }
int top_var(Key k, int S) {
    for (int j = S - 1; j >= 0; --j)
        if (exp_of(k, j)) return j;
    return -1;
}

/* Spelling of the generated code in one precision */
struct Lang {
    bool f64;
    bool x2;  /* two lattice points per thread, one per lane of the packed FP32 instructions */
    const char *real, *cplx, *mk, *cmul, *term, *pre, *pol, *body;
    const char *zero_r, *zero_c, *cre, *cim; /* zero values and the members of a complex value */
};
const Lang kF32{false, true, "float2", "c2", "mkc2", "cmul2", "float4", "qg", "QgPol", "eval_f32x2_body",
                "bc2(0.f)", "zero_c2()", "re", "im"};
const Lang kF64{true, false, "double", "cd", "mk", "cmul", "PackedTerm", "qd", "QdPol", "eval_f64_body",
                "0", "mk(0, 0)", "x", "y"};

struct PolySet {
    int S = 0;
    bool complex_ = false;
    bool hi_only = false; /* FP32: the coefficient's hi part only (see generate) */
    int n_acc = 0;
    std::vector<Entry> constants;
    std::map<Key, std::vector<Entry>> mono; /* every needed monomial (terms' and their parents), key -> terms */
};

/* zeroed: the subset Y of the endpoint subtraction whose coordinates are zero; terms with a positive power of
   one of them vanish there and are left out (adding c * 0 would change nothing) */
void add_term(PolySet &P, int acc, int term, const uint8_t *e, unsigned zeroed = 0) {
    for (int j = 0; j < P.S; ++j)
        if (((zeroed >> j) & 1u) && e[j]) return;
    Key k = key_of(e, P.S);
    if (k == 0) {
        P.constants.push_back({acc, term});
        return;
    }
    P.mono[k].push_back({acc, term});
    /* parents: drop one power of the highest variable until degree 1 */
    for (;;) {
        const int j = top_var(k, P.S);
        const Key par = k - ((Key)1 << (4 * j));
        if (par == 0 || P.mono.count(par)) break;
        P.mono[par];
        k = par;
    }
}

/* one term: FP32 adds (hi + lo) x m with two packed FMAs per component, for both lanes' points (coefficient
   slot (hi, hi, lo, lo)); FP64 one FMA */
void emit_fma(std::string &o, const Lang &L, const PolySet &P, const Entry &E, const std::string &m,
              const std::string &ind) {
    char b[256];
    if (L.x2) {
        std::snprintf(b, sizeof(b), "%sa%d = %s(C[%d], %s, a%d);\n", ind.c_str(), E.acc,
                      P.complex_ ? "cfma2c" : (P.hi_only ? "rfma2h" : "rfma2c"), E.term, m.c_str(), E.acc);
    } else if (L.f64) {
        if (!P.complex_)
            std::snprintf(b, sizeof(b), "%sa%d = fma(C[%d].c, %s, a%d);\n", ind.c_str(), E.acc, E.term, m.c_str(), E.acc);
        else
            std::snprintf(b, sizeof(b), "%sa%d.x = fma(C[%d].c, %s.x, a%d.x); a%d.y = fma(C[%d].c, %s.y, a%d.y);\n",
                          ind.c_str(), E.acc, E.term, m.c_str(), E.acc, E.acc, E.term, m.c_str(), E.acc);
    } else if (!P.complex_) {
        std::snprintf(b, sizeof(b), "%sa%d = fmaf(C[%d].hi, %s, fmaf(C[%d].lo, %s, a%d));\n", ind.c_str(), E.acc,
                      E.term, m.c_str(), E.term, m.c_str(), E.acc);
    } else {
        std::snprintf(b, sizeof(b), "%sa%d = cfma2f(C[%d].hi, C[%d].lo, %s, a%d);\n", ind.c_str(), E.acc, E.term,
                      E.term, m.c_str(), E.acc);
    }
    o += b;
}

void emit_node(std::string &o, const Lang &L, const PolySet &P, Key k, const std::string &parent, int depth, int &id) {
    const int j = top_var(k, P.S);
    const std::string ind(4 + 2 * depth, ' ');
    const std::string name = "m" + std::to_string(id++);
    const std::string var = (P.complex_ ? "z[" : "t[") + std::to_string(j) + "]";
    const std::string type = P.complex_ ? L.cplx : L.real;
    o += ind + "{\n";
    if (parent.empty())
        o += ind + "  const " + type + " " + name + " = " + var + ";\n";
    else if (P.complex_)
        o += ind + "  const " + type + " " + name + " = " + L.cmul + "(" + parent + ", " + var + ");\n";
    else if (L.x2)
        o += ind + "  const " + type + " " + name + " = mul2(" + parent + ", " + var + ");\n";
    else
        o += ind + "  const " + type + " " + name + " = " + parent + " * " + var + ";\n";
    for (const Entry &E : P.mono.at(k)) emit_fma(o, L, P, E, name, ind + "  ");
    for (int jj = j; jj < P.S; ++jj) {
        const Key ch = k + ((Key)1 << (4 * jj));
        if (exp_of(k, jj) >= 15) continue;
        if (P.mono.count(ch)) emit_node(o, L, P, ch, name, depth + 1, id);
    }
    o += ind + "}\n";
}

void emit_body(std::string &o, const Lang &L, const PolySet &P) {
    for (int a = 0; a < P.n_acc; ++a)
        o += P.complex_ ? std::string("    ") + L.cplx + " a" + std::to_string(a) + " = " + L.zero_c + ";\n"
                        : std::string("    ") + L.real + " a" + std::to_string(a) + " = " + L.zero_r + ";\n";
    for (const Entry &E : P.constants) {
        char b[160];
        if (L.x2 && P.hi_only)
            std::snprintf(b, sizeof(b), "    a%d = add2(a%d, bc2(C[%d].x));\n", E.acc, E.acc, E.term);
        else if (L.x2)
            std::snprintf(b, sizeof(b), P.complex_ ? "    a%d.re = add2(a%d.re, bc2(C[%d].x + C[%d].z));\n"
                                                   : "    a%d = add2(a%d, bc2(C[%d].x + C[%d].z));\n",
                          E.acc, E.acc, E.term, E.term);
        else if (L.f64)
            std::snprintf(b, sizeof(b), P.complex_ ? "    a%d.x += C[%d].c;\n" : "    a%d += C[%d].c;\n", E.acc, E.term);
        else
            std::snprintf(b, sizeof(b), P.complex_ ? "    a%d.x += C[%d].hi + C[%d].lo;\n" : "    a%d += C[%d].hi + C[%d].lo;\n",
                          E.acc, E.term, E.term);
        o += b;
    }
    int id = 0;
    for (int j = 0; j < P.S; ++j) {
        const Key k = (Key)1 << (4 * j);
        if (P.mono.count(k)) emit_node(o, L, P, k, "", 0, id);
    }
}

/* source of one family in one precision: per-sector functions, the evaluator and the kernels of every class */
std::string generate(const PackedHeader *h, const Lang &L) {
    const int S = h->dim;
    const int NP = S * (S + 1) / 2;
    const PackedSector *ps = sectors(h);
    const PackedTermF *tf = terms_f(h); /* exponents (the FP64 terms carry the same ones, in the same order) */
    const std::string R = L.real, Cx = L.cplx, TT = L.term, pre = L.pre;
    std::string o;
    o.reserve(1 << 20);
    char b[512];
    std::snprintf(b, sizeof(b),
                  "/* generated: %s polynomial evaluators of one family of %d-dimensional sector tables (%d sectors) */\n"
                  "#include \"qmc_dev.cuh\"\n\n",
                  L.f64 ? "FP64" : "FP32", S, h->n_sectors);
    o += b;
    std::vector<int> cls(h->n_sectors, -1);
    for (int c = 0; c < QMC_N_CLASSES; ++c)
        for (int s = h->class_begin[c]; s < h->class_end[c]; ++s) cls[s] = c;
    /* Small families are inlined into the kernels.  Large ones get one non-inlined function per sector and
       polynomial set (arguments and results by value, so they stay in registers): ptxas then compiles each
       function on its own, which keeps compilation time linear in the family size. */
    const bool out_of_line = h->n_terms_total > QMC_GEN_INLINE_TERMS;
    std::string targs, tvals, zargs, zvals, tcall, zcall;
    for (int j = 0; j < S; ++j) {
        const std::string J = std::to_string(j);
        targs += ", " + R + " t" + J;
        tvals += (j ? ", t" : "t") + J;
        zargs += ", " + R + " z" + J + "r, " + R + " z" + J + "i";
        zvals += std::string(j ? ", " : "") + L.mk + "(z" + J + "r, z" + J + "i)";
        tcall += ", t[" + J + "]";
        zcall += ", z[" + J + "]." + L.cre + ", z[" + J + "]." + L.cim;
    }
    const std::string SR = pre == "qg" ? "QgR" : "QdR", SC = pre == "qg" ? "QgC" : "QdC", SGH = pre == "qg" ? "QgGH" : "QdGH";
    if (out_of_line) {
        o += "struct " + SR + " { " + R + " U, F; };\nstruct " + SC + " { " + Cx + " U, F; };\nstruct " + SGH + " { " + R +
             " g[" + std::to_string(S) + "], h[" + std::to_string(NP) + "]; };\n\n";
    }
    /* one function per sector, polynomial set and zeroed subset Y of the sector's singular variables (Y = 0: no
       coordinate zeroed); the name carries both: <pre>_<kind>_<sector>_<Y> */
    auto head = [&](const char *kind, int s, unsigned Y) {
        const std::string n = std::to_string(s) + "_" + std::to_string(Y);
        const std::string C = "(const " + TT + " *__restrict__ C";
        if (!out_of_line) {
            if (!std::strcmp(kind, "ufr")) return "DEV void " + pre + "_ufr_" + n + C + ", const " + R + " *t, " + R + " &U, " + R + " &F) {\n";
            if (!std::strcmp(kind, "gh")) return "DEV void " + pre + "_gh_" + n + C + ", const " + R + " *t, " + R + " *g, " + R + " *h) {\n";
            return "DEV void " + pre + "_ufc_" + n + C + ", const " + Cx + " *z, " + Cx + " &U, " + Cx + " &F) {\n";
        }
        if (!std::strcmp(kind, "ufr"))
            return "__device__ __noinline__ " + SR + " " + pre + "_ufr_" + n + C + targs + ") {\n    const " + R + " t[] = {" + tvals + "};\n";
        if (!std::strcmp(kind, "gh"))
            return "__device__ __noinline__ " + SGH + " " + pre + "_gh_" + n + C + targs + ") {\n    const " + R + " t[] = {" + tvals + "};\n";
        return "__device__ __noinline__ " + SC + " " + pre + "_ufc_" + n + C + zargs + ") {\n    const " + Cx + " z[] = {" + zvals + "};\n";
    };
    /* the zeroed subsets of a sector that get code of their own: every subset of its singular variables, except in
       the FP32 code of undeformed sectors, where one function serves every subset (measured: the FP64 passes gain
       10-12 % from leaving out the terms that vanish, the deformed FP32 class 8 %, while the undeformed FP32 class of
       the four-pole double box, up to 16 subsets of small polynomials, loses 2 % to instruction fetch) */
    auto per_subset = [&](int s) { return L.f64 || cls[s] == 1; };
    auto subsets = [&](int s) {
        std::vector<unsigned> out;
        const unsigned mask = per_subset(s) ? (unsigned)ps[s].sing_mask : 0u;
        unsigned Y = 0;
        do {
            out.push_back(Y);
            Y = (Y - mask) & mask;
        } while (Y != 0);
        return out;
    };
    for (int s = 0; s < h->n_sectors; ++s) {
        const PackedSector &p = ps[s];
        const PackedTermF *T = tf + p.term0;
        for (const unsigned Y : subsets(s)) {
            if (cls[s] == 0) {
                PolySet P;
                P.S = S;
                P.n_acc = 2;
                for (int k = 0; k < p.nU; ++k) add_term(P, 0, k, T[k].e, Y);
                for (int k = 0; k < p.nF; ++k) add_term(P, 1, p.nU + k, T[p.nU + k].e, Y);
                o += head("ufr", s, Y);
                emit_body(o, L, P);
                o += out_of_line ? "    return " + SR + "{a0, a1};\n}\n" : "    U = a0;\n    F = a1;\n}\n";
            } else if (cls[s] == 1) {
                PolySet P;
                P.S = S;
                P.n_acc = S + NP;
                /* the gradient and Hessian of F~ only shape the contour (Eq. 14) and its Jacobian: in FP32 their
                   coefficients enter rounded to FP32 (hi), so the Jacobian matches the deformation applied to FP32
                   rounding, which bounds that path anyway (measured: 5 % faster, FP32 error unchanged) */
                P.hi_only = !L.f64;
                const int bG = p.nU + p.nF, bH = bG + p.nG;
                for (int j = 0; j < S; ++j)
                    for (int k = bG + p.gstart[j]; k < bG + p.gstart[j + 1]; ++k) add_term(P, j, k, T[k].e, Y);
                for (int q = 0; q < NP; ++q)
                    for (int k = bH + p.hstart[q]; k < bH + p.hstart[q + 1]; ++k) add_term(P, S + q, k, T[k].e, Y);
                o += head("gh", s, Y);
                emit_body(o, L, P);
                const char *gv = out_of_line ? "    r.g[" : "    g[";
                const char *hv = out_of_line ? "    r.h[" : "    h[";
                if (out_of_line) o += "    " + SGH + " r;\n";
                for (int j = 0; j < S; ++j) o += gv + std::to_string(j) + "] = a" + std::to_string(j) + ";\n";
                for (int q = 0; q < NP; ++q) o += hv + std::to_string(q) + "] = a" + std::to_string(S + q) + ";\n";
                o += out_of_line ? "    return r;\n}\n" : "}\n";
                PolySet Q;
                Q.S = S;
                Q.complex_ = true;
                Q.n_acc = 2;
                for (int k = 0; k < p.nU; ++k) add_term(Q, 0, k, T[k].e, Y);
                for (int k = 0; k < p.nF; ++k) add_term(Q, 1, p.nU + k, T[p.nU + k].e, Y);
                o += head("ufc", s, Y);
                emit_body(o, L, Q);
                o += out_of_line ? "    return " + SC + "{a0, a1};\n}\n" : "    U = a0;\n    F = a1;\n}\n";
            }
        }
    }
    /* the evaluator: a warp-uniform switch over (packed sector index, zeroed subset) */
    const std::string Pol = L.pol;
    o += "\nstruct " + Pol + " {\n    const " + TT + " *T;\n    int sec;\n    DEV static " + Pol + " make(const " + TT +
         " *T, const PackedSector &, int psec) { return " + Pol + "{T, psec}; }\n";
    /* case labels: sector * 64 + Y; a sector with one function for all subsets gets the labels of every Y */
    auto labels = [&](int s, unsigned Y) {
        if (per_subset(s) || ps[s].sing_mask == 0) return "case " + std::to_string(s * 64 + (int)Y) + ":";
        std::string out;
        const unsigned mask = (unsigned)ps[s].sing_mask;
        unsigned Z = 0;
        do {
            out += (out.empty() ? "case " : " case ") + std::to_string(s * 64 + (int)Z) + ":";
            Z = (Z - mask) & mask;
        } while (Z != 0);
        return out;
    };
    const std::string sel = "sec * 64 + (int)Y";
    o += "    DEV void UFr(unsigned Y, const " + R + " *t, " + R + " &U, " + R + " &F) const {\n        switch (" + sel + ") {\n";
    for (int s = 0; s < h->n_sectors; ++s)
        if (cls[s] == 0)
            for (const unsigned Y : subsets(s)) {
                const std::string n = std::to_string(s) + "_" + std::to_string(Y);
                o += out_of_line ? "        " + labels(s, Y) + " { const " + SR + " r = " + pre + "_ufr_" + n + "(T" + tcall + "); U = r.U; F = r.F; return; }\n"
                                 : "        " + labels(s, Y) + " " + pre + "_ufr_" + n + "(T, t, U, F); return;\n";
            }
    o += std::string("        default: U = ") + L.zero_r + "; F = " + L.zero_r + ";\n        }\n    }\n";
    o += "    DEV void GH(unsigned Y, const " + R + " *t, " + R + " *g, " + R + " *h) const {\n        switch (" + sel + ") {\n";
    for (int s = 0; s < h->n_sectors; ++s)
        if (cls[s] == 1)
            for (const unsigned Y : subsets(s)) {
                const std::string n = std::to_string(s) + "_" + std::to_string(Y);
                o += out_of_line ? "        " + labels(s, Y) + " { const " + SGH + " r = " + pre + "_gh_" + n + "(T" + tcall +
                                       "); for (int j = 0; j < " + std::to_string(S) + "; ++j) g[j] = r.g[j]; for (int q = 0; q < " +
                                       std::to_string(NP) + "; ++q) h[q] = r.h[q]; return; }\n"
                                 : "        " + labels(s, Y) + " " + pre + "_gh_" + n + "(T, t, g, h); return;\n";
            }
    std::snprintf(b, sizeof(b),
                  "        default:\n            for (int j = 0; j < %d; ++j) g[j] = %s;\n"
                  "            for (int q = 0; q < %d; ++q) h[q] = %s;\n        }\n    }\n",
                  S, L.zero_r, NP, L.zero_r);
    o += b;
    o += "    DEV void UFc(unsigned Y, const " + Cx + " *z, bool, " + Cx + " &U, " + Cx + " &F) const {\n        switch (" + sel + ") {\n";
    for (int s = 0; s < h->n_sectors; ++s)
        if (cls[s] == 1)
            for (const unsigned Y : subsets(s)) {
                const std::string n = std::to_string(s) + "_" + std::to_string(Y);
                o += out_of_line ? "        " + labels(s, Y) + " { const " + SC + " r = " + pre + "_ufc_" + n + "(T" + zcall + "); U = r.U; F = r.F; return; }\n"
                                 : "        " + labels(s, Y) + " " + pre + "_ufc_" + n + "(T, z, U, F); return;\n";
            }
    o += std::string("        default: U = ") + L.zero_c + "; F = " + L.zero_c + ";\n        }\n    }\n};\n\n";
    for (int c = 0; c < 2; ++c) { /* class 2 (alpha <= -2) runs the ahead-of-time FP64 kernel */
        if (h->class_end[c] <= h->class_begin[c]) continue;
        const char *def = c == 1 ? "true" : "false";
        const int mm = maxm_of(h, c);
        /* FP32, 5- and 6-dimensional sectors, 128-thread blocks: the deformed class at 3 blocks per SM (<= 170
           registers, no spills; 13 % faster than 2 blocks, 3 % faster than 4, which spills); the undeformed class
           at 4 blocks per SM (17 % faster than 3 on the four-pole sectors of the massless double box, which are
           latency-bound).  FP32 below 5 dimensions: registers capped for 768 threads per SM (the massive box
           pass is 18 % faster than with the compiler's 125 registers and 512 threads).  FP64 keeps 256. */
        const std::string lb = L.f64 ? "__launch_bounds__(256)"
                               : qmc_gen_max_block(S) == 128
                                   ? (c == 1 ? "__launch_bounds__(128, 3)" : "__launch_bounds__(128, 4)")
                                   : "__launch_bounds__(256, 3)";
        std::snprintf(b, sizeof(b),
                      "extern \"C\" __global__ void %s %s_eval_c%d(const __grid_constant__ JobTable jt) {\n"
                      "    %s<%d, %s, %d, %s>(jt);\n}\n",
                      lb.c_str(), pre.c_str(), c, L.body, S, def, mm, L.pol);
        o += b;
    }
    return o;
}

/* ---------------------------------------------------------------- NVRTC */
const char *k_stdint =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long uint64_t; typedef long intptr_t; typedef unsigned long uintptr_t;\n";
const char *k_stddef = "#pragma once\n";

struct Compiled {
    std::vector<char> cubin;
    std::string log;
    double ms = 0.0;
    size_t source_bytes = 0;
    bool from_disk = false;
};

int compile(const std::string &src, Compiled &out) {
    const auto t0 = std::chrono::steady_clock::now();
    const char *headers[] = {k_stdint, k_stddef, qmc_src_qmcfi_h, qmc_src_qmc_internal_h, qmc_src_qmc_dev_cuh};
    const char *names[] = {"stdint.h", "stddef.h", "../../include/qmcfi.h", "qmc_internal.h", "qmc_dev.cuh"};
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "qmc_generated.cu", 5, headers, names) != NVRTC_SUCCESS)
        return QMC_ERR_CODEGEN;
    /* -default-device: the C-ABI declarations of the included headers become (unused) device declarations */
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-DQMC_GENERATED=1"};
    const nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    if (ls > 1) {
        out.log.resize(ls);
        nvrtcGetProgramLog(prog, &out.log[0]);
    }
    int rc = QMC_OK;
    if (r != NVRTC_SUCCESS) {
        rc = QMC_ERR_CODEGEN;
    } else {
        size_t cs = 0;
        if (nvrtcGetCUBINSize(prog, &cs) != NVRTC_SUCCESS || cs == 0) {
            rc = QMC_ERR_CODEGEN;
        } else {
            out.cubin.resize(cs);
            if (nvrtcGetCUBIN(prog, out.cubin.data()) != NVRTC_SUCCESS) rc = QMC_ERR_CODEGEN;
        }
    }
    nvrtcDestroyProgram(&prog);
    out.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    out.source_bytes = src.size();
    if (rc) std::fprintf(stderr, "qmcfi: generated-code compilation failed:\n%.4000s\n", out.log.c_str());
    return rc;
}

/* ---------------------------------------------------------------- module cache */
struct Module {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t eval[QMC_N_CLASSES] = {};
    bool from_disk = false;
    double compile_ms = 0.0;
    int64_t source_bytes = 0, cubin_bytes = 0;
};

/* Per-family state.  Compilation runs outside the lock (other families' lookups and launches go on); callers
   of the same family wait on the condition variable, or, in the background form, return QMC_PENDING.  The
   state is never destroyed (a background compilation may still run while the process exits). */
enum { GEN_NONE = 0, GEN_COMPILING, GEN_READY, GEN_FAILED };
struct Slot {
    int state = GEN_NONE;
    int rc = QMC_OK;
    std::unique_ptr<Module> mod;
};
struct Cache {
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, Slot> slots;
};
Cache &cache() {
    static Cache *c = new Cache();
    return *c;
}

const Lang &lang_of(int precision) { return precision == QMC_PREC_FP64 ? kF64 : kF32; }

/* cache key: the family and the precision of the generated evaluator */
uint64_t module_key(const PackedHeader *h, int precision) {
    return family_key(h) ^ (precision == QMC_PREC_FP64 ? 0x9E3779B97F4A7C15ull : 0ull);
}

/* compile and load (no lock held) */
/* ---------------------------------------------------------------- optional disk cache of compiled modules
 * With QMC_GEN_CACHE_DIR set, cubins are kept in that directory under a name that covers everything they
 * depend on: the module key (family, precision), the generator version, the embedded device sources and the
 * NVRTC version.  A file is written to a temporary name and renamed, so concurrent processes never read a
 * partial cubin. */
uint64_t sources_hash() {
    Fnv f;
    for (const char *s : {qmc_src_qmcfi_h, qmc_src_qmc_internal_h, qmc_src_qmc_dev_cuh}) f.add(s, std::strlen(s));
    int maj = 0, mnr = 0;
    nvrtcVersion(&maj, &mnr);
    f.add_i(maj * 1000 + mnr);
    f.add_i(QMC_JIT_GENERATOR_VERSION);
    return f.v;
}

std::string cache_path(uint64_t key) {
    const char *dir = std::getenv("QMC_GEN_CACHE_DIR");
    if (!dir || !*dir) return std::string();
    char name[96];
    std::snprintf(name, sizeof(name), "/qmcfi-%016llx-%016llx.cubin", (unsigned long long)key,
                  (unsigned long long)sources_hash());
    return std::string(dir) + name;
}

/* compile the family's source, or read its cubin from the disk cache */
int compile_cached(const PackedHeader *h, int precision, Compiled &cc) {
    const auto t0 = std::chrono::steady_clock::now();
    const std::string path = cache_path(module_key(h, precision));
    if (!path.empty()) {
        if (FILE *f = std::fopen(path.c_str(), "rb")) {
            std::fseek(f, 0, SEEK_END);
            const long sz = std::ftell(f);
            std::fseek(f, 0, SEEK_SET);
            if (sz > 0) {
                cc.cubin.resize((size_t)sz);
                if (std::fread(cc.cubin.data(), 1, (size_t)sz, f) == (size_t)sz) {
                    std::fclose(f);
                    cc.from_disk = true;
                    cc.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                    return QMC_OK;
                }
            }
            std::fclose(f);
            cc.cubin.clear();
        }
    }
    const int rc = compile(generate(h, lang_of(precision)), cc);
    if (!rc && !path.empty()) {
        const std::string tmp =
            path + "." + std::to_string((unsigned long long)std::hash<std::thread::id>()(std::this_thread::get_id())) +
            ".tmp";
        if (FILE *f = std::fopen(tmp.c_str(), "wb")) {
            const bool ok = std::fwrite(cc.cubin.data(), 1, cc.cubin.size(), f) == cc.cubin.size();
            std::fclose(f);
            if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
        }
    }
    return rc;
}

int build_module(const PackedHeader *h, int precision, std::unique_ptr<Module> &out) {
    Compiled cc;
    int rc = compile_cached(h, precision, cc);
    if (rc) return rc;
    std::unique_ptr<Module> m(new Module());
    if (cudaLibraryLoadData(&m->lib, cc.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess)
        return QMC_ERR_CUDA;
    for (int c = 0; c < 2; ++c) {
        if (h->class_end[c] <= h->class_begin[c]) continue;
        const std::string e = std::string(lang_of(precision).pre) + "_eval_c" + std::to_string(c);
        if (cudaLibraryGetKernel(&m->eval[c], m->lib, e.c_str()) != cudaSuccess) {
            cudaLibraryUnload(m->lib);
            return QMC_ERR_CUDA;
        }
    }
    m->compile_ms = cc.ms;
    m->from_disk = cc.from_disk;
    m->source_bytes = (int64_t)cc.source_bytes;
    m->cubin_bytes = (int64_t)cc.cubin.size();
    out = std::move(m);
    return QMC_OK;
}

void finish_slot(uint64_t key, int rc, std::unique_ptr<Module> m) {
    Cache &C = cache();
    {
        std::lock_guard<std::mutex> g(C.mu);
        Slot &s = C.slots[key];
        s.rc = rc;
        s.state = rc ? GEN_FAILED : GEN_READY;
        if (!rc) s.mod = std::move(m);
    }
    C.cv.notify_all();
}

/* mode 0: compile here and wait; mode 1: start a background compilation and return QMC_PENDING until ready */
int get_module(const PackedHeader *h, int precision, const Module **out, bool *was_cached, int mode = 0,
               int device = 0) {
    const uint64_t key = module_key(h, precision);
    Cache &C = cache();
    std::unique_lock<std::mutex> lk(C.mu);
    Slot &s = C.slots[key];
    if (was_cached) *was_cached = s.state == GEN_READY;
    if (s.state == GEN_COMPILING) {
        if (mode == 1) return QMC_PENDING;
        C.cv.wait(lk, [&] { return s.state != GEN_COMPILING; });
    }
    if (s.state == GEN_READY) {
        *out = s.mod.get();
        return QMC_OK;
    }
    if (s.state == GEN_FAILED) return s.rc;
    s.state = GEN_COMPILING;
    lk.unlock();
    if (mode == 1) {
        std::vector<unsigned char> img(reinterpret_cast<const unsigned char *>(h),
                                       reinterpret_cast<const unsigned char *>(h) + h->total_bytes);
        std::thread([key, device, precision](std::vector<unsigned char> im) {
            cudaSetDevice(device);
            std::unique_ptr<Module> m;
            int rc;
            try {
                rc = build_module(reinterpret_cast<const PackedHeader *>(im.data()), precision, m);
            } catch (const std::bad_alloc &) {
                rc = QMC_ERR_MEMORY;
            }
            finish_slot(key, rc, std::move(m));
        }, std::move(img)).detach();
        return QMC_PENDING;
    }
    std::unique_ptr<Module> m;
    int rc;
    try {
        rc = build_module(h, precision, m);
    } catch (const std::bad_alloc &) {
        rc = QMC_ERR_MEMORY;
    }
    const Module *mp = m.get();
    finish_slot(key, rc, std::move(m));
    if (rc) return rc;
    *out = mp;
    return QMC_OK;
}

}  // namespace

/* ---------------------------------------------------------------- internal interface (qmc_internal.h) */
int qmc_gen_max_block(int dim) { return dim >= 5 ? 128 : 256; }

uint64_t qmc_family_key(const void *packed_host) {
    const PackedHeader *h = hdr(packed_host);
    return h ? family_key(h) : 0;
}

int qmc_gen_kernel(const void *packed_host, int precision, int cls, const void **eval_kernel) {
    const PackedHeader *h = hdr(packed_host);
    if (!h || !eval_kernel || cls < 0 || cls >= QMC_N_CLASSES) return QMC_ERR_ARG;
    const Module *m = nullptr;
    const int rc = get_module(h, precision, &m, nullptr);
    if (rc) return rc;
    if (!m->eval[cls]) return QMC_ERR_ARG;
    *eval_kernel = reinterpret_cast<const void *>(m->eval[cls]);
    return QMC_OK;
}

int qmc_gen_blocks_per_sm(const void *kernel, int block, int smem_bytes, int *out) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kernel, block, smem_bytes) == cudaSuccess ? QMC_OK
                                                                                                       : QMC_ERR_CUDA;
}

int qmc_gen_launch_eval(const void *kernel, const JobTable &t, int grid, int block, void *stream) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    void *args[] = {const_cast<JobTable *>(&t)};
    return cudaLaunchKernel(kernel, dim3(grid), dim3(block), args, (size_t)t.smem_bytes, (cudaStream_t)stream) ==
                   cudaSuccess
               ? QMC_OK
               : QMC_ERR_CUDA;
}

/* ---------------------------------------------------------------- public entry points */
extern "C" {

int qmc_gen_source(const void *packed_host, int32_t precision, char *buf, size_t cap, size_t *len) {
    const PackedHeader *h = hdr(packed_host);
    if (!h || (precision != QMC_PREC_FP64 && precision != QMC_PREC_MIXED)) return QMC_ERR_ARG;
    try {
        const std::string s = generate(h, lang_of(precision));
        if (len) *len = s.size() + 1;
        if (buf) {
            if (cap < s.size() + 1) return QMC_ERR_MEMORY;
            std::memcpy(buf, s.c_str(), s.size() + 1);
        }
        return QMC_OK;
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
}

int qmc_gen_compile(const void *packed_host, int32_t precision, int32_t load, qmc_gen_info *info) {
    const PackedHeader *h = hdr(packed_host);
    if (!h || (precision != QMC_PREC_FP64 && precision != QMC_PREC_MIXED)) return QMC_ERR_ARG;
    try {
        if (info) std::memset(info, 0, sizeof(*info));
        if (info) info->family = family_key(h);
        if (!load) {
            Compiled cc;
            const int rc = compile_cached(h, precision, cc);
            if (info) {
                info->compile_ms = cc.ms;
                info->source_bytes = (int64_t)cc.source_bytes;
                info->cubin_bytes = (int64_t)cc.cubin.size();
                info->cached = cc.from_disk ? 2 : 0;
            }
            return rc;
        }
        const Module *m = nullptr;
        bool cached = false;
        int device = 0;
        if (load == 2 && cudaGetDevice(&device) != cudaSuccess) return QMC_ERR_NO_DEVICE;
        const int rc = get_module(h, precision, &m, &cached, load == 2 ? 1 : 0, device);
        if (rc) return rc;
        if (info) {
            info->compile_ms = m->compile_ms;
            info->source_bytes = m->source_bytes;
            info->cubin_bytes = m->cubin_bytes;
            info->cached = cached ? 1 : (m->from_disk ? 2 : 0);
        }
        return QMC_OK;
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
}

}  // extern "C"
