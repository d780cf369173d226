#pragma once
/*
 * GB300 (sm_103a) kernels of the quasi-Monte Carlo sector integrator.
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103.
 *
 * qmc_eval_kernel (persistent, one launch per sector class): blocks take work items from an atomic counter;
 *   an item is (sector, shift, chunk of blockDim * P consecutive lattice indices).  The block stages the
 *   sector's polynomial terms into shared memory (one copy per sector change), each thread walks P lattice
 *   points i = i0 + p * blockDim with integer index arithmetic (Eq. 17: x = {i z / n + Delta}), evaluates
 *   the sector integrand series (periodising transform Eq. 21, contour deformation Eq. 14 with its Jacobian,
 *   endpoint subtraction Eqs. 10-12, eps expansion) and accumulates it with Kahan compensation; the block
 *   reduces with warp shuffles and writes one partial per item and slot.
 * qmc_finalize_kernel: one warp per (sector, shift) sums that pair's item partials in a fixed order
 *   (compensated), so results do not depend on which block ran which item (Eqs. 16 and 18).
 * qmc_points_kernel: the same per-point device code on explicit lattice indices (sampled checks).
 *
 * The path is bound by FP64 arithmetic (no dense contraction, nothing streamed from HBM), so no tensor cores
 * or TMA are used: tables live in shared memory, points are generated, outputs are a few KB.
 *
 * This header holds device code only, so that it also compiles at run time (NVRTC) together with the
 * polynomial code generated for one family of sector tables; the host launchers are in qmc_device.cuh.
 */
#ifndef __CUDACC_RTC__
#include <math.h>
#include <stdint.h>
#endif

#include "qmc_internal.h"

#define DEV __device__ __forceinline__
#define QMC_PI 3.141592653589793

/* ------------------------------------------------------------------ complex double */
struct cd {
    double x, y;
};
DEV cd mk(double x, double y) { return cd{x, y}; }
DEV cd cadd(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
DEV cd csub(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
DEV cd cscale(cd a, double s) { return cd{a.x * s, a.y * s}; }
DEV cd cmul(cd a, cd b) { return cd{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)}; }
DEV cd cinv(cd a) {
    const double d = __drcp_rn(fma(a.x, a.x, a.y * a.y));
    return cd{a.x * d, -a.y * d};
}
DEV cd cdiv(cd a, cd b) { return cmul(a, cinv(b)); }
DEV cd cipow(cd z, int e) {
    cd r = mk(1.0, 0.0);
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r = cmul(r, z);
    return e < 0 ? cinv(r) : r;
}
DEV double ipow(double v, int e) {
    double r = 1.0;
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r *= v;
    return e < 0 ? __drcp_rn(r) : r;
}
/* ------------------------------------------------------------------ table-driven FP64 log and atan2 */
/* Logarithm after Tang (P. T. P. Tang, ACM Trans. Math. Softw. 16 (1990) 378): x = 2^e m with m in [1, 2);
   c = 1 + k/128 is the grid point nearest m (k = 0..128); log x = e ln2 + log c + log1p(r) with r = (m - c)/c,
   |r| <= 2^-8, and log1p(r) from its Taylor series through r^7 (the first omitted term is below 2^-67).  m - c
   is exact.  For k >= 64 the split is recentred on 1, log x = (e + 1) ln2 + log(c/2) + log1p(r), so that
   arguments just below 1 meet no cancellation between e ln2 and log c.
   Arctangent by the same table-driven reduction: for 0 <= u = lo/hi <= 1 and the grid point c = k/128 nearest u,
   atan u = atan c + atan(d) with d = (u - c)/(1 + u c) = (lo - c hi)/(hi + c lo), |d| <= 2^-8 + 2^-20, and atan d
   from its Taylor series through d^7 (omitted term below 2^-77); k comes from an FP32 estimate of u, which only
   has to land on the nearest or a neighbouring grid point.  Octants follow from the signs and the swap.
   The tables {1/c, log c} and {k/128, atan(k/128)} are filled once per block (library functions) by
   logtab_init and read from shared memory; arguments outside the fast paths go to the library. */
struct LogTable {
    double inv_c[129];
    double log_c[129];
    double grid[129];
    double atan_c[129];
};
static __shared__ LogTable qmc_logtab;

/* every thread of the block calls it; a __syncthreads() must follow before the first qlog / qatan2 */
DEV void logtab_init() {
    for (int k = threadIdx.x; k <= 128; k += blockDim.x) {
        const double c = 1.0 + k / 128.0;
        qmc_logtab.inv_c[k] = 1.0 / c;
        qmc_logtab.log_c[k] = k < 64 ? log(c) : log(0.5 * c);
        qmc_logtab.grid[k] = k / 128.0;
        qmc_logtab.atan_c[k] = atan(k / 128.0);
    }
}

DEV double qatan2(double y, double x) {
    const double a = fabs(x), b = fabs(y);
    const bool swap = b > a;
    const double hi = swap ? b : a, lo = swap ? a : b;
    if (!(hi > 1e-30 && hi < 1e30 && lo <= hi)) return atan2(y, x); /* zero, tiny, huge or not a number */
    const int k = min(max(__float2int_rn(128.f * __fdividef((float)lo, (float)hi)), 0), 128);
    const double c = qmc_logtab.grid[k];
    const double d = fma(-c, hi, lo) * __drcp_rn(fma(c, lo, hi));
    const double d2 = d * d;
    double q = fma(d2, -1.0 / 7.0, 1.0 / 5.0);
    q = fma(q, d2, -1.0 / 3.0);
    double th = qmc_logtab.atan_c[k] + fma(d * d2, q, d);
    if (swap) th = 0.5 * QMC_PI - th;
    if (x < 0.0) th = QMC_PI - th;
    return copysign(th, y);
}

DEV double qlog(double x) {
    const long long b = __double_as_longlong(x);
    const long long be = b >> 52; /* biased exponent of a positive number; <= 0 for x <= 0 */
    if (be <= 0 || be >= 2047) return log(x);
    const int k = (int)((((b >> 44) & 0xFF) + 1) >> 1);
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double c = __longlong_as_double(0x3FF0000000000000LL + ((long long)k << 45));
    const double r = (m - c) * qmc_logtab.inv_c[k];
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double p = fma(r * r, q, r);
    const double e = (double)(int)(be - 1023 + (k >= 64));
    const double LN2 = 0.6931471805599453, LN2_LO = 2.3190468138462996e-17; /* ln 2 = LN2 + LN2_LO */
    return fma(e, LN2, qmc_logtab.log_c[k]) + fma(e, LN2_LO, p);
}

/* principal log */
DEV cd clog_p(cd z) { return cd{0.5 * qlog(fma(z.x, z.x, z.y * z.y)), qatan2(z.y, z.x)}; }
/* log(F - i0): a negative real F lies at arg -pi */
DEV cd clog_mi0(cd z) {
    double arg = (z.y == 0.0) ? (z.x < 0.0 ? -QMC_PI : 0.0) : qatan2(z.y, z.x);
    return cd{0.5 * qlog(fma(z.x, z.x, z.y * z.y)), arg};
}

/* ------------------------------------------------------------------ periodising transform (Eq. 21, order r) */
/* t = phi_r(x), tm = phi_r(1-x) = 1 - t, w = phi_r'(x); phi_r' = c_r x^r (1-x)^r, c_r = (2r+1)!/(r!)^2 */
DEV double phi_poly(int r, double x) {
    switch (r) {
        case 0: return x;
        case 1: return x * x * fma(-2.0, x, 3.0);
        case 2: return x * x * x * fma(x, fma(6.0, x, -15.0), 10.0);
        default: {
            const double x2 = x * x;
            return x2 * x2 * fma(x, fma(x, fma(-20.0, x, 70.0), -84.0), 35.0);
        }
    }
}
/* phi is evaluated on the smaller of x and 1-x only; phi_r(1-x) = 1 - phi_r(x) gives the other side, which is
   >= 1/2 and therefore exact to rounding */
DEV void transform(int r, double x, double &t, double &tm, double &w) {
    const double y = 1.0 - x;
    const bool lo = x <= 0.5;
    const double p = phi_poly(r, lo ? x : y);
    const double q = 1.0 - p;
    t = lo ? p : q;
    tm = lo ? q : p;
    const double xy = x * y;
    switch (r) {
        case 0: w = 1.0; break;
        case 1: w = 6.0 * xy; break;
        case 2: w = 30.0 * xy * xy; break;
        default: w = 140.0 * xy * xy * xy; break;
    }
}

/* ------------------------------------------------------------------ polynomials from shared memory */
DEV uint64_t term_exps(const PackedTerm &T) { return *reinterpret_cast<const uint64_t *>(T.e); }

/* sum_a c_a prod_j t_j^{e_aj}: the monomial starts from its first factor and the coefficient enters through
   one FMA into the accumulator; exponents are warp-uniform (every lane reads the same term) */
template <int S>
DEV double poly_r(const PackedTerm *__restrict__ T, int n, const double *t) {
    double acc = 0.0;
    for (int a = 0; a < n; ++a) {
        const double c = T[a].c;
        const uint64_t ew = term_exps(T[a]);
        if (ew == 0) {
            acc += c;
            continue;
        }
        double m = 1.0;
        bool have = false;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            int e = (int)((ew >> (8 * j)) & 0xffu);
            if (e > 0) {
                if (!have) {
                    m = t[j];
                    have = true;
                    --e;
                }
                for (int k = 0; k < e; ++k) m *= t[j];
            }
        }
        acc = fma(c, m, acc);
    }
    return acc;
}

template <int S>
DEV cd poly_c(const PackedTerm *__restrict__ T, int n, const cd *z) {
    cd acc = mk(0.0, 0.0);
    for (int a = 0; a < n; ++a) {
        const double c = T[a].c;
        const uint64_t ew = term_exps(T[a]);
        if (ew == 0) {
            acc.x += c;
            continue;
        }
        cd m = mk(1.0, 0.0);
        bool have = false;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            int e = (int)((ew >> (8 * j)) & 0xffu);
            if (e > 0) {
                if (!have) {
                    m = z[j];
                    have = true;
                    --e;
                }
                for (int k = 0; k < e; ++k) m = cmul(m, z[j]);
            }
        }
        acc.x = fma(c, m.x, acc.x);
        acc.y = fma(c, m.y, acc.y);
    }
    return acc;
}

/* ------------------------------------------------------------------ det(I - i lam A), A real S x S */
template <int S>
DEV cd det_deform(const double (&A)[S][S], double lam) {
    if constexpr (S == 1) {
        return mk(1.0, -lam * A[0][0]);
    } else if constexpr (S == 2) {
        const double tr = A[0][0] + A[1][1];
        const double dt = fma(A[0][0], A[1][1], -A[0][1] * A[1][0]);
        return mk(fma(-lam * lam, dt, 1.0), -lam * tr);
    } else if constexpr (S == 3) {
        /* det(I + cA) = 1 + c tr A + c^2 E2(A) + c^3 det A with c = -i lam */
        const double tr = A[0][0] + A[1][1] + A[2][2];
        const double e2 = fma(A[0][0], A[1][1], -A[0][1] * A[1][0]) + fma(A[0][0], A[2][2], -A[0][2] * A[2][0]) +
                          fma(A[1][1], A[2][2], -A[1][2] * A[2][1]);
        const double dt = A[0][0] * fma(A[1][1], A[2][2], -A[1][2] * A[2][1]) -
                          A[0][1] * fma(A[1][0], A[2][2], -A[1][2] * A[2][0]) +
                          A[0][2] * fma(A[1][0], A[2][1], -A[1][1] * A[2][0]);
        const double l2 = lam * lam;
        return mk(fma(-l2, e2, 1.0), fma(l2 * lam, dt, -lam * tr));
    } else {
        /* Gaussian elimination with partial pivoting on J = I - i lam A */
        cd J[S][S];
#pragma unroll
        for (int r = 0; r < S; ++r)
#pragma unroll
            for (int c = 0; c < S; ++c) J[r][c] = mk(r == c ? 1.0 : 0.0, -lam * A[r][c]);
        cd det = mk(1.0, 0.0);
#pragma unroll
        for (int c = 0; c < S; ++c) {
            int p = c;
            double best = fabs(J[c][c].x) + fabs(J[c][c].y);
#pragma unroll
            for (int r = c + 1; r < S; ++r) {
                const double v = fabs(J[r][c].x) + fabs(J[r][c].y);
                if (v > best) {
                    best = v;
                    p = r;
                }
            }
            if (p != c) {
                det = cscale(det, -1.0);
#pragma unroll
                for (int r = c + 1; r < S; ++r) {
                    if (r == p) {
#pragma unroll
                        for (int k = c; k < S; ++k) {
                            const cd tmp = J[c][k];
                            J[c][k] = J[r][k];
                            J[r][k] = tmp;
                        }
                    }
                }
            }
            det = cmul(det, J[c][c]);
            const cd inv = cinv(J[c][c]);
#pragma unroll
            for (int r = c + 1; r < S; ++r) {
                const cd f = cmul(J[r][c], inv);
#pragma unroll
                for (int k = c + 1; k < S; ++k) J[r][k] = csub(J[r][k], cmul(f, J[c][k]));
            }
        }
        return det;
    }
}

/* ------------------------------------------------------------------ polynomial evaluators (FP64)
   The integrand asks an evaluator for
     UFr(Y, t, U, F)          U~ and F~ at real t (undeformed sectors, Eqs. 7-8),
     GH(Y, t, g, h)           g_j = dF~/dt_j and h_p = d2F~/dt_j dt_k (p over j <= k, row-major upper triangle) at
                              real t, the inputs of the deformation of Eq. 14,
     UFc(Y, z, needU, U, F)   U~ (1 when needU is false) and F~ at the deformed point z,
   where the coordinates in the subset Y (bit j = variable j) of the endpoint subtraction (Eqs. 10-12) are zero.
   TabPol walks the staged term table (and ignores Y: zero coordinates make those terms vanish); the generated
   FP64 evaluator (run-time compiled per family) holds each sector's monomials, per zeroed subset without the
   terms that vanish there, as straight-line code and reads only the coefficients from the same table. */
template <int S>
struct TabPol {
    const PackedTerm *T;
    const PackedSector *s;
    DEV static TabPol make(const PackedTerm *T, const PackedSector &s, int) { return TabPol{T, &s}; }
    DEV void UFr(unsigned, const double *t, double &U, double &F) const {
        U = poly_r<S>(T, s->nU, t);
        F = poly_r<S>(T + s->nU, s->nF, t);
    }
    DEV void GH(unsigned, const double *t, double *g, double *h) const {
        const PackedTerm *TG = T + s->nU + s->nF;
        const PackedTerm *TH = TG + s->nG;
#pragma unroll
        for (int j = 0; j < S; ++j) g[j] = poly_r<S>(TG + s->gstart[j], s->gstart[j + 1] - s->gstart[j], t);
#pragma unroll
        for (int p = 0; p < S * (S + 1) / 2; ++p) h[p] = poly_r<S>(TH + s->hstart[p], s->hstart[p + 1] - s->hstart[p], t);
    }
    DEV void UFc(unsigned, const cd *z, bool needU, cd &U, cd &F) const {
        U = needU ? poly_c<S>(T, s->nU, z) : mk(1.0, 0.0);
        F = poly_c<S>(T + s->nU, s->nF, z);
    }
};

/* ------------------------------------------------------------------ sector integrand */
struct Exps {
    int eU0, eU1, eF0, eF1;
};

/* G at the point tt (t with the subset Y zeroed): returns its eps^0 value G0 and the eps-coefficient X of
   its logarithm, so that G(eps) = G0 exp(X eps) (Sec. II, Eq. 9 with the deformation of Eq. 14). */
template <int S, bool DEF, int MAXM, class Pol>
DEV void eval_G(const PackedSector &s, const Pol &P, unsigned Y, const double *tt, const double *ttm, const double *Lt,
                double lam, int M, const Exps &ex, cd &G0, cd &X, uint32_t &fails) {
    if constexpr (!DEF) {
        double U, F;
        P.UFr(Y, tt, U, F);
        if (s.kind == 1) F = -F;
        double g = s.D * ipow(U, ex.eU0) * ipow(F, -ex.eF0);
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) g *= tt[j];
        G0 = mk(g, 0.0);
        X = mk(0.0, 0.0);
        if (MAXM > 0 && M > 0) {
            /* eU1 log U - eF1 log F as one logarithm: both are real and positive on this path */
            double x = qlog(ipow(U, ex.eU1) * ipow(F, -ex.eF1));
#pragma unroll
            for (int j = 0; j < S; ++j)
                if (s.A[j] != -1 && s.B[j] != 0) x = fma((double)s.B[j], Lt[j], x);
            X = mk(x, 0.0);
        }
    } else {
        double g[S], h[S * (S + 1) / 2];
        P.GH(Y, tt, g, h);
        double A[S][S];
        int p = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
#pragma unroll
            for (int k = j; k < S; ++k) {
                A[j][k] = tt[j] * ttm[j] * h[p];
                if (k != j) A[k][j] = tt[k] * ttm[k] * h[p];
                ++p;
            }
        }
#pragma unroll
        for (int j = 0; j < S; ++j) A[j][j] = fma(ttm[j] - tt[j], g[j], A[j][j]);
        const cd detJ = det_deform<S>(A, lam);
        cd z[S], q[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const double d = lam * ttm[j] * g[j];
            z[j] = mk(tt[j], -tt[j] * d);
            q[j] = mk(1.0, -d);
        }
        const bool needU = ex.eU0 != 0 || (MAXM > 0 && M > 0);
        cd U, F;
        P.UFc(Y, z, needU, U, F);
        fails += (F.y > 0.0) ? 1u : 0u;
        cd G = cscale(detJ, s.D);
        if (ex.eU0 != 0) G = cmul(G, cipow(U, ex.eU0));
        G = cmul(G, cipow(F, -ex.eF0));
        bool any_mono = false;
        double mono = 1.0;
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) {
                mono *= tt[j];
                any_mono = true;
            }
        if (any_mono) G = cscale(G, mono);
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (s.A[j] != 0) G = cmul(G, cipow(q[j], s.A[j]));
        G0 = G;
        X = mk(0.0, 0.0);
        if (MAXM > 0 && M > 0) {
            cd x = csub(cscale(clog_p(U), (double)ex.eU1), cscale(clog_mi0(F), (double)ex.eF1));
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (s.B[j] != 0) {
                    if (s.A[j] != -1) x.x = fma((double)s.B[j], Lt[j], x.x);
                    x = cadd(x, cscale(clog_p(q[j]), (double)s.B[j]));
                }
            }
            X = x;
        }
    }
}

/* w(x) * (sector integrand) at x, as series slots 0..M (slot n = coefficient of eps^(n - sigma)).
   Subtraction of Eq. (11) with alpha = -1, regrouped over the zeroed subsets Y of the singular set S:
   eps^sigma I = sum_Y G_Y(eps) V_Y(eps),  V_Y = prod_{j in S\Y} eps t_j^{-1+B eps} prod_{j in Y} (1/B_j - eps t_j^{-1+B eps}). */
template <int S, bool DEF, int MAXM, class Pol>
DEV void point_integrand(const PackedSector &s, const Pol &P, const double *x, int r, double lam,
                         const Exps &ex, cd (&out)[MAXM + 1], uint32_t &fails) {
    double t[S], tm[S], w = 1.0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        double wj;
        transform(r, x[j], t[j], tm[j], wj);
        w *= wj;
        bad |= x[j] == 0.0; /* the weight and t vanish only there: x < 1 after the wrap */
    }
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = mk(0.0, 0.0);
    if (bad) return;
    const int M = s.M;
    const unsigned smask = (unsigned)s.sing_mask;
    double Lt[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Lt[j] = 0.0;
    if (MAXM > 0 && M > 0) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (((smask >> j) & 1u) || s.B[j] != 0) Lt[j] = qlog(t[j]);
    }
    unsigned Y = 0;
    do {
        double tt[S], ttm[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const bool zj = (Y >> j) & 1u;
            tt[j] = zj ? 0.0 : t[j];
            ttm[j] = zj ? 1.0 : tm[j];
        }
        cd G0, X;
        eval_G<S, DEF, MAXM>(s, P, Y, tt, ttm, Lt, lam, M, ex, G0, X, fails);
        double V[MAXM + 1];
        V[0] = 1.0;
#pragma unroll
        for (int n = 1; n <= MAXM; ++n) V[n] = 0.0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            if ((smask >> j) & 1u) {
                const bool inY = (Y >> j) & 1u;
                const double Bj = (double)s.B[j];
                double f[MAXM + 1];
                f[0] = inY ? 1.0 / Bj : 0.0;
                double c = 1.0 / t[j];
#pragma unroll
                for (int n = 1; n <= MAXM; ++n) {
                    f[n] = inY ? -c : c;
                    c *= Bj * Lt[j] / n;
                }
#pragma unroll
                for (int n = MAXM; n >= 0; --n) {
                    double acc = 0.0;
#pragma unroll
                    for (int k = 0; k <= n; ++k) acc = fma(V[k], f[n - k], acc);
                    V[n] = acc;
                }
            }
        }
        cd g = G0;
#pragma unroll
        for (int n = 0; n <= MAXM; ++n) {
            if (n <= M) {
#pragma unroll
                for (int k = 0; k + n <= MAXM; ++k)
                    if (n + k <= M) out[n + k] = cadd(out[n + k], cscale(g, V[k]));
                g = cscale(cmul(g, X), 1.0 / (n + 1));
            }
        }
        Y = (Y - smask) & smask;
    } while (Y != 0);
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = cscale(out[n], w);
}

/* ------------------------------------------------------------------ staging a sector into shared memory */
DEV void stage_sector(const unsigned char *packed, int64_t sectors_off, int64_t terms_off, int psec,
                      unsigned char *smem) {
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(packed + sectors_off) + psec;
    const int4 *src = reinterpret_cast<const int4 *>(ps);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    constexpr int NS = (int)(sizeof(PackedSector) / 16);
    for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = src[k];
    const int nt = ps->n_terms;
    const int4 *tsrc = reinterpret_cast<const int4 *>(packed + terms_off) + ps->term0;
    int4 *tdst = dst + NS;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) tdst[k] = tsrc[k];
}

/* Smallest integer r with fma(r, 1/n, delta) >= 1: the lattice point x = {r/n + delta} wraps exactly for
   r >= R, so the per-point wrap test is an integer compare (evaluated once per item and shift). */
DEV uint32_t wrap_threshold(double delta, uint32_t n, double invn) {
    double g = ceil((1.0 - delta) * (double)n);
    uint32_t R = g <= 0.0 ? 0u : (g >= (double)n ? n : (uint32_t)g);
    while (R > 0 && fma((double)(R - 1), invn, delta) >= 1.0) --R;
    while (R < n && fma((double)R, invn, delta) < 1.0) ++R;
    return R;
}

/* ------------------------------------------------------------------ FP64 islands of a mixed pass
 * The subtraction of Eq. 11 cancels near the faces t_j = 0 of the singular variables (the remark after Eq. 12),
 * and that is where FP32 loses the digits a sector's error budget needs.  A mixed pass may evaluate a sector in
 * FP32 except at its island points, which the FP64 kernel evaluates: at level L, the points whose product over
 * the singular variables of (k_j + 1) / n is below 10^-(L+1), k_j = floor(n x_j) the integer part of the shifted
 * lattice coordinate (x_j = (k_j + b_j) / n, 0 <= b_j < 1).  The FP32 kernels, the FP64 kernel and the probe take
 * this decision with the functions below alone -- integer steps and correctly rounded FP32 operations -- so
 * every kernel sees the same islands. */
DEV uint32_t shift_floor(double delta, uint32_t n) {
    const double fl = floor(__dmul_rn(delta, (double)n));
    return fl >= (double)n ? n - 1u : (uint32_t)fl;
}

DEV uint32_t shifted_index(uint32_t r, uint32_t a, uint32_t n) {
    const uint32_t k = r + a;
    return k >= n ? k - n : k;
}

DEV float island_rn(uint32_t n) { return __frcp_rn(__uint2float_rn(n)); }

/* prod over the singular variables (mask) of (k_j + 1) / n, floored at 1e-30 after each factor (no subnormals) */
template <int S>
DEV float island_key(const uint32_t (&k)[S], unsigned mask, float rn) {
    float c = 1.f;
#pragma unroll
    for (int j = 0; j < S; ++j)
        if ((mask >> j) & 1u) c = fmaxf(__fmul_rn(c, __fmul_rn(__uint2float_rn(k[j] + 1u), rn)), 1e-30f);
    return c;
}

/* the threshold of level L: 10^-(L+1) rounded to FP32 */
DEV float island_xi(int L) {
    return L == 0 ? 1e-1f : L == 1 ? 1e-2f : L == 2 ? 1e-3f : L == 3 ? 1e-4f : L == 4 ? 1e-5f : 1e-6f;
}

/* the number of levels a point with this key is an island at */
DEV int island_bin(float key) {
    int b = 0;
#pragma unroll
    for (int L = 0; L < QMC_ISLAND_LEVELS; ++L) b += key < island_xi(L) ? 1 : 0;
    return b;
}

/* island level of a sector precision code of a mixed pass (2 + L), or -1 */
DEV int island_level(int code) { return code >= 2 && code < 2 + QMC_ISLAND_LEVELS ? code - 2 : -1; }

DEV void kahan_add(double &s, double &c, double v) {
    const double y = v - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

/* ------------------------------------------------------------------ job lookup */
/* the job whose item range contains `item` (jobs are in increasing item_begin) */
DEV int find_job(const JobTable &jt, long long item) {
    int lo = 0, hi = jt.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jt.jobs[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

/* nonzero once the job's abort flag (device-visible, e.g. mapped pinned host memory) is set */
DEV int job_aborted(const Job &J) { return J.abort ? *J.abort : 0; }

/* ------------------------------------------------------------------ K1: persistent FP64 evaluation */
template <int S, int MAXM>
__device__ __noinline__ void point_integrand_taylor(const PackedSector &s, const PackedTerm *T, const double *x, int r,
                                                    Exps ex, double *out);

/* TAYLOR: the sectors of class 2 (endpoint exponents alpha <= -2), evaluated by point_integrand_taylor */
template <int S, bool DEF, int MAXM, class Pol, bool TAYLOR = false>
DEV void eval_f64_body(const JobTable &jt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_job, s_abort;
    __shared__ double s_red[16][2 * (MAXM + 1)];
    __shared__ uint32_t s_fail[16];
    /* per warp: lattice residues r_j of the points gathered for evaluation (at most 63 wait between batches) */
    __shared__ uint32_t s_queue[8][64 * S];
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTerm *T = reinterpret_cast<const PackedTerm *>(smem + sizeof(PackedSector));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *queue = s_queue[warp & 7];
    int cur = -1, cur_job = -1;
    logtab_init(); /* made visible by the __syncthreads() after the first item fetch */
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(jt.counter, 1ull);
            s_item = it;
            s_job = it < jt.total_items ? find_job(jt, it) : 0;
            s_abort = it < jt.total_items ? job_aborted(jt.jobs[s_job]) : 0;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= jt.total_items) break;
        const int jb = s_job;
        const Job &J = jt.jobs[jb];
        const long long local = item - J.item_begin;
        if (s_abort) { /* the pass was stopped: its remaining items contribute nothing */
            if ((int)threadIdx.x < J.n_slots * 2) J.partials[local * J.n_slots * 2 + threadIdx.x] = 0.0;
            if (threadIdx.x == 0) J.part_fails[local] = 0;
            __syncthreads();
            continue;
        }
        const long long per_sector = (long long)J.m * J.chunks;
        const int ls = (int)(local / per_sector);
        const long long rem = local - (long long)ls * per_sector;
        const int shift = (int)(rem / J.chunks);
        const long long chunk = rem - (long long)shift * J.chunks;
        const int psec = J.sector_begin + ls;
        int level = -1; /* island level: this kernel evaluates only the sector's island points */
        if (J.sector_prec) {
            /* mixed pass: items of sectors evaluated in FP32 belong to the other kernel; of sectors with FP64
               islands, this kernel takes the islands and writes the item's partial first (it launches first) */
            const PackedSector *gps = reinterpret_cast<const PackedSector *>(J.packed + J.sectors_off) + psec;
            const int code = J.sector_prec[gps->orig_index];
            if (code == 1) {
                __syncthreads();
                continue;
            }
            level = island_level(code);
        }
        if (psec != cur || jb != cur_job) {
            stage_sector(J.packed, J.sectors_off, J.terms_off, psec, smem);
            __syncthreads();
            cur = psec;
            cur_job = jb;
        }
        const Exps ex{J.eU0, J.eU1, J.eF0, J.eF1};
        const Pol pol = Pol::make(T, sec, psec);
        const uint32_t n = J.n;
        const double invn = J.invn;
        const double lam = J.lambda[sec.orig_index];
        double delta[S];
        uint32_t rj[S], Rj[S], zs[S], aj[S];
        const long long i0 = chunk * (long long)blockDim.x * jt.P + threadIdx.x;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            delta[j] = J.shifts[6 * shift + j];
            rj[j] = (uint32_t)(((unsigned long long)i0 * J.z[j]) % n);
            Rj[j] = wrap_threshold(delta[j], n, invn);
            zs[j] = J.zstep[j];
            aj[j] = shift_floor(delta[j], n);
        }
        const float rn = island_rn(n), xi = island_xi(level < 0 ? 0 : level);
        const unsigned smask = (unsigned)sec.sing_mask;
        /* a thread sums its points plainly; the block combines threads by a shuffle tree, warps and items
           with compensated (Kahan) sums */
        double acc[2 * (MAXM + 1)];
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) acc[q] = 0.0;
        uint32_t fails = 0;
        /* The warp gathers its points (every point, or the islands) into its queue 32 lanes at a time and
           evaluates them in batches of 32, so island points keep whole warps busy.  With every point taken,
           lane l evaluates its own points in order, as a plain loop would. */
        int qn = 0, p = 0;
        for (;;) {
            while (qn < 32 && p < jt.P) {
                const long long i = i0 + (long long)p * blockDim.x;
                bool take = i < (long long)n;
                if (take && level >= 0) {
                    uint32_t k[S];
#pragma unroll
                    for (int j = 0; j < S; ++j) k[j] = shifted_index(rj[j], aj[j], n);
                    take = island_key<S>(k, smask, rn) < xi;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const int pos = qn + __popc(bal & ((1u << lane) - 1u));
#pragma unroll
                    for (int j = 0; j < S; ++j) queue[pos * S + j] = rj[j];
                }
                qn += __popc(bal);
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const uint32_t v = rj[j] + zs[j];
                    rj[j] = v >= n ? v - n : v;
                }
                ++p;
            }
            if (qn == 0) break;
            __syncwarp();
            if (lane < qn) {
                double x[S];
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const uint32_t r = queue[lane * S + j];
                    x[j] = fma((double)r, invn, delta[j]) - (r >= Rj[j] ? 1.0 : 0.0);
                }
                cd val[MAXM + 1];
                if constexpr (TAYLOR) {
                    double v[MAXM + 1];
                    point_integrand_taylor<S, MAXM>(sec, T, x, jt.r, ex, v);
#pragma unroll
                    for (int m = 0; m <= MAXM; ++m) val[m] = mk(v[m], 0.0);
                } else {
                    point_integrand<S, DEF, MAXM>(sec, pol, x, jt.r, lam, ex, val, fails);
                }
#pragma unroll
                for (int m = 0; m <= MAXM; ++m) {
                    acc[2 * m] += val[m].x;
                    acc[2 * m + 1] += val[m].y;
                }
            }
            __syncwarp();
            const int rest = qn > 32 ? qn - 32 : 0;
            if (lane < rest) {
#pragma unroll
                for (int j = 0; j < S; ++j) queue[lane * S + j] = queue[(32 + lane) * S + j];
            }
            __syncwarp();
            qn = rest;
        }
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) {
            double v = acc[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) s_red[warp][q] = v;
        }
        uint32_t f = fails;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
        if (lane == 0) s_fail[warp] = f;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            if (q < J.n_slots * 2) {
                double s2 = 0.0, c2 = 0.0;
                if (q < 2 * (MAXM + 1))
                    for (int w = 0; w < nwarps; ++w) kahan_add(s2, c2, s_red[w][q]);
                J.partials[local * J.n_slots * 2 + q] = s2 - c2;
            }
            if (q == 0) {
                uint32_t tf = 0;
                for (int w = 0; w < nwarps; ++w) tf += s_fail[w];
                J.part_fails[local] = tf;
            }
        }
        __syncthreads();
    }
}

template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(256) qmc_eval_kernel(const __grid_constant__ JobTable jt) {
    eval_f64_body<S, DEF, MAXM, TabPol<S>>(jt);
}

/* ================================================================== endpoint exponents alpha <= -2 (class 2)
 * Sec. II, Eq. (11) with p > 0: for a variable with t^{a + b eps}, a = -1 - p,
 *   int_0^1 t^{a+b eps} f(t) dt = int_0^1 t^{a+b eps} [f(t) - sum_{k<=p} f^(k)(0) t^k/k!] dt
 *                                 + sum_{k<=p} f^(k)(0) / (k! (a + k + 1 + b eps)),
 * applied to every variable with alpha_j <= -1 of the sector (the operators of different variables commute).
 * Per point each such variable takes one of three roles: its value (factor t^{a+b eps}), a subtracted Taylor term,
 * or a pole term.  The Taylor coefficients of f in the variables set to zero (the subset Z) are the coefficients of
 * truncated power series ("jets"): the jets of U~ and F~ restricted to those variables, raised to their
 * eps-dependent powers by the power recurrence of a series, P0 |k| R_k = sum_{0<l<=k} (a |l| - |k-l|) P_l R_{k-l}
 * (from P E R = a R E P with the Euler operator E), and multiplied.  The remainder of a variable with
 * t_j < QMC_TAYLOR_SMALL_T is taken from its own series (orders p_j < k <= p_j + QMC_TAYLOR_EXTRA), because the
 * difference loses its digits there.  Undeformed sectors only (F~ of one sign); FP64, table evaluator. */
#define QMC_TAYLOR_JET (QMC_TAYLOR_Q * QMC_TAYLOR_Q)

/* c = a * b for eps series of length L (truncated) */
template <int L>
DEV void ser_mul(const double *a, const double *b, double *c, int n) {
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s = fma(a[k], b[i - k], s);
        c[i] = s;
    }
}

/* exp(x eps) t^A as a series: t^A x^m / m! */
template <int L>
DEV void ser_power_exp(double tA, double x, double *out, int n) {
    double c = tA;
    for (int m = 0; m < n; ++m) {
        out[m] = c;
        c = c * x / (m + 1);
    }
}

/* R = P^{a0 + a1 eps} for a jet P over d0 x d1 orders (row-major, P[0] > 0); R holds L-term series per entry */
template <int L>
DEV void jet_power(const double *P, int d0, int d1, int a0, int a1, double *R, int n) {
    const double P0 = P[0];
    ser_power_exp<L>(ipow(P0, a0), (double)a1 * qlog(P0), R, n);
    const double inv0 = 1.0 / P0;
    for (int k0 = 0; k0 < d0; ++k0)
        for (int k1 = 0; k1 < d1; ++k1) {
            const int kk = k0 + k1;
            if (kk == 0) continue;
            double acc[L];
            for (int m = 0; m < n; ++m) acc[m] = 0.0;
            for (int l0 = 0; l0 <= k0; ++l0)
                for (int l1 = 0; l1 <= k1; ++l1) {
                    const int ll = l0 + l1;
                    if (ll == 0) continue;
                    const double p = P[l0 * d1 + l1];
                    if (p == 0.0) continue;
                    const double *r = R + ((k0 - l0) * d1 + (k1 - l1)) * L;
                    const double c0 = p * (double)(a0 * ll - (kk - ll)), c1 = p * (double)(a1 * ll);
                    for (int m = n - 1; m >= 0; --m) acc[m] = fma(c0, r[m], m > 0 ? fma(c1, r[m - 1], acc[m]) : acc[m]);
                }
            double *Rk = R + (k0 * d1 + k1) * L;
            const double s = inv0 / (double)kk;
            for (int m = 0; m < n; ++m) Rk[m] = acc[m] * s;
        }
}

/* w(x) * (sector integrand) at x for a class-2 sector, slots 0..M (slot n = coefficient of eps^(n - sigma)) */
template <int S, int MAXM>
__device__ __noinline__ void point_integrand_taylor(const PackedSector &s, const PackedTerm *T, const double *x, int r,
                                                    Exps ex, double *out) {
    constexpr int L = MAXM + 1;
    const int n = s.M + 1;
    for (int m = 0; m < L; ++m) out[m] = 0.0;
    double t[S], lt[S], w = 1.0;
    for (int j = 0; j < S; ++j) {
        double tm, wj;
        if (!(x[j] > 0.0)) return; /* the weight vanishes at x = 0 */
        transform(r, x[j], t[j], tm, wj);
        w *= wj;
        lt[j] = qlog(t[j]);
    }
    int sv[QMC_TAYLOR_MAX_Z], pv[QMC_TAYLOR_MAX_Z];
    bool small[QMC_TAYLOR_MAX_Z];
    int sigma = 0;
    double base[L];
    for (int m = 0; m < L; ++m) base[m] = 0.0;
    base[0] = s.D;
    for (int j = 0; j < S; ++j) {
        if (s.A[j] <= -1) {
            sv[sigma] = j;
            pv[sigma] = -s.A[j] - 1;
            small[sigma] = t[j] < QMC_TAYLOR_SMALL_T;
            ++sigma;
        } else if (s.A[j] != 0 || s.B[j] != 0) {
            double f[L];
            ser_power_exp<L>(ipow(t[j], s.A[j]), (double)s.B[j] * lt[j], f, n);
            ser_mul<L>(base, f, base, n);
        }
    }
    double tpow[QMC_TAYLOR_MAX_Z][L];
    for (int i = 0; i < sigma; ++i) {
        const int j = sv[i];
        ser_power_exp<L>(ipow(t[j], s.A[j]), (double)s.B[j] * lt[j], tpow[i], n);
    }
    const double sgnF = s.kind == 1 ? -1.0 : 1.0; /* F~ < 0 everywhere: |F~| here, the phase on the host */
    double PU[QMC_TAYLOR_JET], PF[QMC_TAYLOR_JET];
    double RU[QMC_TAYLOR_JET * L], RF[QMC_TAYLOR_JET * L];
    for (unsigned zm = 0; zm < (1u << sigma); ++zm) {
        int zi[QMC_TAYLOR_MAX_Z], q[QMC_TAYLOR_MAX_Z], nz = 0;
        for (int i = 0; i < sigma; ++i)
            if ((zm >> i) & 1u) {
                zi[nz] = i;
                q[nz] = small[i] ? pv[i] + QMC_TAYLOR_EXTRA : pv[i];
                ++nz;
            }
        /* the values of the variables outside Z: their remainder as a difference, so zero where it is small */
        double pre[L];
        for (int m = 0; m < L; ++m) pre[m] = base[m];
        bool dead = false;
        for (int i = 0; i < sigma; ++i)
            if (!((zm >> i) & 1u)) {
                if (small[i]) dead = true;
                else ser_mul<L>(pre, tpow[i], pre, n);
            }
        if (dead) continue;
        const int d0 = nz >= 1 ? q[0] + 1 : 1, d1 = nz == 2 ? q[1] + 1 : 1;
        const int nj = d0 * d1;
        for (int k = 0; k < nj; ++k) PU[k] = PF[k] = 0.0;
        for (int a = 0; a < s.nU + s.nF; ++a) {
            const PackedTerm &tm = T[a];
            const int k0 = nz >= 1 ? tm.e[sv[zi[0]]] : 0, k1 = nz == 2 ? tm.e[sv[zi[1]]] : 0;
            if (k0 >= d0 || k1 >= d1) continue;
            double v = a < s.nU ? tm.c : sgnF * tm.c;
            for (int j = 0; j < S; ++j) {
                bool inZ = false;
                for (int i = 0; i < nz; ++i) inZ |= sv[zi[i]] == j;
                if (!inZ) v *= ipow(t[j], tm.e[j]);
            }
            (a < s.nU ? PU : PF)[k0 * d1 + k1] += v;
        }
        jet_power<L>(PU, d0, d1, ex.eU0, ex.eU1, RU, n);
        jet_power<L>(PF, d0, d1, -ex.eF0, -ex.eF1, RF, n);
        /* roles: every subset of Z takes the pole role, the rest of Z the subtracted one */
        for (unsigned tmk = 0; tmk < (1u << nz); ++tmk)
            for (int k0 = 0; k0 < d0; ++k0)
                for (int k1 = 0; k1 < d1; ++k1) {
                    const int kk[2] = {k0, k1};
                    bool skip = false;
                    for (int i = 0; i < nz; ++i) {
                        const int vi = zi[i];
                        const bool pole = (tmk >> i) & 1u;
                        if (pole && kk[i] > pv[vi]) skip = true;
                        /* subtracted: Taylor terms k <= p where the remainder is a difference, series terms
                           k > p where it comes from its series */
                        if (!pole && ((kk[i] <= pv[vi]) == small[vi])) skip = true;
                    }
                    if (skip) continue;
                    double g[L];
                    for (int m = 0; m < L; ++m) g[m] = 0.0;
                    for (int l0 = 0; l0 <= k0; ++l0)
                        for (int l1 = 0; l1 <= k1; ++l1) {
                            double pr[L];
                            ser_mul<L>(RU + (l0 * d1 + l1) * L, RF + ((k0 - l0) * d1 + (k1 - l1)) * L, pr, n);
                            for (int m = 0; m < n; ++m) g[m] += pr[m];
                        }
                    double term[L];
                    ser_mul<L>(pre, g, term, n);
                    int shift = 0;
                    for (int i = 0; i < nz; ++i) {
                        const int vi = zi[i], j = sv[vi];
                        if ((tmk >> i) & 1u) {
                            const int c = s.A[j] + kk[i] + 1;
                            if (c == 0) {
                                for (int m = 0; m < n; ++m) term[m] /= (double)s.B[j];
                                ++shift;
                            } else {
                                double sr[L], f = 1.0 / c;
                                const double ratio = -(double)s.B[j] / c;
                                for (int m = 0; m < n; ++m) {
                                    sr[m] = f;
                                    f *= ratio;
                                }
                                ser_mul<L>(term, sr, term, n);
                            }
                        } else {
                            const double sg = kk[i] <= pv[vi] ? -1.0 : 1.0;
                            double f[L];
                            const double tk = sg * ipow(t[j], kk[i]);
                            for (int m = 0; m < n; ++m) f[m] = tk * tpow[vi][m];
                            ser_mul<L>(term, f, term, n);
                        }
                    }
                    const int lo = sigma - shift;
                    for (int m = lo; m < n; ++m) out[m] += term[m - lo];
                }
    }
    for (int m = 0; m < n; ++m) out[m] *= w;
}

template <int S, int MAXM>
__global__ void __launch_bounds__(256) qmc_eval_kernel_taylor(const __grid_constant__ JobTable jt) {
    eval_f64_body<S, false, MAXM, TabPol<S>, true>(jt);
}

/* ================================================================== FP32 path of the mixed-precision pass
 * The integrand is evaluated in FP32: GB300 issues ~58x more FP32 than FP64 operations.  What stays exact or
 * FP64: the lattice index arithmetic (integers), 1 - x (formed from integers, never by subtraction), the
 * accumulation of the point values (double-float per thread, FP64 per work item and across items). */
struct cf {
    float x, y;
};
DEV cf mkf(float x, float y) { return cf{x, y}; }
/* Complex FP32 arithmetic on GB300's packed two-lane FP32 instructions (one instruction for the real and the
   imaginary part); each lane rounds exactly like the scalar form (x*y + z with one rounding, products rounded
   before they are added). */
DEV float2 f2_(cf a) { return make_float2(a.x, a.y); }
DEV cf cf_(float2 a) { return cf{a.x, a.y}; }
DEV cf caddf(cf a, cf b) { return cf_(__fadd2_rn(f2_(a), f2_(b))); }
DEV cf csubf(cf a, cf b) { return cf_(__fadd2_rn(f2_(a), make_float2(-b.x, -b.y))); }
DEV cf cscalef(cf a, float s) { return cf_(__fmul2_rn(f2_(a), make_float2(s, s))); }
/* (a.x b.x - a.y b.y, a.x b.y + a.y b.x) = (a.x, a.x) * (b.x, b.y) + rn((-a.y, a.y) * (b.y, b.x)) */
DEV cf cmulf(cf a, cf b) {
    return cf_(__ffma2_rn(make_float2(a.x, a.x), f2_(b), __fmul2_rn(make_float2(-a.y, a.y), make_float2(b.y, b.x))));
}
/* a + (c_hi + c_lo) m for a real coefficient split in two floats and a complex monomial m */
DEV cf cfma2f(float hi, float lo, cf m, cf a) {
    return cf_(__ffma2_rn(make_float2(hi, hi), f2_(m), __ffma2_rn(make_float2(lo, lo), f2_(m), f2_(a))));
}
/* the reciprocal of the squared modulus from the fast approximate division (2 ulp): the FP32 path's error is set by
   its rounding of products and sums, and an IEEE-rounded reciprocal costs several instructions more */
DEV cf cinvf(cf a) {
    const float d = __fdividef(1.f, fmaf(a.x, a.x, a.y * a.y));
    return cf{a.x * d, -a.y * d};
}
DEV cf cipowf(cf z, int e) {
    cf r = mkf(1.f, 0.f);
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r = cmulf(r, z);
    return e < 0 ? cinvf(r) : r;
}
DEV float ipowf_(float v, int e) {
    float r = 1.f;
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r *= v;
    return e < 0 ? __frcp_rn(r) : r;
}
DEV cf clogf_p(cf z) { return cf{0.5f * __logf(fmaf(z.x, z.x, z.y * z.y)), atan2f(z.y, z.x)}; }
DEV cf clogf_mi0(cf z) {
    const float arg = (z.y == 0.f) ? (z.x < 0.f ? -3.14159265358979f : 0.f) : atan2f(z.y, z.x);
    return cf{0.5f * __logf(fmaf(z.x, z.x, z.y * z.y)), arg};
}

DEV float phi_poly_f(int r, float x) {
    switch (r) {
        case 0: return x;
        case 1: return x * x * fmaf(-2.f, x, 3.f);
        case 2: return x * x * x * fmaf(x, fmaf(6.f, x, -15.f), 10.f);
        default: {
            const float x2 = x * x;
            return x2 * x2 * fmaf(x, fmaf(x, fmaf(-20.f, x, 70.f), -84.f), 35.f);
        }
    }
}
/* x and y = 1 - x are both given (each accurate relative to itself) */
DEV void transform_f(int r, float x, float y, float &t, float &tm, float &w) {
    const bool lo = x <= y;
    const float p = phi_poly_f(r, lo ? x : y);
    const float q = 1.f - p;
    t = lo ? p : q;
    tm = lo ? q : p;
    const float xy = x * y;
    switch (r) {
        case 0: w = 1.f; break;
        case 1: w = 6.f * xy; break;
        case 2: w = 30.f * xy * xy; break;
        default: w = 140.f * xy * xy * xy; break;
    }
}

DEV uint64_t term_exps_f(const PackedTermF &T) { return *reinterpret_cast<const uint64_t *>(T.e); }

/* Term table of the FP32 path in shared memory (every lane of a warp reads the same term: a broadcast). */
struct SmemTabF {
    const PackedTermF *T;
    DEV float hi(int i) const { return T[i].hi; }
    DEV float lo(int i) const { return T[i].lo; }
    DEV uint64_t ex(int i) const { return term_exps_f(T[i]); }
};

/* coefficient as hi + lo float pair: two FMAs per term keep the coefficient exact to ~2^-48 */
template <int S, class Tab>
DEV float poly_rf(const Tab &T, int base, int n, const float *t) {
    float acc = 0.f;
    for (int a = base; a < base + n; ++a) {
        const uint64_t ew = T.ex(a);
        const float hi = T.hi(a), lo = T.lo(a);
        if (ew == 0) {
            acc += hi + lo;
            continue;
        }
        float m = 1.f;
        bool have = false;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            int e = (int)((ew >> (8 * j)) & 0xffu);
            if (e > 0) {
                if (!have) {
                    m = t[j];
                    have = true;
                    --e;
                }
                for (int k = 0; k < e; ++k) m *= t[j];
            }
        }
        acc = fmaf(hi, m, fmaf(lo, m, acc));
    }
    return acc;
}

template <int S, class Tab>
DEV cf poly_cf(const Tab &T, int base, int n, const cf *z) {
    cf acc = mkf(0.f, 0.f);
    for (int a = base; a < base + n; ++a) {
        const uint64_t ew = T.ex(a);
        const float hi = T.hi(a), lo = T.lo(a);
        if (ew == 0) {
            acc.x += hi + lo;
            continue;
        }
        cf m = mkf(1.f, 0.f);
        bool have = false;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            int e = (int)((ew >> (8 * j)) & 0xffu);
            if (e > 0) {
                if (!have) {
                    m = z[j];
                    have = true;
                    --e;
                }
                for (int k = 0; k < e; ++k) m = cmulf(m, z[j]);
            }
        }
        acc = cfma2f(hi, lo, m, acc);
    }
    return acc;
}

/* Polynomial evaluators of the FP32 path.  The integrand code below asks an evaluator for
     UFr(t, U, F)          U~ and F~ at real t (undeformed sectors, Eqs. 7-8),
     GH(t, g, h)           g_j = dF~/dt_j and h_p = d2F~/dt_j dt_k (p runs over j <= k, row-major upper
                           triangle) at real t, the inputs of the deformation of Eq. 14,
     UFc(z, needU, U, F)   U~ (1 when needU is false) and F~ at the deformed complex point z.
   TabPolF walks the staged term table and decodes each term's exponent bytes.  A generated evaluator
   (compiled at run time for one family of sector tables) holds every sector's monomials as straight-line code
   with shared sub-products and reads only the coefficients (hi + lo) from the same staged table. */
template <int S>
struct TabPolF {
    const PackedTermF *T;
    const PackedSector *s;
    DEV static TabPolF make(const PackedTermF *T, const PackedSector &s, int) { return TabPolF{T, &s}; }
    DEV void UFr(unsigned, const float *t, float &U, float &F) const {
        const SmemTabF tab{T};
        U = poly_rf<S>(tab, 0, s->nU, t);
        F = poly_rf<S>(tab, s->nU, s->nF, t);
    }
    DEV void GH(unsigned, const float *t, float *g, float *h) const {
        const SmemTabF tab{T};
        const int bG = s->nU + s->nF, bH = bG + s->nG;
#pragma unroll
        for (int j = 0; j < S; ++j) g[j] = poly_rf<S>(tab, bG + s->gstart[j], s->gstart[j + 1] - s->gstart[j], t);
#pragma unroll
        for (int p = 0; p < S * (S + 1) / 2; ++p)
            h[p] = poly_rf<S>(tab, bH + s->hstart[p], s->hstart[p + 1] - s->hstart[p], t);
    }
    DEV void UFc(unsigned, const cf *z, bool needU, cf &U, cf &F) const {
        const SmemTabF tab{T};
        U = needU ? poly_cf<S>(tab, 0, s->nU, z) : mkf(1.f, 0.f);
        F = poly_cf<S>(tab, s->nU, s->nF, z);
    }
};

template <int S>
DEV cf det_deform_f(const float (&A)[S][S], float lam) {
    if constexpr (S == 1) {
        return mkf(1.f, -lam * A[0][0]);
    } else if constexpr (S == 2) {
        const float tr = A[0][0] + A[1][1];
        const float dt = fmaf(A[0][0], A[1][1], -A[0][1] * A[1][0]);
        return mkf(fmaf(-lam * lam, dt, 1.f), -lam * tr);
    } else if constexpr (S == 3) {
        const float tr = A[0][0] + A[1][1] + A[2][2];
        const float e2 = fmaf(A[0][0], A[1][1], -A[0][1] * A[1][0]) + fmaf(A[0][0], A[2][2], -A[0][2] * A[2][0]) +
                         fmaf(A[1][1], A[2][2], -A[1][2] * A[2][1]);
        const float dt = A[0][0] * fmaf(A[1][1], A[2][2], -A[1][2] * A[2][1]) -
                         A[0][1] * fmaf(A[1][0], A[2][2], -A[1][2] * A[2][0]) +
                         A[0][2] * fmaf(A[1][0], A[2][1], -A[1][1] * A[2][0]);
        const float l2 = lam * lam;
        return mkf(fmaf(-l2, e2, 1.f), fmaf(l2 * lam, dt, -lam * tr));
    } else {
        cf J[S][S];
#pragma unroll
        for (int r = 0; r < S; ++r)
#pragma unroll
            for (int c = 0; c < S; ++c) J[r][c] = mkf(r == c ? 1.f : 0.f, -lam * A[r][c]);
        cf det = mkf(1.f, 0.f);
#pragma unroll
        for (int c = 0; c < S; ++c) {
            int p = c;
            float best = fabsf(J[c][c].x) + fabsf(J[c][c].y);
#pragma unroll
            for (int r = c + 1; r < S; ++r) {
                const float v = fabsf(J[r][c].x) + fabsf(J[r][c].y);
                if (v > best) {
                    best = v;
                    p = r;
                }
            }
            if (p != c) {
                det = cscalef(det, -1.f);
#pragma unroll
                for (int r = c + 1; r < S; ++r) {
                    if (r == p) {
#pragma unroll
                        for (int k = c; k < S; ++k) {
                            const cf tmp = J[c][k];
                            J[c][k] = J[r][k];
                            J[r][k] = tmp;
                        }
                    }
                }
            }
            det = cmulf(det, J[c][c]);
            const cf inv = cinvf(J[c][c]);
#pragma unroll
            for (int r = c + 1; r < S; ++r) {
                const cf f = cmulf(J[r][c], inv);
#pragma unroll
                for (int k = c + 1; k < S; ++k) J[r][k] = csubf(J[r][k], cmulf(f, J[c][k]));
            }
        }
        return det;
    }
}

/* det(I - i lam A) for S >= 4 in FP32, A = D + T H (D = diag((1-2t)g), T = diag(t(1-t)), H the Hessian of F):
   with s = T^(1/2), A is similar to the symmetric B = D + s H s, so the determinant is that of the complex
   symmetric N = I - i lam B, whose Hermitian part is the identity.  Gaussian elimination without pivoting is
   stable for matrices with a positive definite Hermitian part (every Schur complement keeps one, so no pivot
   vanishes); symmetric elimination works on the upper triangle only.  N holds the upper triangle row-major
   (S(S+1)/2 entries) and is overwritten. */
template <int S>
DEV cf det_sym_f(cf (&N)[S * (S + 1) / 2]) {
    auto at = [](int i, int j) { return i * S - i * (i - 1) / 2 + (j - i); }; /* i <= j */
    cf det = mkf(1.f, 0.f);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const cf dk = N[at(k, k)];
        det = cmulf(det, dk);
        if (k + 1 < S) {
            const cf inv = cinvf(dk);
#pragma unroll
            for (int i = k + 1; i < S; ++i) {
                const cf l = cmulf(N[at(k, i)], inv);
#pragma unroll
                for (int j = i; j < S; ++j) N[at(i, j)] = csubf(N[at(i, j)], cmulf(l, N[at(k, j)]));
            }
        }
    }
    return det;
}

/* FP32 sign check: rounding leaves |Im F| ~ 1e-7 |F| where the deformation vanishes; a point fails when
   Im F(z) exceeds that noise */
#define QMC_F32_SIGN_NOISE 4e-6f

template <int S, bool DEF, int MAXM, class Pol>
DEV void eval_G_f(const PackedSector &s, const Pol &P, unsigned Y, const float *tt, const float *ttm, const float *Lt,
                  float lam, int M, const Exps &ex, cf &G0, cf &X, uint32_t &fails) {
    const float D = s.Df;
    if constexpr (!DEF) {
        float U, F;
        P.UFr(Y, tt, U, F);
        if (s.kind == 1) F = -F;
        float g = D * ipowf_(U, ex.eU0) * ipowf_(F, -ex.eF0);
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) g *= tt[j];
        G0 = mkf(g, 0.f);
        X = mkf(0.f, 0.f);
        if (MAXM > 0 && M > 0) {
            float x = __logf(ipowf_(U, ex.eU1) * ipowf_(F, -ex.eF1));
#pragma unroll
            for (int j = 0; j < S; ++j)
                if (s.A[j] != -1 && s.B[j] != 0) x = fmaf((float)s.B[j], Lt[j], x);
            X = mkf(x, 0.f);
        }
    } else {
        float g[S], h[S * (S + 1) / 2];
        P.GH(Y, tt, g, h);
        cf detJ;
        if constexpr (S >= 4) {
            float s[S];
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const float pj = tt[j] * ttm[j];
                s[j] = pj > 0.f ? pj * rsqrtf(pj) : 0.f;
            }
            cf N[S * (S + 1) / 2];
            int p = 0;
#pragma unroll
            for (int j = 0; j < S; ++j) {
#pragma unroll
                for (int k = j; k < S; ++k) {
                    const float b = (k == j) ? fmaf(ttm[j] - tt[j], g[j], tt[j] * ttm[j] * h[p]) : s[j] * s[k] * h[p];
                    N[p] = mkf(k == j ? 1.f : 0.f, -lam * b);
                    ++p;
                }
            }
            detJ = det_sym_f<S>(N);
        } else {
            float A[S][S];
            int p = 0;
#pragma unroll
            for (int j = 0; j < S; ++j) {
#pragma unroll
                for (int k = j; k < S; ++k) {
                    A[j][k] = tt[j] * ttm[j] * h[p];
                    if (k != j) A[k][j] = tt[k] * ttm[k] * h[p];
                    ++p;
                }
            }
#pragma unroll
            for (int j = 0; j < S; ++j) A[j][j] = fmaf(ttm[j] - tt[j], g[j], A[j][j]);
            detJ = det_deform_f<S>(A, lam);
        }
        cf z[S], q[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float d = lam * ttm[j] * g[j];
            z[j] = mkf(tt[j], -tt[j] * d);
            q[j] = mkf(1.f, -d);
        }
        const bool needU = ex.eU0 != 0 || (MAXM > 0 && M > 0);
        cf U, F;
        P.UFc(Y, z, needU, U, F);
        fails += (F.y > QMC_F32_SIGN_NOISE * (fabsf(F.x) + fabsf(F.y))) ? 1u : 0u;
        cf G = cscalef(detJ, D);
        if (ex.eU0 != 0) G = cmulf(G, cipowf(U, ex.eU0));
        G = cmulf(G, cipowf(F, -ex.eF0));
        bool any_mono = false;
        float mono = 1.f;
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) {
                mono *= tt[j];
                any_mono = true;
            }
        if (any_mono) G = cscalef(G, mono);
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (s.A[j] != 0) G = cmulf(G, cipowf(q[j], s.A[j]));
        G0 = G;
        X = mkf(0.f, 0.f);
        if (MAXM > 0 && M > 0) {
            cf x = csubf(cscalef(clogf_p(U), (float)ex.eU1), cscalef(clogf_mi0(F), (float)ex.eF1));
            /* log q_j with q_j = 1 - i d_j: (log(1 + d_j^2) / 2, -atan d_j) */
            float lr = 0.f;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (s.B[j] != 0) {
                    const float Bj = (float)s.B[j];
                    if (s.A[j] != -1) x.x = fmaf(Bj, Lt[j], x.x);
                    const float d = -q[j].y;
                    lr = fmaf(Bj, __logf(fmaf(d, d, 1.f)), lr);
                    x.y = fmaf(-Bj, atanf(d), x.y);
                }
            }
            x.x = fmaf(0.5f, lr, x.x);
            X = x;
        }
    }
}

template <int S, bool DEF, int MAXM, class Pol>
DEV void point_integrand_f(const PackedSector &s, const Pol &P, const float *x, const float *y, int r, float lam,
                           const Exps &ex, cf (&out)[MAXM + 1], uint32_t &fails) {
    float t[S], tm[S], w = 1.f;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        float wj;
        transform_f(r, x[j], y[j], t[j], tm[j], wj);
        w *= wj;
        bad |= !(t[j] > 0.f) || !(tm[j] > 0.f);
    }
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = mkf(0.f, 0.f);
    if (bad || !(w > 0.f)) return;
    const int M = s.M;
    const unsigned smask = (unsigned)s.sing_mask;
    float Lt[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Lt[j] = 0.f;
    if (MAXM > 0 && M > 0) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (((smask >> j) & 1u) || s.B[j] != 0) Lt[j] = __logf(t[j]);
    }
    unsigned Y = 0;
    do {
        float tt[S], ttm[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const bool zj = (Y >> j) & 1u;
            tt[j] = zj ? 0.f : t[j];
            ttm[j] = zj ? 1.f : tm[j];
        }
        cf G0, X;
        eval_G_f<S, DEF, MAXM>(s, P, Y, tt, ttm, Lt, lam, M, ex, G0, X, fails);
        float V[MAXM + 1];
        V[0] = 1.f;
#pragma unroll
        for (int n = 1; n <= MAXM; ++n) V[n] = 0.f;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            if ((smask >> j) & 1u) {
                const bool inY = (Y >> j) & 1u;
                const float Bj = (float)s.B[j];
                float f[MAXM + 1];
                f[0] = inY ? __fdividef(1.f, Bj) : 0.f;
                float c = __fdividef(1.f, t[j]);
#pragma unroll
                for (int n = 1; n <= MAXM; ++n) {
                    f[n] = inY ? -c : c;
                    c *= Bj * Lt[j] / n;
                }
#pragma unroll
                for (int n = MAXM; n >= 0; --n) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k <= n; ++k) acc = fmaf(V[k], f[n - k], acc);
                    V[n] = acc;
                }
            }
        }
        cf g = G0;
#pragma unroll
        for (int n = 0; n <= MAXM; ++n) {
            if (n <= M) {
#pragma unroll
                for (int k = 0; k + n <= MAXM; ++k)
                    if (n + k <= M) out[n + k] = caddf(out[n + k], cscalef(g, V[k]));
                g = cscalef(cmulf(g, X), 1.f / (n + 1));
            }
        }
        Y = (Y - smask) & smask;
    } while (Y != 0);
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = cscalef(out[n], w);
}

/* x = ((r + a) mod n + b)/n and 1 - x = ((n - 1 - (r + a) mod n) + (1 - b))/n, with delta * n = a + b */
DEV void lattice_f32(uint32_t r, uint32_t a, float b, uint32_t n, float invnf, float &x, float &y) {
    const uint32_t k = shifted_index(r, a, n);
    x = ((float)k + b) * invnf;
    y = ((float)(n - 1u - k) + (1.f - b)) * invnf;
}

DEV void split_shift(double delta, uint32_t n, uint32_t &a, float &b) {
    a = shift_floor(delta, n);
    b = (float)(__dmul_rn(delta, (double)n) - (double)a);
}

/* TwoSum: s + v = (s') + err exactly; the error goes into the compensation term */
DEV void two_sum_acc(float &s, float &c, float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

DEV void stage_sector_f(const unsigned char *packed, int64_t sectors_off, int64_t termsf_off, int psec,
                        unsigned char *smem) {
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(packed + sectors_off) + psec;
    const int4 *src = reinterpret_cast<const int4 *>(ps);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    constexpr int NS = (int)(sizeof(PackedSector) / 16);
    for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = src[k];
    const int nt = ps->n_terms;
    const int4 *tsrc = reinterpret_cast<const int4 *>(packed + termsf_off) + ps->term0;
    int4 *tdst = dst + NS;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) tdst[k] = tsrc[k];
}

/* ------------------------------------------------------------------ K2: persistent FP32 evaluation */
template <int S, bool DEF, int MAXM, class Pol>
DEV void eval_f32_body(const JobTable &jt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_job, s_abort;
    __shared__ double s_red[16][2 * (MAXM + 1)];
    __shared__ uint32_t s_fail[16];
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTermF *T = reinterpret_cast<const PackedTermF *>(smem + sizeof(PackedSector));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int cur = -1, cur_job = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(jt.counter, 1ull);
            s_item = it;
            s_job = it < jt.total_items ? find_job(jt, it) : 0;
            s_abort = it < jt.total_items ? job_aborted(jt.jobs[s_job]) : 0;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= jt.total_items) break;
        const int jb = s_job;
        const Job &J = jt.jobs[jb];
        const long long local = item - J.item_begin;
        if (s_abort) { /* the pass was stopped: its remaining items contribute nothing */
            if ((int)threadIdx.x < J.n_slots * 2) J.partials[local * J.n_slots * 2 + threadIdx.x] = 0.0;
            if (threadIdx.x == 0) J.part_fails[local] = 0;
            __syncthreads();
            continue;
        }
        const long long per_sector = (long long)J.m * J.chunks;
        const int ls = (int)(local / per_sector);
        const long long rem = local - (long long)ls * per_sector;
        const int shift = (int)(rem / J.chunks);
        const long long chunk = rem - (long long)shift * J.chunks;
        const int psec = J.sector_begin + ls;
        int level = -1; /* island level: the FP64 kernel has evaluated the island points and written the partial */
        if (J.sector_prec) {
            /* mixed pass: items of sectors evaluated in FP64 belong to the other kernel */
            const PackedSector *gps = reinterpret_cast<const PackedSector *>(J.packed + J.sectors_off) + psec;
            const int code = J.sector_prec[gps->orig_index];
            level = island_level(code);
            if (code != 1 && level < 0) {
                __syncthreads();
                continue;
            }
        }
        if (psec != cur || jb != cur_job) {
            stage_sector_f(J.packed, J.sectors_off, J.termsf_off, psec, smem);
            __syncthreads();
            cur = psec;
            cur_job = jb;
        }
        const Exps ex{J.eU0, J.eU1, J.eF0, J.eF1};
        const Pol pol = Pol::make(T, sec, psec);
        const uint32_t n = J.n;
        const float invnf = 1.f / (float)n;
        const float lam = (float)J.lambda[sec.orig_index];
        uint32_t rj[S], aj[S], zs[S];
        float bj[S];
        const long long i0 = chunk * (long long)blockDim.x * jt.P + threadIdx.x;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            split_shift(J.shifts[6 * shift + j], n, aj[j], bj[j]);
            rj[j] = (uint32_t)(((unsigned long long)i0 * J.z[j]) % n);
            zs[j] = J.zstep[j];
        }
        float acc[2 * (MAXM + 1)], cmp[2 * (MAXM + 1)];
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) acc[q] = cmp[q] = 0.f;
        uint32_t fails = 0;
        const float rn = island_rn(n), xi = island_xi(level < 0 ? 0 : level);
        for (int p = 0; p < jt.P; ++p) {
            const long long i = i0 + (long long)p * blockDim.x;
            bool take = i < (long long)n;
            if (take && level >= 0) {
                uint32_t k[S];
#pragma unroll
                for (int j = 0; j < S; ++j) k[j] = shifted_index(rj[j], aj[j], n);
                take = !(island_key<S>(k, (unsigned)sec.sing_mask, rn) < xi);
            }
            if (take) {
                float x[S], y[S];
#pragma unroll
                for (int j = 0; j < S; ++j) lattice_f32(rj[j], aj[j], bj[j], n, invnf, x[j], y[j]);
                cf val[MAXM + 1];
                point_integrand_f<S, DEF, MAXM>(sec, pol, x, y, jt.r, lam, ex, val, fails);
#pragma unroll
                for (int m = 0; m <= MAXM; ++m) {
                    two_sum_acc(acc[2 * m], cmp[2 * m], val[m].x);
                    two_sum_acc(acc[2 * m + 1], cmp[2 * m + 1], val[m].y);
                }
            }
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const uint32_t v = rj[j] + zs[j];
                rj[j] = v >= n ? v - n : v;
            }
        }
        /* warp: double-float shuffle tree; warps and items in FP64 */
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) {
            float s1 = acc[q], c1 = cmp[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float so = __shfl_down_sync(0xffffffffu, s1, off);
                const float co = __shfl_down_sync(0xffffffffu, c1, off);
                two_sum_acc(s1, c1, so);
                c1 += co;
            }
            if (lane == 0) s_red[warp][q] = (double)s1 + (double)c1;
        }
        uint32_t f = fails;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
        if (lane == 0) s_fail[warp] = f;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            if (q < J.n_slots * 2) {
                double s2 = 0.0, c2 = 0.0;
                if (q < 2 * (MAXM + 1))
                    for (int w = 0; w < nwarps; ++w) kahan_add(s2, c2, s_red[w][q]);
                double *dst = &J.partials[local * J.n_slots * 2 + q];
                *dst = level >= 0 ? *dst + (s2 - c2) : s2 - c2;
            }
            if (q == 0) {
                uint32_t tf = 0;
                for (int w = 0; w < nwarps; ++w) tf += s_fail[w];
                J.part_fails[local] = level >= 0 ? J.part_fails[local] + tf : tf;
            }
        }
        __syncthreads();
    }
}

template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(256) qmc_eval_kernel_f32(const __grid_constant__ JobTable jt) {
    eval_f32_body<S, DEF, MAXM, TabPolF<S>>(jt);
}

/* ================================================================== FP32 path, two lattice points per thread
 * The generated evaluators of the mixed pass evaluate two lattice points per thread, one in each lane of GB300's
 * packed FP32 instructions (__ffma2_rn, __fmul2_rn, __fadd2_rn): every arithmetic step of the per-point code is
 * issued once for both points, the staged coefficients are read once for both, and the control flow of the
 * subtraction subsets is shared.  Each lane rounds exactly as the scalar code of the one-point path does, so a
 * lane's value equals that path's value for its point.  Steps without a packed form run per lane with the scalar
 * code: the transcendentals, the reciprocals and the elimination of the deformation determinant (which would
 * need twice the registers in packed form).
 * Coefficients are staged as (hi, hi, lo, lo): one 128-bit shared load gives both packed operands of a term. */
DEV float2 bc2(float v) { return make_float2(v, v); }
DEV float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
DEV float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
DEV float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
DEV float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
DEV float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
DEV float lane(float2 v, int k) { return k ? v.y : v.x; }

/* two complex numbers: lane a = (re.x, im.x), lane b = (re.y, im.y) */
struct c2 {
    float2 re, im;
};
DEV c2 mkc2(float2 re, float2 im) { return c2{re, im}; }
DEV c2 zero_c2() { return c2{bc2(0.f), bc2(0.f)}; }
DEV c2 cadd2(c2 a, c2 b) { return c2{add2(a.re, b.re), add2(a.im, b.im)}; }
DEV c2 csub2(c2 a, c2 b) { return c2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
DEV c2 cscale2(c2 a, float2 s) { return c2{mul2(a.re, s), mul2(a.im, s)}; }
/* as cmulf per lane: (fma(a.re, b.re, rn(-a.im b.im)), fma(a.re, b.im, rn(a.im b.re))) */
DEV c2 cmul2(c2 a, c2 b) { return c2{fma2(a.re, b.re, neg2(mul2(a.im, b.im))), fma2(a.re, b.im, mul2(a.im, b.re))}; }
/* a + (hi + lo) m for a staged coefficient (hi, hi, lo, lo), as cfma2f per lane */
DEV c2 cfma2c(const float4 &c, c2 m, c2 a) {
    const float2 h = make_float2(c.x, c.y), l = make_float2(c.z, c.w);
    return c2{fma2(h, m.re, fma2(l, m.re, a.re)), fma2(h, m.im, fma2(l, m.im, a.im))};
}
/* a + hi m, real (coefficients that only shape the contour deformation) */
DEV float2 rfma2h(const float4 &c, float2 m, float2 a) { return fma2(make_float2(c.x, c.y), m, a); }
/* a + (hi + lo) m, real */
DEV float2 rfma2c(const float4 &c, float2 m, float2 a) {
    return fma2(make_float2(c.x, c.y), m, fma2(make_float2(c.z, c.w), m, a));
}
DEV cf lane_c(c2 v, int k) { return cf{lane(v.re, k), lane(v.im, k)}; }
DEV c2 join_c(cf a, cf b) { return c2{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
DEV c2 cinv2(c2 a) {
    const float2 d2 = fma2(a.re, a.re, mul2(a.im, a.im));
    const float2 d = make_float2(__fdividef(1.f, d2.x), __fdividef(1.f, d2.y));
    return c2{mul2(a.re, d), neg2(mul2(a.im, d))};
}
DEV c2 cipow2(c2 z, int e) {
    c2 r = c2{bc2(1.f), bc2(0.f)};
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r = cmul2(r, z);
    return e < 0 ? cinv2(r) : r;
}
DEV float2 ipow2(float2 v, int e) {
    float2 r = bc2(1.f);
    int k = e < 0 ? -e : e;
    for (int i = 0; i < k; ++i) r = mul2(r, v);
    return e < 0 ? make_float2(__frcp_rn(r.x), __frcp_rn(r.y)) : r;
}

/* the periodising transform of both points (transform_f per lane) */
DEV void transform2(int r, float2 x, float2 y, float2 &t, float2 &tm, float2 &w) {
    const bool la = x.x <= y.x, lb = x.y <= y.y;
    const float2 u = make_float2(la ? x.x : y.x, lb ? x.y : y.y);
    float2 p;
    switch (r) {
        case 0: p = u; break;
        case 1: p = mul2(mul2(u, u), fma2(bc2(-2.f), u, bc2(3.f))); break;
        case 2: p = mul2(mul2(mul2(u, u), u), fma2(u, fma2(bc2(6.f), u, bc2(-15.f)), bc2(10.f))); break;
        default: {
            const float2 u2 = mul2(u, u);
            p = mul2(mul2(u2, u2), fma2(u, fma2(u, fma2(bc2(-20.f), u, bc2(70.f)), bc2(-84.f)), bc2(35.f)));
        }
    }
    const float2 q = sub2(bc2(1.f), p);
    t = make_float2(la ? p.x : q.x, lb ? p.y : q.y);
    tm = make_float2(la ? q.x : p.x, lb ? q.y : p.y);
    const float2 xy = mul2(x, y);
    switch (r) {
        case 0: w = bc2(1.f); break;
        case 1: w = mul2(bc2(6.f), xy); break;
        case 2: w = mul2(mul2(bc2(30.f), xy), xy); break;
        default: w = mul2(mul2(mul2(bc2(140.f), xy), xy), xy); break;
    }
}

/* G at the points tt of both lanes (eval_G_f per lane): its eps^0 value G0 and the eps-coefficient X of its
   logarithm.  live: lanes whose point is evaluated (a sign failure is counted only there). */
template <int S, bool DEF, int MAXM, class Pol>
DEV void eval_G_f2(const PackedSector &s, const Pol &P, unsigned Y, const float2 *tt, const float2 *ttm,
                   const float2 *Lt, float lam, int M, const Exps &ex, const bool (&live)[2], c2 &G0, c2 &X,
                   uint32_t &fails) {
    const float2 D = bc2(s.Df);
    if constexpr (!DEF) {
        float2 U, F;
        P.UFr(Y, tt, U, F);
        if (s.kind == 1) F = neg2(F);
        float2 g = mul2(mul2(D, ipow2(U, ex.eU0)), ipow2(F, -ex.eF0));
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) g = mul2(g, tt[j]);
        G0 = c2{g, bc2(0.f)};
        X = zero_c2();
        if (MAXM > 0 && M > 0) {
            const float2 a = mul2(ipow2(U, ex.eU1), ipow2(F, -ex.eF1));
            float2 x = make_float2(__logf(a.x), __logf(a.y));
#pragma unroll
            for (int j = 0; j < S; ++j)
                if (s.A[j] != -1 && s.B[j] != 0) x = fma2(bc2((float)s.B[j]), Lt[j], x);
            X = c2{x, bc2(0.f)};
        }
    } else {
        float2 g[S], h[S * (S + 1) / 2];
        P.GH(Y, tt, g, h);
        cf dets[2];
        if constexpr (S >= 4) {
            /* the matrix entries of both lanes in packed form (rounded as eval_G_f rounds them), then the
               elimination per lane with the lane fixed at compile time (no per-element lane selects) */
            float2 sq[S];
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const float2 pj = mul2(tt[j], ttm[j]);
                sq[j] = make_float2(pj.x > 0.f ? pj.x * rsqrtf(pj.x) : 0.f, pj.y > 0.f ? pj.y * rsqrtf(pj.y) : 0.f);
            }
            float2 bm[S * (S + 1) / 2];
            int p = 0;
#pragma unroll
            for (int j = 0; j < S; ++j) {
#pragma unroll
                for (int i = j; i < S; ++i) {
                    bm[p] = (i == j) ? fma2(sub2(ttm[j], tt[j]), g[j], mul2(mul2(tt[j], ttm[j]), h[p]))
                                     : mul2(mul2(sq[j], sq[i]), h[p]);
                    ++p;
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                cf N[S * (S + 1) / 2];
                int q = 0;
#pragma unroll
                for (int j = 0; j < S; ++j) {
#pragma unroll
                    for (int i = j; i < S; ++i) {
                        N[q] = mkf(i == j ? 1.f : 0.f, -lam * (k ? bm[q].y : bm[q].x));
                        ++q;
                    }
                }
                dets[k] = det_sym_f<S>(N);
            }
        } else {
#pragma unroll 1
            for (int k = 0; k < 2; ++k) {
                /* the determinant per lane, as eval_G_f computes it (one lane at a time: registers) */
                float A[S][S];
                int p = 0;
#pragma unroll
                for (int j = 0; j < S; ++j) {
#pragma unroll
                    for (int i = j; i < S; ++i) {
                        A[j][i] = lane(tt[j], k) * lane(ttm[j], k) * lane(h[p], k);
                        if (i != j) A[i][j] = lane(tt[i], k) * lane(ttm[i], k) * lane(h[p], k);
                        ++p;
                    }
                }
#pragma unroll
                for (int j = 0; j < S; ++j)
                    A[j][j] = fmaf(lane(ttm[j], k) - lane(tt[j], k), lane(g[j], k), A[j][j]);
                dets[k] = det_deform_f<S>(A, lam);
            }
        }
        const c2 detJ = join_c(dets[0], dets[1]);
        c2 z[S], q[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float2 d = mul2(mul2(bc2(lam), ttm[j]), g[j]);
            z[j] = c2{tt[j], neg2(mul2(tt[j], d))};
            q[j] = c2{bc2(1.f), neg2(d)};
        }
        const bool needU = ex.eU0 != 0 || (MAXM > 0 && M > 0);
        c2 U, F;
        P.UFc(Y, z, needU, U, F);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float fr = lane(F.re, k), fi = lane(F.im, k);
            fails += (live[k] && fi > QMC_F32_SIGN_NOISE * (fabsf(fr) + fabsf(fi))) ? 1u : 0u;
        }
        c2 G = cscale2(detJ, D);
        if (ex.eU0 != 0) G = cmul2(G, cipow2(U, ex.eU0));
        G = cmul2(G, cipow2(F, -ex.eF0));
        bool any_mono = false;
        float2 mono = bc2(1.f);
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) {
                mono = mul2(mono, tt[j]);
                any_mono = true;
            }
        if (any_mono) G = cscale2(G, mono);
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (s.A[j] != 0) G = cmul2(G, cipow2(q[j], s.A[j]));
        G0 = G;
        X = zero_c2();
        if (MAXM > 0 && M > 0) {
            cf xs[2];
#pragma unroll 1
            for (int k = 0; k < 2; ++k) {
                cf x = csubf(cscalef(clogf_p(lane_c(U, k)), (float)ex.eU1), cscalef(clogf_mi0(lane_c(F, k)), (float)ex.eF1));
                float lr = 0.f;
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    if (s.B[j] != 0) {
                        const float Bj = (float)s.B[j];
                        if (s.A[j] != -1) x.x = fmaf(Bj, lane(Lt[j], k), x.x);
                        const float d = -lane(q[j].im, k);
                        lr = fmaf(Bj, __logf(fmaf(d, d, 1.f)), lr);
                        x.y = fmaf(-Bj, atanf(d), x.y);
                    }
                }
                x.x = fmaf(0.5f, lr, x.x);
                xs[k] = x;
            }
            X = join_c(xs[0], xs[1]);
        }
    }
}

/* w(x) * (sector integrand) at the points (x, y = 1 - x) of both lanes, as point_integrand_f per lane; live[k]:
   lane k holds a lattice point (its value is zero otherwise) */
template <int S, bool DEF, int MAXM, class Pol>
DEV void point_integrand_f2(const PackedSector &s, const Pol &P, const float2 *x, const float2 *y, int r, float lam,
                            const Exps &ex, bool (&live)[2], c2 (&out)[MAXM + 1], uint32_t &fails) {
    float2 t[S], tm[S], w = bc2(1.f);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        float2 wj;
        transform2(r, x[j], y[j], t[j], tm[j], wj);
        w = mul2(w, wj);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        bool bad = !(lane(w, k) > 0.f);
#pragma unroll
        for (int j = 0; j < S; ++j) bad |= !(lane(t[j], k) > 0.f) || !(lane(tm[j], k) > 0.f);
        live[k] = live[k] && !bad;
    }
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = zero_c2();
    if (!live[0] && !live[1]) return;
    /* a lane without a point evaluates the other lane's point; its value is discarded */
    if (!live[0] || !live[1]) {
        const int from = live[0] ? 0 : 1;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            t[j] = bc2(lane(t[j], from));
            tm[j] = bc2(lane(tm[j], from));
        }
        w = bc2(lane(w, from));
    }
    const int M = s.M;
    const unsigned smask = (unsigned)s.sing_mask;
    float2 Lt[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Lt[j] = bc2(0.f);
    if (MAXM > 0 && M > 0) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (((smask >> j) & 1u) || s.B[j] != 0) Lt[j] = make_float2(__logf(t[j].x), __logf(t[j].y));
    }
    unsigned Y = 0;
    do {
        float2 tt[S], ttm[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const bool zj = (Y >> j) & 1u;
            tt[j] = zj ? bc2(0.f) : t[j];
            ttm[j] = zj ? bc2(1.f) : tm[j];
        }
        c2 G0, X;
        eval_G_f2<S, DEF, MAXM>(s, P, Y, tt, ttm, Lt, lam, M, ex, live, G0, X, fails);
        float2 V[MAXM + 1];
        V[0] = bc2(1.f);
#pragma unroll
        for (int n = 1; n <= MAXM; ++n) V[n] = bc2(0.f);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            if ((smask >> j) & 1u) {
                const bool inY = (Y >> j) & 1u;
                const float Bj = (float)s.B[j];
                float2 f[MAXM + 1];
                f[0] = bc2(inY ? __fdividef(1.f, Bj) : 0.f);
                float2 c = make_float2(__fdividef(1.f, t[j].x), __fdividef(1.f, t[j].y));
#pragma unroll
                for (int n = 1; n <= MAXM; ++n) {
                    f[n] = inY ? neg2(c) : c;
                    /* c *= B_j Lt_j / n, per lane as the one-point code */
                    c = make_float2(c.x * (Bj * Lt[j].x / n), c.y * (Bj * Lt[j].y / n));
                }
#pragma unroll
                for (int n = MAXM; n >= 0; --n) {
                    float2 acc = bc2(0.f);
#pragma unroll
                    for (int k = 0; k <= n; ++k) acc = fma2(V[k], f[n - k], acc);
                    V[n] = acc;
                }
            }
        }
        c2 g = G0;
#pragma unroll
        for (int n = 0; n <= MAXM; ++n) {
            if (n <= M) {
#pragma unroll
                for (int k = 0; k + n <= MAXM; ++k)
                    if (n + k <= M) out[n + k] = cadd2(out[n + k], cscale2(g, V[k]));
                g = cscale2(cmul2(g, X), bc2(1.f / (n + 1)));
            }
        }
        Y = (Y - smask) & smask;
    } while (Y != 0);
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) {
        out[n] = cscale2(out[n], w);
        if (!live[0]) out[n] = c2{make_float2(0.f, out[n].re.y), make_float2(0.f, out[n].im.y)};
        if (!live[1]) out[n] = c2{make_float2(out[n].re.x, 0.f), make_float2(out[n].im.x, 0.f)};
    }
}

/* stage a sector for the two-point path: the record, then each term's coefficient as (hi, hi, lo, lo) */
DEV void stage_sector_f2(const unsigned char *packed, int64_t sectors_off, int64_t termsf_off, int psec,
                         unsigned char *smem) {
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(packed + sectors_off) + psec;
    const int4 *src = reinterpret_cast<const int4 *>(ps);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    constexpr int NS = (int)(sizeof(PackedSector) / 16);
    for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = src[k];
    const int nt = ps->n_terms;
    const PackedTermF *tsrc = reinterpret_cast<const PackedTermF *>(packed + termsf_off) + ps->term0;
    float4 *tdst = reinterpret_cast<float4 *>(dst + NS);
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
        const float hi = tsrc[k].hi, lo = tsrc[k].lo;
        tdst[k] = make_float4(hi, hi, lo, lo);
    }
}

/* ------------------------------------------------------------------ K2x2: persistent FP32 evaluation, two points
   per thread (generated evaluators).  Work items and their partials are those of eval_f32_body; a thread takes its
   P points in pairs (p, p + 1) and accumulates lane a before lane b, i.e. in the one-point path's order. */
template <int S, bool DEF, int MAXM, class Pol>
DEV void eval_f32x2_body(const JobTable &jt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_job, s_abort;
    __shared__ double s_red[16][2 * (MAXM + 1)];
    __shared__ uint32_t s_fail[16];
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const float4 *T = reinterpret_cast<const float4 *>(smem + sizeof(PackedSector));
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int cur = -1, cur_job = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(jt.counter, 1ull);
            s_item = it;
            s_job = it < jt.total_items ? find_job(jt, it) : 0;
            s_abort = it < jt.total_items ? job_aborted(jt.jobs[s_job]) : 0;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= jt.total_items) break;
        const int jb = s_job;
        const Job &J = jt.jobs[jb];
        const long long local = item - J.item_begin;
        if (s_abort) { /* the pass was stopped: its remaining items contribute nothing */
            if ((int)threadIdx.x < J.n_slots * 2) J.partials[local * J.n_slots * 2 + threadIdx.x] = 0.0;
            if (threadIdx.x == 0) J.part_fails[local] = 0;
            __syncthreads();
            continue;
        }
        const long long per_sector = (long long)J.m * J.chunks;
        const int ls = (int)(local / per_sector);
        const long long rem = local - (long long)ls * per_sector;
        const int shift = (int)(rem / J.chunks);
        const long long chunk = rem - (long long)shift * J.chunks;
        const int psec = J.sector_begin + ls;
        int level = -1; /* island level: the FP64 kernel has evaluated the island points and written the partial */
        if (J.sector_prec) {
            const PackedSector *gps = reinterpret_cast<const PackedSector *>(J.packed + J.sectors_off) + psec;
            const int code = J.sector_prec[gps->orig_index];
            level = island_level(code);
            if (code != 1 && level < 0) {
                __syncthreads();
                continue;
            }
        }
        if (psec != cur || jb != cur_job) {
            stage_sector_f2(J.packed, J.sectors_off, J.termsf_off, psec, smem);
            __syncthreads();
            cur = psec;
            cur_job = jb;
        }
        const Exps ex{J.eU0, J.eU1, J.eF0, J.eF1};
        const Pol pol = Pol::make(T, sec, psec);
        const uint32_t n = J.n;
        const float invnf = 1.f / (float)n;
        const float lam = (float)J.lambda[sec.orig_index];
        uint32_t rj[S], aj[S], zs[S];
        float bj[S];
        const long long i0 = chunk * (long long)blockDim.x * jt.P + threadIdx.x;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            split_shift(J.shifts[6 * shift + j], n, aj[j], bj[j]);
            rj[j] = (uint32_t)(((unsigned long long)i0 * J.z[j]) % n);
            zs[j] = J.zstep[j];
        }
        float acc[2 * (MAXM + 1)], cmp[2 * (MAXM + 1)];
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) acc[q] = cmp[q] = 0.f;
        uint32_t fails = 0;
        const float rn = island_rn(n), xi = island_xi(level < 0 ? 0 : level);
        for (int p = 0; p < jt.P; p += 2) {
            bool live[2];
            float2 x[S], y[S];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const long long i = i0 + (long long)(p + k) * blockDim.x;
                live[k] = (p + k < jt.P) && i < (long long)n;
                if (live[k] && level >= 0) {
                    uint32_t kk[S];
#pragma unroll
                    for (int j = 0; j < S; ++j) kk[j] = shifted_index(rj[j], aj[j], n);
                    live[k] = !(island_key<S>(kk, (unsigned)sec.sing_mask, rn) < xi);
                }
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    float xv, yv;
                    lattice_f32(rj[j], aj[j], bj[j], n, invnf, xv, yv);
                    if (k == 0) {
                        x[j].x = xv;
                        y[j].x = yv;
                    } else {
                        x[j].y = xv;
                        y[j].y = yv;
                    }
                    const uint32_t v = rj[j] + zs[j];
                    rj[j] = v >= n ? v - n : v;
                }
            }
            if (live[0] || live[1]) {
                c2 val[MAXM + 1];
                point_integrand_f2<S, DEF, MAXM>(sec, pol, x, y, jt.r, lam, ex, live, val, fails);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (!live[k]) continue;
#pragma unroll
                    for (int m = 0; m <= MAXM; ++m) {
                        two_sum_acc(acc[2 * m], cmp[2 * m], lane(val[m].re, k));
                        two_sum_acc(acc[2 * m + 1], cmp[2 * m + 1], lane(val[m].im, k));
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) {
            float s1 = acc[q], c1 = cmp[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float so = __shfl_down_sync(0xffffffffu, s1, off);
                const float co = __shfl_down_sync(0xffffffffu, c1, off);
                two_sum_acc(s1, c1, so);
                c1 += co;
            }
            if (lane_id == 0) s_red[warp][q] = (double)s1 + (double)c1;
        }
        uint32_t f = fails;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
        if (lane_id == 0) s_fail[warp] = f;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            if (q < J.n_slots * 2) {
                double s2 = 0.0, c2v = 0.0;
                if (q < 2 * (MAXM + 1))
                    for (int w = 0; w < nwarps; ++w) kahan_add(s2, c2v, s_red[w][q]);
                double *dst = &J.partials[local * J.n_slots * 2 + q];
                *dst = level >= 0 ? *dst + (s2 - c2v) : s2 - c2v;
            }
            if (q == 0) {
                uint32_t tf = 0;
                for (int w = 0; w < nwarps; ++w) tf += s_fail[w];
                J.part_fails[local] = level >= 0 ? J.part_fails[local] + tf : tf;
            }
        }
        __syncthreads();
    }
}

/* ------------------------------------------------------------------ K3: FP32-versus-FP64 probe per sector
 * One thread-block cluster per sector (cluster size = the launch's cluster dimension, 1 when clusters cannot be
 * had): block r of the cluster takes the sample points k = r * blockDim + thread (+ blockDim * cluster size), each
 * block reduces its threads in fixed order into shared memory, and block 0 adds the blocks' totals in rank order
 * through distributed shared memory -- deterministic, and no scratch in global memory. */
DEV unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
DEV unsigned cluster_blocks() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
/* every thread of every block of the cluster; orders the cluster's shared-memory writes before later reads */
DEV void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
/* a double in the shared memory of block `rank` of this cluster, at the address of `p` in this block */
DEV double ld_cluster(const double *p, unsigned rank) {
    const unsigned local = (unsigned)__cvta_generic_to_shared(p);
    unsigned remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
    return v;
}

template <int S, bool DEF, int MAXM, class Pol>
DEV void probe_body(const ProbeArgs &a) {
    extern __shared__ __align__(16) unsigned char smem[];
    /* per bin: points, then per slot sum |e|, sum e re, sum e im, sum |e|^2 (e = v32 - v64) */
    constexpr int NBIN = 1 + 4 * (MAXM + 1);
    constexpr int NB = QMC_ISLAND_BINS * NBIN;
    constexpr int NA = 4 * (MAXM + 1);
    __shared__ double s_red[4][NA + NB];
    __shared__ double s_tot[NA + NB];
    const unsigned crank = cluster_rank(), csize = cluster_blocks();
    const int psec = a.sector_begin + (int)(blockIdx.x / csize);
    logtab_init();
    /* FP64 record + terms, then the FP32 terms */
    stage_sector(a.packed, a.sectors_off, a.terms_off, psec, smem);
    const PackedSector *gps = reinterpret_cast<const PackedSector *>(a.packed + a.sectors_off) + psec;
    const int nt = gps->n_terms;
    unsigned char *smf = smem + sizeof(PackedSector) + (size_t)nt * sizeof(PackedTerm);
    {
        const int4 *tsrc = reinterpret_cast<const int4 *>(a.packed + a.termsf_off) + gps->term0;
        int4 *tdst = reinterpret_cast<int4 *>(smf);
        for (int k = threadIdx.x; k < nt; k += blockDim.x) tdst[k] = tsrc[k];
    }
    __syncthreads();
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTerm *T = reinterpret_cast<const PackedTerm *>(smem + sizeof(PackedSector));
    const PackedTermF *TF = reinterpret_cast<const PackedTermF *>(smf);
    const Pol pol = Pol::make(TF, sec, psec);
    const Exps ex{a.eU0, a.eU1, a.eF0, a.eF1};
    const double lam = a.lambda[sec.orig_index];
    const float invnf = 1.f / (float)a.n;
    const unsigned long long stride = a.n_sample >= (int64_t)a.n ? 1ull : (unsigned long long)(a.n / a.n_sample);
    double acc[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) acc[q] = 0.0;
    double bacc[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) bacc[q] = 0.0;
    const float rn = island_rn(a.n);
    uint32_t Rj[S], aj[S];
    float bj[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        Rj[j] = wrap_threshold(a.shift[j], a.n, a.invn);
        split_shift(a.shift[j], a.n, aj[j], bj[j]);
    }
    uint32_t f64 = 0, f32 = 0;
    const long long step = (long long)blockDim.x * csize;
    for (long long k = (long long)crank * blockDim.x + threadIdx.x;
         k < a.n_sample && (unsigned long long)k * stride < a.n; k += step) {
        const unsigned long long i = (unsigned long long)k * stride;
        double x[S];
        float xf[S], yf[S];
        uint32_t kk[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const uint32_t r = (uint32_t)((i * a.z[j]) % a.n);
            x[j] = fma((double)r, a.invn, a.shift[j]) - (r >= Rj[j] ? 1.0 : 0.0);
            lattice_f32(r, aj[j], bj[j], a.n, invnf, xf[j], yf[j]);
            kk[j] = shifted_index(r, aj[j], a.n);
        }
        const int bin = island_bin(island_key<S>(kk, (unsigned)sec.sing_mask, rn));
        cd v64[MAXM + 1];
        cf v32[MAXM + 1];
        point_integrand<S, DEF, MAXM>(sec, TabPol<S>{T, &sec}, x, a.r, lam, ex, v64, f64);
        point_integrand_f<S, DEF, MAXM>(sec, pol, xf, yf, a.r, (float)lam, ex, v32, f32);
#pragma unroll
        for (int b = 0; b < QMC_ISLAND_BINS; ++b) {
            if (b != bin) continue;
            bacc[b * NBIN] += 1.0;
        }
#pragma unroll
        for (int n = 0; n <= MAXM; ++n) {
            const double dr = (double)v32[n].x - v64[n].x, di = (double)v32[n].y - v64[n].y;
            const double m = hypot(dr, di);
            acc[4 * n] += hypot(v64[n].x, v64[n].y);
            acc[4 * n + 1] += m;
            acc[4 * n + 2] += dr;
            acc[4 * n + 3] += di;
#pragma unroll
            for (int b = 0; b < QMC_ISLAND_BINS; ++b) {
                if (b != bin) continue;
                double *e = &bacc[b * NBIN + 1 + 4 * n];
                e[0] += m;
                e[1] += dr;
                e[2] += di;
                e[3] = fma(m, m, e[3]);
            }
        }
    }
    /* threads -> warps (shuffle tree) -> block (warps in order) -> cluster (blocks in rank order) */
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
#pragma unroll
    for (int q = 0; q < NA + NB; ++q) {
        double v = q < NA ? acc[q] : bacc[q - NA];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) s_red[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NA + NB; q += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += s_red[w][q];
        s_tot[q] = v;
    }
    cluster_sync_all();
    if (crank == 0) {
        for (int q = threadIdx.x; q < 4 * a.n_slots; q += blockDim.x) {
            double v = 0.0;
            if (q < NA)
                for (unsigned r = 0; r < csize; ++r) v += ld_cluster(&s_tot[q], r);
            a.out[(size_t)sec.orig_index * a.n_slots * 4 + q] = v;
        }
        if (a.bins) {
            const int per = QMC_ISLAND_BIN_WORDS(a.n_slots);
            for (int q = threadIdx.x; q < QMC_ISLAND_BINS * per; q += blockDim.x) {
                const int b = q / per, e = q - b * per; /* e = 0: points; 1 + 4 slot + {0,1,2,3}: errors */
                double v = 0.0;
                if (e < NBIN)
                    for (unsigned r = 0; r < csize; ++r) v += ld_cluster(&s_tot[NA + b * NBIN + e], r);
                a.bins[(size_t)sec.orig_index * QMC_ISLAND_BINS * per + q] = v;
            }
        }
    }
    /* the other blocks keep their shared memory until block 0 has read it */
    cluster_sync_all();
}

template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(128) qmc_probe_kernel(ProbeArgs a) {
    probe_body<S, DEF, MAXM, TabPolF<S>>(a);
}

/* ------------------------------------------------------------------ per-point values on explicit indices */
template <int S, int MAXM>
__global__ void __launch_bounds__(256) qmc_points_kernel_taylor(PointArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    logtab_init();
    stage_sector(a.packed, a.sectors_off, a.terms_off, a.sector, smem);
    __syncthreads();
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTerm *T = reinterpret_cast<const PackedTerm *>(smem + sizeof(PackedSector));
    const Exps ex{a.eU0, a.eU1, a.eF0, a.eF1};
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < a.npts;
         j += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = (unsigned long long)a.idx[j];
        double x[S];
#pragma unroll
        for (int d = 0; d < S; ++d) {
            const uint32_t rj = (uint32_t)((i * a.z[d]) % a.n);
            const double v = fma((double)rj, a.invn, a.shift[d]);
            x[d] = v >= 1.0 ? v - 1.0 : v;
        }
        double val[MAXM + 1];
        point_integrand_taylor<S, MAXM>(sec, T, x, a.r, ex, val);
        for (int n = 0; n < a.n_slots; ++n) {
            a.out[(j * a.n_slots + n) * 2] = n <= MAXM ? val[n < MAXM + 1 ? n : 0] : 0.0;
            a.out[(j * a.n_slots + n) * 2 + 1] = 0.0;
        }
        a.fails[j] = 0;
    }
}

template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(256) qmc_points_kernel(PointArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    logtab_init();
    stage_sector(a.packed, a.sectors_off, a.terms_off, a.sector, smem);
    __syncthreads();
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTerm *T = reinterpret_cast<const PackedTerm *>(smem + sizeof(PackedSector));
    const Exps ex{a.eU0, a.eU1, a.eF0, a.eF1};
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < a.npts;
         j += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = (unsigned long long)a.idx[j];
        double x[S];
#pragma unroll
        for (int d = 0; d < S; ++d) {
            const uint32_t rj = (uint32_t)((i * a.z[d]) % a.n);
            const double v = fma((double)rj, a.invn, a.shift[d]);
            x[d] = v >= 1.0 ? v - 1.0 : v;
        }
        cd val[MAXM + 1];
        uint32_t f = 0;
        point_integrand<S, DEF, MAXM>(sec, TabPol<S>{T, &sec}, x, a.r, a.lambda, ex, val, f);
        for (int n = 0; n < a.n_slots; ++n) {
            const cd v = n <= MAXM ? val[n < MAXM + 1 ? n : 0] : mk(0.0, 0.0);
            a.out[(j * a.n_slots + n) * 2] = v.x;
            a.out[(j * a.n_slots + n) * 2 + 1] = v.y;
        }
        a.fails[j] = (int32_t)f;
    }
}
