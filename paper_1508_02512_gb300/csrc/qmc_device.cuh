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
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qmc_internal.h"

#define DEV __device__ __forceinline__

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
    double d = 1.0 / fma(a.x, a.x, a.y * a.y);
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
    return e < 0 ? 1.0 / r : r;
}
/* principal log */
DEV cd clog_p(cd z) { return cd{0.5 * log(fma(z.x, z.x, z.y * z.y)), atan2(z.y, z.x)}; }
/* log(F - i0): a negative real F lies at arg -pi */
DEV cd clog_mi0(cd z) {
    double arg = (z.y == 0.0) ? (z.x < 0.0 ? -M_PI : 0.0) : atan2(z.y, z.x);
    return cd{0.5 * log(fma(z.x, z.x, z.y * z.y)), arg};
}

/* ------------------------------------------------------------------ periodising transform (Eq. 21, order r) */
/* t = phi_r(x), tm = phi_r(1-x) = 1 - t, w = phi_r'(x); phi_r' = c_r x^r (1-x)^r, c_r = (2r+1)!/(r!)^2 */
DEV void transform(int r, double x, double &t, double &tm, double &w) {
    const double y = 1.0 - x;
    switch (r) {
        case 0:
            t = x;
            tm = y;
            w = 1.0;
            break;
        case 1:
            t = x * x * fma(-2.0, x, 3.0);
            tm = y * y * fma(-2.0, y, 3.0);
            w = 6.0 * x * y;
            break;
        case 2: {
            t = x * x * x * fma(x, fma(6.0, x, -15.0), 10.0);
            tm = y * y * y * fma(y, fma(6.0, y, -15.0), 10.0);
            const double xy = x * y;
            w = 30.0 * xy * xy;
            break;
        }
        default: {
            const double x2 = x * x, y2 = y * y;
            t = x2 * x2 * fma(x, fma(x, fma(-20.0, x, 70.0), -84.0), 35.0);
            tm = y2 * y2 * fma(y, fma(y, fma(-20.0, y, 70.0), -84.0), 35.0);
            const double xy = x * y;
            w = 140.0 * xy * xy * xy;
            break;
        }
    }
}

/* ------------------------------------------------------------------ polynomials from shared memory */
DEV uint64_t term_exps(const PackedTerm &T) { return *reinterpret_cast<const uint64_t *>(T.e); }

template <int S>
DEV double poly_r(const PackedTerm *__restrict__ T, int n, const double *t) {
    double acc = 0.0;
    for (int a = 0; a < n; ++a) {
        double m = T[a].c;
        const uint64_t ew = term_exps(T[a]);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int e = (int)((ew >> (8 * j)) & 0xffu);
            for (int k = 0; k < e; ++k) m *= t[j];
        }
        acc += m;
    }
    return acc;
}

template <int S>
DEV cd poly_c(const PackedTerm *__restrict__ T, int n, const cd *z) {
    cd acc = mk(0.0, 0.0);
    for (int a = 0; a < n; ++a) {
        const uint64_t ew = term_exps(T[a]);
        cd m = mk(T[a].c, 0.0);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int e = (int)((ew >> (8 * j)) & 0xffu);
            for (int k = 0; k < e; ++k) m = cmul(m, z[j]);
        }
        acc = cadd(acc, m);
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

/* ------------------------------------------------------------------ sector integrand */
struct Exps {
    int eU0, eU1, eF0, eF1;
};

/* G at the point tt (t with the subset Y zeroed): returns its eps^0 value G0 and the eps-coefficient X of
   its logarithm, so that G(eps) = G0 exp(X eps) (Sec. II, Eq. 9 with the deformation of Eq. 14). */
template <int S, bool DEF, int MAXM>
DEV void eval_G(const PackedSector &s, const PackedTerm *__restrict__ T, const double *tt, const double *ttm,
                const double *Lt, double lam, int M, const Exps &ex, cd &G0, cd &X, uint32_t &fails) {
    const PackedTerm *TU = T;
    const PackedTerm *TF = T + s.nU;
    if constexpr (!DEF) {
        const double U = poly_r<S>(TU, s.nU, tt);
        double F = poly_r<S>(TF, s.nF, tt);
        if (s.kind == 1) F = -F;
        double g = s.D * ipow(U, ex.eU0) * ipow(F, -ex.eF0);
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) g *= tt[j];
        G0 = mk(g, 0.0);
        X = mk(0.0, 0.0);
        if (MAXM > 0 && M > 0) {
            double x = ex.eU1 * log(U) - ex.eF1 * log(F);
#pragma unroll
            for (int j = 0; j < S; ++j)
                if (s.A[j] != -1 && s.B[j] != 0) x = fma((double)s.B[j], Lt[j], x);
            X = mk(x, 0.0);
        }
    } else {
        const PackedTerm *TG = TF + s.nF;
        const PackedTerm *TH = TG + s.nG;
        double g[S];
#pragma unroll
        for (int j = 0; j < S; ++j) g[j] = poly_r<S>(TG + s.gstart[j], s.gstart[j + 1] - s.gstart[j], tt);
        double A[S][S];
        int p = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
#pragma unroll
            for (int k = j; k < S; ++k) {
                const double h = poly_r<S>(TH + s.hstart[p], s.hstart[p + 1] - s.hstart[p], tt);
                ++p;
                A[j][k] = tt[j] * ttm[j] * h;
                if (k != j) A[k][j] = tt[k] * ttm[k] * h;
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
        const cd U = poly_c<S>(TU, s.nU, z);
        const cd F = poly_c<S>(TF, s.nF, z);
        fails += (F.y > 0.0) ? 1u : 0u;
        cd G = cscale(detJ, s.D);
        if (ex.eU0 != 0) G = cmul(G, cipow(U, ex.eU0));
        G = cmul(G, cipow(F, -ex.eF0));
        double mono = 1.0;
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < s.A[j]; ++k) mono *= tt[j];
        G = cscale(G, mono);
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
template <int S, bool DEF, int MAXM>
DEV void point_integrand(const PackedSector &s, const PackedTerm *__restrict__ T, const double *x, int r, double lam,
                         const Exps &ex, cd (&out)[MAXM + 1], uint32_t &fails) {
    double t[S], tm[S], w = 1.0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        double wj;
        transform(r, x[j], t[j], tm[j], wj);
        w *= wj;
        bad |= !(t[j] > 0.0) || !(tm[j] > 0.0);
    }
#pragma unroll
    for (int n = 0; n <= MAXM; ++n) out[n] = mk(0.0, 0.0);
    if (bad || !(w > 0.0)) return;
    const int M = s.M;
    const unsigned smask = (unsigned)s.sing_mask;
    double Lt[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Lt[j] = 0.0;
    if (MAXM > 0 && M > 0) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (((smask >> j) & 1u) || s.B[j] != 0) Lt[j] = log(t[j]);
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
        eval_G<S, DEF, MAXM>(s, T, tt, ttm, Lt, lam, M, ex, G0, X, fails);
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

DEV void kahan_add(double &s, double &c, double v) {
    const double y = v - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

/* ------------------------------------------------------------------ K1: persistent evaluation */
template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(256) qmc_eval_kernel(EvalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ double s_red[16][2 * (MAXM + 1)];
    __shared__ uint32_t s_fail[16];
    const PackedSector &sec = *reinterpret_cast<const PackedSector *>(smem);
    const PackedTerm *T = reinterpret_cast<const PackedTerm *>(smem + sizeof(PackedSector));
    const Exps ex{a.eU0, a.eU1, a.eF0, a.eF1};
    const long long per_sector = (long long)a.m * a.chunks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total_items) break;
        const int ls = (int)(item / per_sector);
        const long long rem = item - (long long)ls * per_sector;
        const int shift = (int)(rem / a.chunks);
        const long long chunk = rem - (long long)shift * a.chunks;
        const int psec = a.sector_begin + ls;
        if (psec != cur) {
            stage_sector(a.packed, a.sectors_off, a.terms_off, psec, smem);
            __syncthreads();
            cur = psec;
        }
        const double lam = a.lambda[sec.orig_index];
        double delta[S];
        uint32_t rj[S];
        const long long i0 = chunk * (long long)blockDim.x * a.P + threadIdx.x;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            delta[j] = a.shifts[6 * shift + j];
            rj[j] = (uint32_t)(((unsigned long long)i0 * a.z[j]) % a.n);
        }
        double acc[2 * (MAXM + 1)], cmp[2 * (MAXM + 1)];
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) acc[q] = cmp[q] = 0.0;
        uint32_t fails = 0;
        for (int p = 0; p < a.P; ++p) {
            const long long i = i0 + (long long)p * blockDim.x;
            if (i < (long long)a.n) {
                double x[S];
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const double v = fma((double)rj[j], a.invn, delta[j]);
                    x[j] = v >= 1.0 ? v - 1.0 : v;
                }
                cd val[MAXM + 1];
                point_integrand<S, DEF, MAXM>(sec, T, x, a.r, lam, ex, val, fails);
#pragma unroll
                for (int n = 0; n <= MAXM; ++n) {
                    kahan_add(acc[2 * n], cmp[2 * n], val[n].x);
                    kahan_add(acc[2 * n + 1], cmp[2 * n + 1], val[n].y);
                }
            }
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const uint32_t v = rj[j] + a.zstep[j];
                rj[j] = v >= a.n ? v - a.n : v;
            }
        }
        /* block reduction: warp shuffles, then warp 0 over the warps in a fixed order */
#pragma unroll
        for (int q = 0; q < 2 * (MAXM + 1); ++q) {
            double v = acc[q] - cmp[q];
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
            if (q < a.n_slots * 2) {
                double s = 0.0, c = 0.0;
                if (q < 2 * (MAXM + 1))
                    for (int w = 0; w < nwarps; ++w) kahan_add(s, c, s_red[w][q]);
                a.partials[item * a.n_slots * 2 + q] = s - c;
            }
            if (q == 0) {
                uint32_t tf = 0;
                for (int w = 0; w < nwarps; ++w) tf += s_fail[w];
                a.part_fails[item] = tf;
            }
        }
        __syncthreads();
    }
}

/* ------------------------------------------------------------------ per-point values on explicit indices */
template <int S, bool DEF, int MAXM>
__global__ void __launch_bounds__(256) qmc_points_kernel(PointArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
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
        point_integrand<S, DEF, MAXM>(sec, T, x, a.r, a.lambda, ex, val, f);
        for (int n = 0; n < a.n_slots; ++n) {
            const cd v = n <= MAXM ? val[n < MAXM + 1 ? n : 0] : mk(0.0, 0.0);
            a.out[(j * a.n_slots + n) * 2] = v.x;
            a.out[(j * a.n_slots + n) * 2 + 1] = v.y;
        }
        a.fails[j] = (int32_t)f;
    }
}

/* ------------------------------------------------------------------ dispatch */
template <int S, bool DEF, int MAXM>
static int launch_eval_t(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    auto k = qmc_eval_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    k<<<grid, block, a.smem_bytes, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int occupancy_t(int block, int smem, int *out) {
    auto k = qmc_eval_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return QMC_ERR_CUDA;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, block, smem) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int launch_points_t(const PointArgs &a, cudaStream_t st) {
    auto k = qmc_points_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    const int block = 128;
    long long g = (a.npts + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    k<<<(int)g, block, a.smem_bytes, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

