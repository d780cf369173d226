/*
 * Plain FP64 reference of the sector integrand and of the shifted rank-1 lattice sums.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the CPU-baseline leg of the benchmark;
 * never by the product path.  It shares no code with the GPU library.
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103.
 *
 * A sector (Sec. II, Eq. 9) is  D * prod_j t_j^{A_j + B_j eps} * Ut(t)^{eU0 + eU1 eps} * Ft(t)^{-(eF0 + eF1 eps)}
 * on [0,1]^dim, with Ut, Ft polynomials whose constant terms are nonzero.
 *
 * Per point x of the shifted lattice (Eqs. 17-18):
 *   1. periodising transform (Eq. 21, generalised to order r): t_j = phi_r(x_j), weight w = prod_j phi_r'(x_j),
 *      phi_r(x) = int_0^x c_r u^r (1-u)^r du, c_r = (2r+1)!/(r!)^2  (r = 1 is the paper's 3x^2 - 2x^3);
 *      1 - t_j is taken as phi_r(1 - x_j);
 *   2. contour deformation (Eq. 14), for sectors whose Ft changes sign: z_j = t_j - i lam t_j (1-t_j) dFt/dt_j,
 *      applied as a change of variables: Jacobian det(dz/dt) and (z_j/t_j)^{A_j + B_j eps}; the branch of
 *      log Ft follows Ft - i0;
 *   3. endpoint subtraction (Eqs. 10-12 with alpha = -1): for each singular variable j (A_j = -1),
 *      int dt t^{-1+B eps} f = f(0)/(B eps) + int dt t^{-1+B eps} (f(t) - f(0)), applied variable by variable;
 *   4. eps expansion: everything is a truncated Laurent series in eps (Sec. II, after Eq. 12).
 * Lattice sums (Eqs. 16, 18): sum_i w * integrand over the n points of each shift, Kahan-compensated.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXDIM 12
#define OR_MAXSER 24 /* Laurent array length: orders -sigma .. M */

typedef double complex cplx;

typedef struct {
    int dim, kind;           /* kind 0: Ft > 0; 1: Ft < 0; 2: deformed (or sign-indefinite and undeformed) */
    const int *A, *B;
    double D;
    int eU0, eU1, eF0, eF1;
    int nU, nF;
    const double *cU, *cF;   /* coefficients */
    const int *xU, *xF;      /* exponents, row-major terms x dim */
    double lam;
    int r;                   /* transform order */
    int M;                   /* series computed to eps^M before the 1/eps pole factors */
} or_sector;

/* ------------------------------------------------------------------ periodising transform (Eq. 21) */
static double binom(int n, int k) {
    double b = 1.0;
    for (int i = 1; i <= k; ++i) b = b * (n - k + i) / i;
    return b;
}
static double korobov_c(int r) {
    double f = 1.0;
    for (int i = 2; i <= 2 * r + 1; ++i) f *= i;
    double g = 1.0;
    for (int i = 2; i <= r; ++i) g *= i;
    return f / (g * g);
}
static double phi(int r, double x) {
    if (r == 0) return x;
    double s = 0.0;
    for (int i = 0; i <= r; ++i) s += binom(r, i) * ((i % 2) ? -1.0 : 1.0) * pow(x, r + i + 1) / (r + i + 1);
    return korobov_c(r) * s;
}
static double dphi(int r, double x) {
    if (r == 0) return 1.0;
    return korobov_c(r) * pow(x, r) * pow(1.0 - x, r);
}

/* ------------------------------------------------------------------ polynomials */
static double rmono(const double *t, const int *e, int dim) {
    double m = 1.0;
    for (int j = 0; j < dim; ++j)
        for (int k = 0; k < e[j]; ++k) m *= t[j];
    return m;
}
static cplx cmono(const cplx *z, const int *e, int dim) {
    cplx m = 1.0;
    for (int j = 0; j < dim; ++j)
        for (int k = 0; k < e[j]; ++k) m *= z[j];
    return m;
}
static cplx cpoly(int n, const double *c, const int *x, int dim, const cplx *z) {
    cplx s = 0.0;
    for (int a = 0; a < n; ++a) s += c[a] * cmono(z, x + a * dim, dim);
    return s;
}
/* gradient and Hessian of a real polynomial at a real point, by the power rule */
static void grad_hess(int n, const double *c, const int *x, int dim, const double *t, double *g, double *H) {
    int e[OR_MAXDIM];
    for (int j = 0; j < dim; ++j) {
        g[j] = 0.0;
        for (int k = 0; k < dim; ++k) H[j * dim + k] = 0.0;
    }
    for (int a = 0; a < n; ++a) {
        const int *ea = x + a * dim;
        for (int j = 0; j < dim; ++j) {
            if (ea[j] == 0) continue;
            memcpy(e, ea, sizeof(int) * dim);
            e[j] -= 1;
            g[j] += c[a] * ea[j] * rmono(t, e, dim);
            for (int k = 0; k < dim; ++k) {
                if (e[k] == 0) continue;
                int f[OR_MAXDIM];
                memcpy(f, e, sizeof(int) * dim);
                f[k] -= 1;
                H[j * dim + k] += c[a] * ea[j] * e[k] * rmono(t, f, dim);
            }
        }
    }
}

/* determinant by Gaussian elimination with partial pivoting */
static cplx cdet(cplx *m, int n) {
    cplx det = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(m[r * n + c]) > cabs(m[p * n + c])) p = r;
        if (m[p * n + c] == 0.0) return 0.0;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                cplx tmp = m[c * n + k];
                m[c * n + k] = m[p * n + k];
                m[p * n + k] = tmp;
            }
            det = -det;
        }
        det *= m[c * n + c];
        for (int r = c + 1; r < n; ++r) {
            cplx f = m[r * n + c] / m[c * n + c];
            for (int k = c; k < n; ++k) m[r * n + k] -= f * m[c * n + k];
        }
    }
    return det;
}

static cplx cipow(cplx z, int e) {
    cplx r = 1.0;
    int a = e < 0 ? -e : e;
    for (int k = 0; k < a; ++k) r *= z;
    return e < 0 ? 1.0 / r : r;
}

/* log(F - i0): principal branch, with a negative real F taken at arg -pi */
static cplx log_minus_i0(cplx f) {
    double re = creal(f), im = cimag(f);
    double arg = (im == 0.0) ? (re < 0.0 ? -M_PI : 0.0) : atan2(im, re);
    return 0.5 * log(re * re + im * im) + I * arg;
}

/* ------------------------------------------------------------------ the unsubtracted function G (power series) */
/* G(t) = D detJ prod_{j not in S} t_j^{A_j + B_j eps} prod_j (z_j/t_j)^{A_j + B_j eps} Ut(z)^{eU} Ft(z)^{-eF}
   at the point t with t_Y = 0, as coefficients of eps^0..eps^M.  Returns the sign-failure flag. */
static int g_series(const or_sector *s, const double *t0, const double *tm0, unsigned Y, cplx *out) {
    int d = s->dim;
    double t[OR_MAXDIM], tm[OR_MAXDIM];
    for (int j = 0; j < d; ++j) {
        int zeroed = (Y >> j) & 1u;
        t[j] = zeroed ? 0.0 : t0[j];
        tm[j] = zeroed ? 1.0 : tm0[j];
    }
    cplx z[OR_MAXDIM], q[OR_MAXDIM];
    cplx detJ = 1.0;
    int fail = 0;
    if (s->kind == 2) {
        double g[OR_MAXDIM], H[OR_MAXDIM * OR_MAXDIM];
        grad_hess(s->nF, s->cF, s->xF, d, t, g, H);
        cplx J[OR_MAXDIM * OR_MAXDIM];
        for (int j = 0; j < d; ++j) {
            z[j] = t[j] - I * s->lam * t[j] * tm[j] * g[j];
            q[j] = 1.0 - I * s->lam * tm[j] * g[j];
            for (int k = 0; k < d; ++k) {
                double a = t[j] * tm[j] * H[j * d + k] + (j == k ? (tm[j] - t[j]) * g[j] : 0.0);
                J[j * d + k] = (j == k ? 1.0 : 0.0) - I * s->lam * a;
            }
        }
        detJ = cdet(J, d);
    } else {
        for (int j = 0; j < d; ++j) {
            z[j] = t[j];
            q[j] = 1.0;
        }
    }
    cplx Uv = cpoly(s->nU, s->cU, s->xU, d, z);
    cplx Fv = cpoly(s->nF, s->cF, s->xF, d, z);
    if (s->kind == 2 && cimag(Fv) > 0.0) fail = 1;
    cplx g0 = s->D * detJ * cipow(Uv, s->eU0) * cipow(Fv, -s->eF0);
    cplx X = s->eU1 * clog(Uv) - s->eF1 * log_minus_i0(Fv);
    for (int j = 0; j < d; ++j) {
        if (s->A[j] != -1) {
            for (int k = 0; k < s->A[j]; ++k) g0 *= t[j];
            if (s->B[j] != 0) X += s->B[j] * log(t[j]);
        }
        g0 *= cipow(q[j], s->A[j]);
        if (s->B[j] != 0 && s->kind == 2) X += s->B[j] * clog(q[j]);
    }
    cplx term = g0;
    for (int n = 0; n <= s->M; ++n) {
        out[n] = term;
        term *= X / (n + 1);
    }
    return fail;
}

/* ------------------------------------------------------------------ endpoint subtraction, Eq. (11) with p = 0 */
/* Laurent arrays hold orders -sig .. M at indices 0 .. sig+M. */
typedef struct {
    const or_sector *s;
    const double *t, *tm;
    int sing[OR_MAXDIM], sig;
    cplx memo[1 << 6][OR_MAXSER];
    double amemo[1 << 6][OR_MAXSER]; /* |coefficients| of the same leaves */
    int have[1 << 6];
    int fail;
} sub_ctx;

/* res: the subtracted Laurent series; mag: the same recursion applied to magnitudes (|t^{-1+B eps}| (|a| + |b|)
   + |b|/|B|), i.e. the size of the terms that cancel in Eq. (11) -- the scale of its rounding errors. */
static void subtracted(sub_ctx *c, int i, unsigned Y, cplx *res, double *mag) {
    int L = c->sig + c->s->M + 1;
    if (i == c->sig) {
        int slot = 0;
        for (int k = 0; k < c->sig; ++k)
            if ((Y >> c->sing[k]) & 1u) slot |= 1 << k;
        if (!c->have[slot]) {
            cplx g[OR_MAXSER];
            c->fail |= g_series(c->s, c->t, c->tm, Y, g);
            for (int k = 0; k < L; ++k) {
                c->memo[slot][k] = 0.0;
                c->amemo[slot][k] = 0.0;
            }
            for (int n = 0; n <= c->s->M; ++n) {
                c->memo[slot][c->sig + n] = g[n];
                c->amemo[slot][c->sig + n] = cabs(g[n]);
            }
            c->have[slot] = 1;
        }
        memcpy(res, c->memo[slot], sizeof(cplx) * L);
        memcpy(mag, c->amemo[slot], sizeof(double) * L);
        return;
    }
    int j = c->sing[i];
    cplx a[OR_MAXSER], b[OR_MAXSER], tser[OR_MAXSER];
    double am[OR_MAXSER], bm[OR_MAXSER];
    subtracted(c, i + 1, Y, a, am);
    subtracted(c, i + 1, Y | (1u << j), b, bm);
    /* t_j^{-1 + B eps} = (1/t_j) exp(B eps log t_j): power series in eps */
    double lt = log(c->t[j]), Bj = c->s->B[j];
    double term = 1.0 / c->t[j];
    for (int n = 0; n <= c->s->M; ++n) {
        tser[n] = term;
        term *= Bj * lt / (n + 1);
    }
    for (int o = 0; o < L; ++o) {
        cplx acc = 0.0;
        for (int n = 0; n <= o; ++n) acc += tser[n] * (a[o - n] - b[o - n]);
        /* pole term: b / (B eps) moves every order down by one */
        cplx pole = (o + 1 < L) ? b[o + 1] / Bj : 0.0;
        res[o] = acc + pole;
        double macc = 0.0;
        for (int n = 0; n <= o; ++n) macc += cabs(tser[n]) * (am[o - n] + bm[o - n]);
        mag[o] = macc + ((o + 1 < L) ? bm[o + 1] / fabs(Bj) : 0.0);
    }
}

/* Sector integrand times transform weight at the (already shifted) point x in [0,1)^dim.
   out: 2*(sig+kmax+1) doubles (re, im) for orders -sig .. kmax, where kmax = M - sig.  Returns sign-failure flag. */
static int point_value(const or_sector *s, const double *x, cplx *out, double *mag, int nout) {
    int d = s->dim;
    double t[OR_MAXDIM], tm[OR_MAXDIM], w = 1.0;
    for (int j = 0; j < d; ++j) {
        t[j] = phi(s->r, x[j]);
        tm[j] = phi(s->r, 1.0 - x[j]);
        w *= dphi(s->r, x[j]);
    }
    for (int k = 0; k < nout; ++k) {
        out[k] = 0.0;
        mag[k] = 0.0;
    }
    if (w == 0.0) return 0;
    for (int j = 0; j < d; ++j)
        if (t[j] == 0.0 || tm[j] == 0.0) return 0;
    sub_ctx *c = (sub_ctx *)calloc(1, sizeof(sub_ctx));
    c->s = s;
    c->t = t;
    c->tm = tm;
    c->sig = 0;
    for (int j = 0; j < d; ++j)
        if (s->A[j] == -1) c->sing[c->sig++] = j;
    cplx res[OR_MAXSER];
    double rm[OR_MAXSER];
    subtracted(c, 0, 0u, res, rm);
    int fail = c->fail;
    int L = c->sig + s->M + 1;
    for (int k = 0; k < nout && k < L; ++k) {
        out[k] = w * res[k];
        mag[k] = w * rm[k];
    }
    free(c);
    return fail;
}

static void fill_sector(or_sector *s, int dim, int kind, const int *A, const int *B, double D, const int *e4,
                        int nU, const double *cU, const int *xU, int nF, const double *cF, const int *xF,
                        double lam, int r, int M) {
    s->dim = dim;
    s->kind = kind;
    s->A = A;
    s->B = B;
    s->D = D;
    s->eU0 = e4[0];
    s->eU1 = e4[1];
    s->eF0 = e4[2];
    s->eF1 = e4[3];
    s->nU = nU;
    s->cU = cU;
    s->xU = xU;
    s->nF = nF;
    s->cF = cF;
    s->xF = xF;
    s->lam = lam;
    s->r = r;
    s->M = M;
}

/* ------------------------------------------------------------------ exported entry points */
/* integrand series at one point; out has 2*nout doubles */
int oracle_point(int dim, int kind, const int *A, const int *B, double D, const int *e4, int nU, const double *cU,
                 const int *xU, int nF, const double *cF, const int *xF, double lam, int r, int M, const double *x,
                 double *out, int nout) {
    if (dim < 1 || dim > OR_MAXDIM || M + dim + 1 > OR_MAXSER) return -1;
    or_sector s;
    fill_sector(&s, dim, kind, A, B, D, e4, nU, cU, xU, nF, cF, xF, lam, r, M);
    cplx v[OR_MAXSER];
    double mg[OR_MAXSER];
    int f = point_value(&s, x, v, mg, nout);
    for (int k = 0; k < nout; ++k) {
        out[2 * k] = creal(v[k]);
        out[2 * k + 1] = cimag(v[k]);
    }
    return f;
}

/* Shifted lattice sums: for each shift k, sums[k][o] = sum_{i<n} w * integrand({i z/n + Delta_k}) (Kahan),
   l1[k][o] = sum_i |value|, l1c[k][o] = sum_i (magnitude of the terms the subtraction cancels, see
   subtracted()), fails[k] = number of points with Im Ft(z) > 0.  shifts: m x 6 doubles. */
int oracle_lattice_sums(int dim, int kind, const int *A, const int *B, double D, const int *e4, int nU,
                        const double *cU, const int *xU, int nF, const double *cF, const int *xF, double lam, int r,
                        int M, int nout, long long n, const long long *z, const double *shifts, int m, int nthreads,
                        double *sums, double *l1, double *l1c, long long *fails) {
    if (dim < 1 || dim > OR_MAXDIM || M + dim + 1 > OR_MAXSER || n < 1) return -1;
    or_sector s;
    fill_sector(&s, dim, kind, A, B, D, e4, nU, cU, xU, nF, cF, xF, lam, r, M);
    if (nthreads < 1) nthreads = 1;
    for (int k = 0; k < m; ++k) {
        const double *delta = shifts + 6 * k;
        double *part = (double *)calloc((size_t)nthreads * nout * 6, sizeof(double));
        long long *pf = (long long *)calloc((size_t)nthreads, sizeof(long long));
#pragma omp parallel num_threads(nthreads)
        {
            int tid = 0, nt = 1;
#ifdef _OPENMP
            tid = omp_get_thread_num();
            nt = omp_get_num_threads();
#endif
            long long lo = n * tid / nt, hi = n * (tid + 1) / nt;
            double *ps = part + (size_t)tid * nout * 6; /* re, im, cre, cim, l1, l1c per order */
            double x[OR_MAXDIM];
            cplx v[OR_MAXSER];
            double mg[OR_MAXSER];
            for (long long i = lo; i < hi; ++i) {
                for (int j = 0; j < dim; ++j) {
                    double xi = (double)((i * z[j]) % n) / (double)n + delta[j];
                    x[j] = xi >= 1.0 ? xi - 1.0 : xi;
                }
                pf[tid] += point_value(&s, x, v, mg, nout);
                for (int o = 0; o < nout; ++o) {
                    double *a = ps + 6 * o;
                    double y = creal(v[o]) - a[2];
                    double tt = a[0] + y;
                    a[2] = (tt - a[0]) - y;
                    a[0] = tt;
                    y = cimag(v[o]) - a[3];
                    tt = a[1] + y;
                    a[3] = (tt - a[1]) - y;
                    a[1] = tt;
                    a[4] += cabs(v[o]);
                    a[5] += mg[o];
                }
            }
        }
        for (int o = 0; o < nout; ++o) {
            double re = 0, im = 0, cre = 0, cim = 0, ab = 0, abc = 0;
            for (int tid = 0; tid < nthreads; ++tid) {
                double *a = part + (size_t)tid * nout * 6 + 6 * o;
                double y = a[0] - cre, tt = re + y;
                cre = (tt - re) - y;
                re = tt;
                y = a[1] - cim;
                tt = im + y;
                cim = (tt - im) - y;
                im = tt;
                ab += a[4];
                abc += a[5];
            }
            sums[2 * (k * nout + o)] = re;
            sums[2 * (k * nout + o) + 1] = im;
            l1[k * nout + o] = ab;
            l1c[k * nout + o] = abc;
        }
        long long f = 0;
        for (int tid = 0; tid < nthreads; ++tid) f += pf[tid];
        fails[k] = f;
        free(part);
        free(pf);
    }
    return 0;
}

/* CBC criterion sums for every candidate of one component: vals[c] = sum_i p[i] * omega((i*cand[c]) mod n / n),
   scale[c] = sum_i |p[i] * omega(...)|, omega(x) = 2 pi^2 (x^2 - x + 1/6).  Plain double loop. */
int oracle_cbc_component(long long n, const double *p, const long long *cand, long long ncand, int nthreads,
                         double *vals, double *scale) {
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long long c = 0; c < ncand; ++c) {
        double v = 0.0, a = 0.0;
        for (long long i = 0; i < n; ++i) {
            double x = (double)((i * cand[c]) % n) / (double)n;
            double om = 2.0 * M_PI * M_PI * (x * x - x + 1.0 / 6.0);
            v += p[i] * om;
            a += fabs(p[i] * om);
        }
        vals[c] = v;
        scale[c] = a;
    }
    return 0;
}
