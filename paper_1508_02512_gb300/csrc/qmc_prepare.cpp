/*
 * Host preparation of a sector table (qmc_prepare): parsing and validation of the table format, the Gamma
 * prefactor series of Eq. 2, and packing of the relocatable device image (coefficients evaluated at the
 * kinematic point, sector classes, derivative polynomials for the deformation of Eq. 14, the FP32 coefficient
 * pairs, the algorithmic work count).
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103:
 * Sec. II (Eqs. 2, 9-14) fixes the sector integrand.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lattice_table.h"
#include "qmc_host_internal.h"

namespace {

/* ------------------------------------------------------------------ sector table */
struct TTerm {
    uint8_t e[8];
    std::vector<double> c;  // 1 + K
};

struct TSector {
    std::vector<int> A, B;
    double D;
    std::vector<TTerm> U, F;
};

struct Table {
    int n_sectors = 0, dim = 0, loops = 0, n_props = 0, n_nu = 0, K = 0;
    int eU0 = 0, eU1 = 0, eF0 = 0, eF1 = 0;
    std::vector<int> nu;
    std::vector<TSector> sectors;
};

struct Reader {
    const unsigned char *p;
    size_t n, off = 0;
    bool ok = true;
    template <class T>
    T get() {
        T v{};
        if (off + sizeof(T) > n) {
            ok = false;
            return v;
        }
        std::memcpy(&v, p + off, sizeof(T));
        off += sizeof(T);
        return v;
    }
    void align8() { off = (off + 7) & ~size_t(7); }
};

int parse_table(const void *blob, size_t bytes, Table &t) {
    if (!blob || bytes < 64) return QMC_ERR_ARG;
    Reader r{static_cast<const unsigned char *>(blob), bytes};
    if (std::memcmp(blob, "QMCSEC01", 8) != 0) return QMC_ERR_TABLE;
    r.off = 8;
    const int version = r.get<int32_t>();
    t.n_sectors = r.get<int32_t>();
    t.dim = r.get<int32_t>();
    t.loops = r.get<int32_t>();
    t.n_props = r.get<int32_t>();
    t.n_nu = r.get<int32_t>();
    t.K = r.get<int32_t>();
    t.eU0 = r.get<int32_t>();
    t.eU1 = r.get<int32_t>();
    t.eF0 = r.get<int32_t>();
    t.eF1 = r.get<int32_t>();
    const int header_bytes = r.get<int32_t>();
    if (!r.ok || version != 1) return QMC_ERR_TABLE;
    if (t.n_sectors < 1 || t.n_sectors > 1000000 || t.loops < 1 || t.loops > 8 || t.n_props < 1 ||
        t.n_props > 64 || t.K < 0 || t.K > 64)
        return QMC_ERR_TABLE;
    if (t.dim != t.n_props - 1) return QMC_ERR_TABLE;
    if (t.dim < 1 || t.dim > QMC_MAX_DIM) return QMC_ERR_UNSUPPORTED;
    /* the exponents of U and F follow from N_nu and L (Eq. 2 with D = 4 - 2 eps) */
    if (t.eU0 != t.n_nu - 2 * (t.loops + 1) || t.eU1 != t.loops + 1 || t.eF0 != t.n_nu - 2 * t.loops ||
        t.eF1 != t.loops)
        return QMC_ERR_TABLE;
    r.off = 64;
    t.nu.resize(t.n_props);
    int sum_nu = 0;
    for (int i = 0; i < t.n_props; ++i) {
        t.nu[i] = r.get<int32_t>();
        if (t.nu[i] < 1 || t.nu[i] > 16) return QMC_ERR_UNSUPPORTED;
        sum_nu += t.nu[i];
    }
    if (sum_nu != t.n_nu) return QMC_ERR_TABLE;
    if (header_bytes < 64 || (size_t)header_bytes > bytes) return QMC_ERR_TABLE;
    r.off = header_bytes;
    const int d = t.dim;
    t.sectors.resize(t.n_sectors);
    for (auto &s : t.sectors) {
        const int nU = r.get<int32_t>(), nF = r.get<int32_t>();
        if (!r.ok || nU < 1 || nF < 1 || nU > QMC_MAX_SECTOR_TERMS || nF > QMC_MAX_SECTOR_TERMS)
            return QMC_ERR_TABLE;
        s.A.resize(d);
        s.B.resize(d);
        for (int j = 0; j < d; ++j) s.A[j] = r.get<int32_t>();
        for (int j = 0; j < d; ++j) s.B[j] = r.get<int32_t>();
        r.align8();
        s.D = r.get<double>();
        if (!r.ok || !std::isfinite(s.D)) return QMC_ERR_TABLE;
        for (int j = 0; j < d; ++j) {
            if (s.A[j] < -1 - QMC_TAYLOR_MAX_P || s.A[j] > QMC_MAX_EXP)
                return s.A[j] < 0 ? QMC_ERR_UNSUPPORTED : QMC_ERR_TABLE;
            if (s.A[j] <= -1 && s.B[j] == 0) return QMC_ERR_TABLE; /* unregulated endpoint singularity */
            if (std::abs(s.B[j]) > 64) return QMC_ERR_TABLE;
        }
        for (int pass = 0; pass < 2; ++pass) {
            auto &poly = pass ? s.F : s.U;
            poly.resize(pass ? nF : nU);
            bool has_const = false;
            for (auto &term : poly) {
                for (int k = 0; k < 8; ++k) term.e[k] = r.get<uint8_t>();
                bool zero = true;
                for (int k = 0; k < 8; ++k) {
                    if (k >= d && term.e[k] != 0) return QMC_ERR_TABLE;
                    if (term.e[k] > QMC_MAX_EXP) return QMC_ERR_UNSUPPORTED;
                    zero &= term.e[k] == 0;
                }
                has_const |= zero;
                term.c.resize(1 + t.K);
                for (int k = 0; k <= t.K; ++k) {
                    term.c[k] = r.get<double>();
                    if (!std::isfinite(term.c[k])) return QMC_ERR_TABLE;
                }
            }
            if (!has_const) return QMC_ERR_TABLE; /* factorised form of Eqs. (7)-(8) needs a constant term */
        }
        if (!r.ok) return QMC_ERR_TABLE;
    }
    if (r.off != bytes) return QMC_ERR_TABLE;
    return QMC_OK;
}

/* ------------------------------------------------------------------ Gamma prefactor series (Eq. 2) */
/* zeta(k), k >= 2, from the alternating series eta(k) = (1 - 2^{1-k}) zeta(k) accelerated with Borwein's
   d_k weights (P. Borwein, "An efficient algorithm for the Riemann zeta function", 2000). */
double zeta_int(int s) {
    const int n = 28;
    std::vector<double> dk(n + 1);
    double acc = 0.0;
    for (int i = 0; i <= n; ++i) {
        /* term_i = n (n+i-1)! 4^i / ((n-i)! (2i)!) */
        double lt = std::log((double)n) + std::lgamma((double)(n + i)) + i * std::log(4.0) -
                    std::lgamma((double)(n - i + 1)) - std::lgamma((double)(2 * i + 1));
        acc += std::exp(lt);
        dk[i] = acc;
    }
    double sum = 0.0;
    for (int k = 0; k < n; ++k) sum += ((k % 2) ? -1.0 : 1.0) * (dk[k] - dk[n]) / std::pow(k + 1.0, s);
    const double eta = -sum / dk[n];
    return eta / (1.0 - std::pow(2.0, 1 - s));
}

const double kEulerGamma = 0.57721566490153286061;

/* exp of a power series p (p[0] = 0) up to x^order */
std::vector<double> series_exp(const std::vector<double> &p, int order) {
    std::vector<double> e(order + 1, 0.0);
    e[0] = 1.0;
    for (int n = 1; n <= order; ++n) {
        double s = 0.0;
        for (int k = 1; k <= n && k < (int)p.size(); ++k) s += k * p[k] * e[n - k];
        e[n] = s / n;
    }
    return e;
}

/* Gamma(n + a eps) = eps^low * sum_k out[k] eps^k up to eps^order (order counted from eps^0) */
void gamma_series(int n, int a, int order, int &low, std::vector<double> &out) {
    if (n >= 1) {
        /* log Gamma(n + x) = log Gamma(n) + psi(n) x + sum_{k>=2} psi^{(k-1)}(n) x^k / k! */
        std::vector<double> p(order + 1, 0.0);
        double fact = 1.0;
        for (int k = 1; k <= order; ++k) {
            double psi;
            if (k == 1) {
                psi = -kEulerGamma;
                for (int j = 1; j < n; ++j) psi += 1.0 / j;
            } else {
                const int m = k - 1;
                double h = 0.0;
                for (int j = 1; j < n; ++j) h += std::pow((double)j, -(m + 1));
                double mf = 1.0;
                for (int i = 2; i <= m; ++i) mf *= i;
                psi = ((m % 2) ? 1.0 : -1.0) * mf * (zeta_int(m + 1) - h); /* (-1)^{m+1} m! (...) */
            }
            fact *= k;
            p[k] = psi * std::pow((double)a, k) / fact;
        }
        std::vector<double> e = series_exp(p, order);
        double g = 1.0;
        for (int i = 2; i < n; ++i) g *= i;
        low = 0;
        out.resize(order + 1);
        for (int k = 0; k <= order; ++k) out[k] = g * e[k];
        return;
    }
    /* Gamma(n + x) = Gamma(1 + x) / prod_{j=n}^{0} (j + x): one pole from j = 0 */
    int l1;
    std::vector<double> g1;
    gamma_series(1, a, order + 1, l1, g1);
    for (int j = n; j < 0; ++j) {
        /* 1/(j + a eps) = (1/j) sum_k (-a eps / j)^k */
        std::vector<double> inv(order + 2);
        for (int k = 0; k < order + 2; ++k) inv[k] = (1.0 / j) * std::pow(-(double)a / j, k);
        std::vector<double> r(order + 2, 0.0);
        for (int u = 0; u < order + 2; ++u)
            for (int v = 0; u + v < order + 2; ++v) r[u + v] += g1[u] * inv[v];
        g1 = r;
    }
    low = -1;
    out.resize(order + 1);
    for (int k = 0; k <= order; ++k) out[k] = g1[k] / a;
}

/* ------------------------------------------------------------------ packing */
struct PTerm {
    double c;
    uint8_t e[8];
};

int deg_of(const PTerm &t, int d) {
    int s = 0;
    for (int j = 0; j < d; ++j) s += t.e[j];
    return s;
}

double transform_flops(int r) {
    /* per dimension: lattice point (fma + wrap: 3), the transform polynomial on one side by Horner, 1 - p,
       1 - x, the weight c_r (x(1-x))^r and its product into w */
    switch (r) {
        case 0: return 3.0 + 0.0 + 1.0 + 1.0 + 0.0 + 1.0;
        case 1: return 3.0 + 4.0 + 1.0 + 1.0 + 2.0 + 1.0;
        case 2: return 3.0 + 7.0 + 1.0 + 1.0 + 3.0 + 1.0;
        default: return 3.0 + 9.0 + 1.0 + 1.0 + 4.0 + 1.0;
    }
}

/* Algorithmic FP work of one evaluation of a sector: every add or multiply is 1 flop, an FMA 2, a complex
   multiply 6, a real-times-complex product 2.  Counted from the sector's tables: transform, and per zeroed
   subset (2^sigma of them) the polynomial terms (real term of degree d >= 1: d+1; complex: 6(d-1)+4;
   constants: 1), for deformed sectors the matrix A, det(I - i lam A), z and q, integer powers and monomials,
   the eps-series products; finally weight and accumulation.  Reciprocals count 1; logarithms and atan2 are
   transcendentals, counted separately. */
void sector_work(const PackedSector &s, const PTerm *T, int d, int r, int eU0, int eF0, double &flops,
                 double &transc) {
    const int M = s.M;
    if (s.taylor) {
        /* class 2 (Eq. 11 with p > 0), counted where no remainder comes from its series: per subset Z of the
           singular variables, the jets of U~ and F~ (J = prod (p_j + 1) orders), two power recurrences, the jet
           product per role and the role factors; eps series of L = M + 1 terms */
        const int L = M + 1;
        int pv[QMC_MAX_DIM], ns = 0;
        for (int j = 0; j < d; ++j)
            if (s.A[j] <= -1) pv[ns++] = -s.A[j] - 1;
        double f = d * transform_flops(r);
        for (int zm = 0; zm < (1 << ns); ++zm) {
            double J = 1.0;
            int nz = 0;
            for (int i = 0; i < ns; ++i)
                if ((zm >> i) & 1) {
                    J *= pv[i] + 1;
                    ++nz;
                }
            f += (s.nU + s.nF) * (d - nz + 1.0);
            f += 2.0 * (J * (J + 1.0) / 2.0) * 4.0 * L;
            f += (double)(1 << nz) * J * (J * L * L + (2.0 + nz) * L * L);
            f += (ns - nz) * (double)L * L;
        }
        flops = f + 4.0 * L;
        transc = d + 2.0 * (1 << ns);
        return;
    }
    double per_subset = 0.0, trans_subset = 0.0;
    auto real_poly = [&](int off, int n) {
        double f = 0.0;
        for (int a = 0; a < n; ++a) {
            const int g = deg_of(T[off + a], d);
            f += g == 0 ? 1.0 : g + 1.0;
        }
        return f;
    };
    auto cplx_poly = [&](int off, int n) {
        double f = 0.0;
        for (int a = 0; a < n; ++a) {
            const int g = deg_of(T[off + a], d);
            f += g == 0 ? 1.0 : 6.0 * (g - 1) + 4.0;
        }
        return f;
    };
    int mono = 0, nb = 0, nq = 0, nneg = 0;
    for (int j = 0; j < d; ++j) {
        mono += std::max(0, s.A[j]);
        nb += (s.A[j] != -1 && s.B[j] != 0);
        nq += std::abs(s.A[j]);
        nneg += s.A[j] < 0;
    }
    if (s.kind != 2) {
        per_subset += real_poly(0, s.nU) + real_poly(s.nU, s.nF);
        per_subset += std::abs(eU0) + std::abs(eF0) + 1.0 + mono; /* powers (one reciprocal), D, monomial */
        if (M > 0) {
            per_subset += 3.0 + 2.0 * nb; /* U^eU1 F^-eF1, log argument, B_j log t_j */
            trans_subset += 1;
        }
    } else {
        per_subset += real_poly(s.nU + s.nF, s.nG) + real_poly(s.nU + s.nF + s.nG, s.nH);
        per_subset += 2.0 * d * d + 3.0 * d; /* A = diag((1-2t) g) + diag(t(1-t)) H */
        if (d == 1) per_subset += 1;
        else if (d == 2) per_subset += 7;
        else if (d == 3) per_subset += 32;
        else {
            double lu = 0.0;
            for (int c = 0; c < d; ++c) {
                const int rest = d - c - 1;
                lu += 12.0 + rest * (6.0 + 8.0 * rest);
            }
            per_subset += lu;
        }
        per_subset += 3.0 * d; /* z_j and q_j */
        const bool needU = eU0 != 0 || M > 0;
        if (needU) per_subset += cplx_poly(0, s.nU);
        per_subset += cplx_poly(s.nU, s.nF);
        per_subset += 6.0 * (std::abs(eU0) + std::abs(eF0)) + 6.0 + 2.0 + (mono ? 2.0 + mono : 0.0);
        per_subset += 6.0 * nq + 6.0 * nneg;
        if (M > 0) {
            int nlq = 0;
            for (int j = 0; j < d; ++j) nlq += s.B[j] != 0;
            per_subset += 4.0 + 2.0 * nb + 4.0 * nlq;
            trans_subset += 2 + nlq; /* complex logs of U, F and of the q_j */
        }
    }
    const int nsub = 1 << s.sigma;
    double series = s.sigma * ((M + 1) * (M + 2) / 2 * 2.0 + 2.0 * M);
    series += (M + 1) * (M + 2) / 2 * 4.0 + M * 8.0;
    flops = d * transform_flops(r) + nsub * (per_subset + series) + 4.0 * (M + 1);
    transc = nsub * trans_subset + (M > 0 ? (double)s.sigma : 0.0);
}

struct Packed {
    std::vector<unsigned char> bytes;
};

int pack_table(const Table &t, const double *inv, int n_inv, int order_min, int order_max, int r_for_count,
               std::vector<unsigned char> &out, qmc_info *info) {
    if (n_inv != t.K || (t.K > 0 && !inv)) return QMC_ERR_ARG;
    for (int k = 0; k < t.K; ++k)
        if (!std::isfinite(inv[k])) return QMC_ERR_ARG;
    if (order_max < order_min || order_max - order_min + 1 > QMC_MAX_ORDERS) return QMC_ERR_ARG;
    const int d = t.dim;
    int pre_low;
    std::vector<double> pre;
    gamma_series(t.n_nu - 2 * t.loops, t.loops, QMC_MAX_ORDERS + 3, pre_low, pre);
    {
        double norm = 1.0;
        for (int v : t.nu) norm *= std::tgamma((double)v);
        for (double &x : pre) x /= norm;
    }
    const int kmax = order_max - pre_low;

    struct Work {
        PackedSector ps;
        std::vector<PTerm> terms;
        int cls;
    };
    std::vector<Work> work(t.n_sectors);
    int n_def = 0, n_neg = 0, max_sigma = 0, max_terms = 0, n_slots = 1;
    for (int si = 0; si < t.n_sectors; ++si) {
        const TSector &s = t.sectors[si];
        Work &w = work[si];
        std::memset(&w.ps, 0, sizeof(w.ps));
        auto eval = [&](const std::vector<TTerm> &poly, std::vector<PTerm> &dst, bool &const_ok, int &npos,
                        int &nneg) {
            const_ok = false;
            npos = nneg = 0;
            for (const TTerm &term : poly) {
                double v = term.c[0];
                for (int k = 0; k < t.K; ++k) v += term.c[1 + k] * inv[k];
                if (v == 0.0) continue;
                PTerm p;
                p.c = v;
                std::memcpy(p.e, term.e, 8);
                bool zero = true;
                for (int j = 0; j < d; ++j) zero &= p.e[j] == 0;
                const_ok |= zero;
                npos += v > 0;
                nneg += v < 0;
                dst.push_back(p);
            }
        };
        std::vector<PTerm> U, F;
        bool cu, cf;
        int pu, nu_, pf, nf;
        eval(s.U, U, cu, pu, nu_);
        eval(s.F, F, cf, pf, nf);
        if (!cu || !cf) return QMC_ERR_KINEMATICS;
        const int kind = (nf == 0) ? 0 : (pf == 0 ? 1 : 2);
        PackedSector &ps = w.ps;
        ps.kind = kind;
        ps.D = s.D;
        ps.Df = (float)s.D;
        ps.orig_index = si;
        int sigma = 0, mask = 0;
        bool taylor = false;
        for (int j = 0; j < d; ++j) {
            ps.A[j] = s.A[j];
            ps.B[j] = s.B[j];
            if (s.A[j] <= -1) {
                ++sigma;
                mask |= 1 << j;
            }
            taylor |= s.A[j] <= -2;
        }
        /* alpha <= -2 (Eq. 11 with p > 0): undeformed sectors with at most QMC_TAYLOR_MAX_Z singular variables */
        if (taylor && (kind == 2 || sigma > QMC_TAYLOR_MAX_Z)) return QMC_ERR_UNSUPPORTED;
        ps.taylor = taylor ? 1 : 0;
        ps.sigma = sigma;
        ps.sing_mask = mask;
        ps.M = kmax + sigma;
        if (ps.M < 0) ps.M = 0; /* nothing at or below the requested orders: leading slot only */
        if (ps.M + 1 > QMC_MAX_SLOTS) return QMC_ERR_UNSUPPORTED;
        n_slots = std::max(n_slots, ps.M + 1);
        max_sigma = std::max(max_sigma, sigma);
        w.terms = U;
        w.terms.insert(w.terms.end(), F.begin(), F.end());
        ps.nU = (int)U.size();
        ps.nF = (int)F.size();
        if (kind == 2) {
            /* gradient polynomials dF/dt_j and Hessian d2F/dt_j dt_k (j <= k) by the power rule */
            std::vector<std::vector<PTerm>> G(d);
            for (const PTerm &p : F)
                for (int j = 0; j < d; ++j)
                    if (p.e[j] > 0) {
                        PTerm q = p;
                        q.c = p.c * p.e[j];
                        q.e[j] -= 1;
                        G[j].push_back(q);
                    }
            int off = 0;
            for (int j = 0; j < d; ++j) {
                ps.gstart[j] = (int16_t)off;
                off += (int)G[j].size();
                w.terms.insert(w.terms.end(), G[j].begin(), G[j].end());
            }
            ps.gstart[d] = (int16_t)off;
            ps.nG = off;
            off = 0;
            int pidx = 0;
            for (int j = 0; j < d; ++j)
                for (int k = j; k < d; ++k) {
                    ps.hstart[pidx++] = (int16_t)off;
                    for (const PTerm &p : G[j])
                        if (p.e[k] > 0) {
                            PTerm q = p;
                            q.c = p.c * p.e[k];
                            q.e[k] -= 1;
                            w.terms.push_back(q);
                            ++off;
                        }
                }
            ps.hstart[pidx] = (int16_t)off;
            ps.nH = off;
            ++n_def;
        } else if (kind == 1) {
            ++n_neg;
        }
        ps.n_terms = (int)w.terms.size();
        if (ps.n_terms > QMC_MAX_SECTOR_TERMS || ps.nG > 32767 || ps.nH > 32767) return QMC_ERR_UNSUPPORTED;
        max_terms = std::max(max_terms, ps.n_terms);
        w.cls = taylor ? 2 : (kind == 2 ? 1 : 0);
        double fl, tr;
        sector_work(ps, w.terms.data(), d, r_for_count, t.eU0, t.eF0, fl, tr);
        ps.flops = fl;
        ps.transc = tr;
    }
    /* order: undeformed sectors first, then deformed (stable) */
    std::vector<int> order(t.n_sectors);
    for (int i = 0; i < t.n_sectors; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a].cls < work[b].cls; });

    PackedHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = QMC_PACK_MAGIC;
    h.n_sectors = t.n_sectors;
    h.dim = d;
    h.loops = t.loops;
    h.n_nu = t.n_nu;
    h.n_props = t.n_props;
    h.eU0 = t.eU0;
    h.eU1 = t.eU1;
    h.eF0 = t.eF0;
    h.eF1 = t.eF1;
    h.order_min = order_min;
    h.order_max = order_max;
    h.kmax = kmax;
    h.n_slots = n_slots;
    h.pre_low = pre_low;
    h.n_pre = std::min((int)pre.size(), QMC_MAX_ORDERS + 4);
    for (int k = 0; k < h.n_pre; ++k) h.pre[k] = pre[k];
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        h.class_begin[c] = h.class_end[c] = 0;
        h.class_maxm[c] = 0;
    }
    int64_t n_terms_total = 0;
    double fsum = 0.0, tsum = 0.0;
    for (int pi = 0; pi < t.n_sectors; ++pi) {
        Work &w = work[order[pi]];
        w.ps.term0 = (int32_t)n_terms_total;
        n_terms_total += w.ps.n_terms;
        fsum += w.ps.flops;
        tsum += w.ps.transc;
    }
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        int b = -1, e = -1, mm = 0;
        for (int pi = 0; pi < t.n_sectors; ++pi)
            if (work[order[pi]].cls == c) {
                if (b < 0) b = pi;
                e = pi + 1;
                mm = std::max(mm, work[order[pi]].ps.M);
            }
        h.class_begin[c] = b < 0 ? 0 : b;
        h.class_end[c] = e < 0 ? 0 : e;
        h.class_maxm[c] = mm;
    }
    if (n_terms_total > (int64_t)1 << 30) return QMC_ERR_UNSUPPORTED;
    h.max_terms = max_terms;
    h.n_terms_total = (int32_t)n_terms_total;
    h.sectors_off = sizeof(PackedHeader);
    h.terms_off = h.sectors_off + (int64_t)sizeof(PackedSector) * t.n_sectors;
    h.termsf_off = h.terms_off + (int64_t)sizeof(PackedTerm) * n_terms_total;
    h.total_bytes = h.termsf_off + (int64_t)sizeof(PackedTermF) * n_terms_total;
    h.flops_per_eval = fsum / t.n_sectors;
    h.transc_per_eval = tsum / t.n_sectors;
    h.n_deformed = n_def;
    h.n_negative = n_neg;
    h.max_sigma = max_sigma;
    out.assign((size_t)h.total_bytes, 0);
    std::memcpy(out.data(), &h, sizeof(h));
    for (int pi = 0; pi < t.n_sectors; ++pi) {
        const Work &w = work[order[pi]];
        std::memcpy(out.data() + h.sectors_off + (int64_t)sizeof(PackedSector) * pi, &w.ps, sizeof(PackedSector));
        for (size_t k = 0; k < w.terms.size(); ++k) {
            PackedTerm pt;
            pt.c = w.terms[k].c;
            std::memcpy(pt.e, w.terms[k].e, 8);
            std::memcpy(out.data() + h.terms_off + (int64_t)sizeof(PackedTerm) * (w.ps.term0 + k), &pt, sizeof(pt));
            PackedTermF pf;
            pf.hi = (float)w.terms[k].c;
            pf.lo = (float)(w.terms[k].c - (double)pf.hi);
            std::memcpy(pf.e, w.terms[k].e, 8);
            std::memcpy(out.data() + h.termsf_off + (int64_t)sizeof(PackedTermF) * (w.ps.term0 + k), &pf, sizeof(pf));
        }
    }
    reinterpret_cast<PackedHeader *>(out.data())->family = qmc_family_key(out.data());
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->n_sectors = t.n_sectors;
        info->dim = d;
        info->loops = t.loops;
        info->n_invariants = t.K;
        info->order_min = order_min;
        info->order_max = order_max;
        info->kmax = kmax;
        info->n_slots = n_slots;
        info->n_deformed = n_def;
        info->n_negative = n_neg;
        info->max_sigma = max_sigma;
        info->max_terms = max_terms;
        info->pre_low = pre_low;
        info->n_pre = h.n_pre;
        for (int k = 0; k < h.n_pre; ++k) info->pre[k] = h.pre[k];
        info->packed_bytes = h.total_bytes;
        info->flops_per_eval = h.flops_per_eval;
        info->transcendentals_per_eval = h.transc_per_eval;
    }
    return QMC_OK;
}

}  // namespace

int qmci::validate_table(const void *blob, size_t bytes) {
    Table t;
    try {
        return parse_table(blob, bytes, t);
    } catch (...) {
        return QMC_ERR_TABLE;
    }
}

extern "C" {

const char *qmc_strerror(int s) {
    switch (s) {
        case QMC_OK: return "ok";
        case QMC_PENDING: return "pending";
        case QMC_ERR_ARG: return "invalid argument";
        case QMC_ERR_TABLE: return "malformed sector table";
        case QMC_ERR_UNSUPPORTED: return "unsupported by the kernels";
        case QMC_ERR_KINEMATICS: return "kinematics make a leading coefficient vanish";
        case QMC_ERR_CUDA: return "CUDA runtime error";
        case QMC_ERR_MEMORY: return "device memory budget or buffer capacity exceeded";
        case QMC_ERR_DEFORMATION: return "contour deformation keeps failing the sign check";
        case QMC_ERR_TIMEOUT: return "time limit reached";
        case QMC_ERR_CANCELLED: return "cancelled";
        case QMC_ERR_NOT_FOUND: return "unknown id";
        case QMC_ERR_NO_DEVICE: return "no CUDA device";
        case QMC_ERR_NOT_CONVERGED: return "lattice ladder exhausted before the requested accuracy";
        case QMC_ERR_CODEGEN: return "run-time compilation of the generated evaluator failed";
        case QMC_ERR_NONFINITE: return "a sector's FP64 sums are not finite";
        default: return "unknown status";
    }
}

int qmc_version(void) { return 100; }

int qmc_prepare(const void *table, size_t table_bytes, const double *invariants, int32_t n_invariants,
                int32_t order_min, int32_t order_max, void *packed, size_t packed_capacity, qmc_info *info) {
    try {
        Table t;
        int rc = parse_table(table, table_bytes, t);
        if (rc) return rc;
        std::vector<unsigned char> img;
        rc = pack_table(t, invariants, n_invariants, order_min, order_max, 3, img, info);
        if (rc) return rc;
        if (packed) {
            if (packed_capacity < img.size()) return QMC_ERR_MEMORY;
            std::memcpy(packed, img.data(), img.size());
        }
        return QMC_OK;
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    } catch (...) {
        return QMC_ERR_TABLE;
    }
}

int qmc_sector_desc_get(const void *packed, int32_t sector, qmc_sector_desc *out) {
    const PackedHeader *h = header_of(packed);
    if (!h || !out || sector < 0 || sector >= h->n_sectors) return QMC_ERR_ARG;
    const PackedSector *ps = sectors_of(packed);
    for (int i = 0; i < h->n_sectors; ++i)
        if (ps[i].orig_index == sector) {
            out->kind = ps[i].kind;
            out->sigma = ps[i].sigma;
            out->n_slots = ps[i].M + 1;
            out->n_terms = ps[i].n_terms;
            out->flops = ps[i].flops;
            return QMC_OK;
        }
    return QMC_ERR_ARG;
}

}  // extern "C"
