/*
 * Host runtime of the qmcfi library: sector-table parsing and validation, packing of the device image,
 * the Gamma prefactor series, launch planning for the evaluation kernels, combination of per-shift sums
 * into Laurent coefficients with errors, and the integrate-to-accuracy loop of a context.
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103:
 * Sec. II (Eqs. 2, 9-14) fixes the sector integrand, Sec. III (Eqs. 16-21) the shifted-lattice estimator.
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
#include "qmc_internal.h"

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
            if (s.A[j] < -1 || s.A[j] > QMC_MAX_EXP) return s.A[j] < -1 ? QMC_ERR_UNSUPPORTED : QMC_ERR_TABLE;
            if (s.A[j] == -1 && s.B[j] == 0) return QMC_ERR_TABLE; /* unregulated endpoint singularity */
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
        for (int j = 0; j < d; ++j) {
            ps.A[j] = s.A[j];
            ps.B[j] = s.B[j];
            if (s.A[j] == -1) {
                ++sigma;
                mask |= 1 << j;
            }
        }
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
        w.cls = kind == 2 ? 1 : 0;
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

const PackedHeader *header_of(const void *packed) {
    if (!packed) return nullptr;
    const PackedHeader *h = static_cast<const PackedHeader *>(packed);
    return h->magic == QMC_PACK_MAGIC ? h : nullptr;
}

const PackedSector *sectors_of(const void *packed) {
    const PackedHeader *h = header_of(packed);
    return reinterpret_cast<const PackedSector *>(static_cast<const unsigned char *>(packed) + h->sectors_off);
}

/* ------------------------------------------------------------------ launch planning */
struct Plan {
    int block, P;
    int64_t chunks;
    int64_t items[QMC_N_CLASSES];
    int64_t item_off[QMC_N_CLASSES];
    int64_t total_items;
    size_t partial_bytes, fail_bytes, counter_bytes, total_bytes;
};

int make_plan(const PackedHeader *h, const qmc_pass *p, Plan &pl) {
    if (!h || !p) return QMC_ERR_ARG;
    if (p->lattice.n < 2 || p->lattice.n >= ((int64_t)1 << 31)) return QMC_ERR_ARG;
    if (p->n_shifts < 1 || p->n_shifts > 4096) return QMC_ERR_ARG;
    if (p->transform_r < 0 || p->transform_r > 3) return QMC_ERR_ARG;
    if (p->precision != QMC_PREC_FP64 && p->precision != QMC_PREC_MIXED) return QMC_ERR_ARG;
    pl.block = p->block ? p->block : 128;
    if (pl.block < 32 || pl.block > 256 || pl.block % 32) return QMC_ERR_ARG;
    pl.P = p->points_per_thread ? p->points_per_thread : (p->precision == QMC_PREC_MIXED ? 16 : 8);
    if (pl.P < 1 || pl.P > 64) return QMC_ERR_ARG;
    for (int j = 0; j < h->dim; ++j)
        if (p->lattice.z[j] == 0 || (int64_t)p->lattice.z[j] >= p->lattice.n) return QMC_ERR_ARG;
    const int64_t C = (int64_t)pl.block * pl.P;
    pl.chunks = (p->lattice.n + C - 1) / C;
    int64_t off = 0;
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        const int64_t ns = h->class_end[c] - h->class_begin[c];
        pl.items[c] = ns * p->n_shifts * pl.chunks;
        pl.item_off[c] = off;
        off += pl.items[c];
    }
    pl.total_items = off;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    pl.partial_bytes = up((size_t)pl.total_items * h->n_slots * 2 * sizeof(double));
    pl.fail_bytes = up((size_t)pl.total_items * sizeof(uint32_t));
    /* work counters: per class and precision, plus one per launch of the parameter-table FP32 kernel */
    pl.counter_bytes = up((2 * QMC_N_CLASSES + QMC_MAX_GROUP_LAUNCHES) * sizeof(unsigned long long));
    pl.total_bytes = pl.partial_bytes + pl.fail_bytes + pl.counter_bytes;
    return QMC_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA; }

/* ------------------------------------------------------------------ shifts */
void splitmix_shifts(uint64_t seed, int m, std::vector<double> &out) {
    out.resize((size_t)m * 6);
    uint64_t state = seed;
    for (size_t k = 0; k < out.size(); ++k) {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[k] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}

}  // namespace

/* ====================================================================== C ABI */
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

size_t qmc_scratch_bytes(const void *packed, const qmc_pass *pass) {
    Plan pl;
    if (make_plan(header_of(packed), pass, pl) != QMC_OK) return 0;
    return pl.total_bytes;
}

}  // extern "C"

namespace {

/* Validates the arguments shared by the evaluation entry points and lays out the scratch buffer. */
struct Scratch {
    double *partials;
    uint32_t *pfails;
    unsigned long long *counters;
};

int check_pass(const PackedHeader *h, const void *packed_dev, const qmc_pass *pass, void *scratch_dev,
               size_t scratch_bytes, Plan &pl, Scratch &sc) {
    if (!h || !packed_dev || !pass || !scratch_dev) return QMC_ERR_ARG;
    if (((uintptr_t)scratch_dev & 255) || ((uintptr_t)packed_dev & 15)) return QMC_ERR_ARG;
    int rc = make_plan(h, pass, pl);
    if (rc) return rc;
    if (scratch_bytes < pl.total_bytes) return QMC_ERR_MEMORY;
    unsigned char *scr = static_cast<unsigned char *>(scratch_dev);
    sc.partials = reinterpret_cast<double *>(scr);
    sc.pfails = reinterpret_cast<uint32_t *>(scr + pl.partial_bytes);
    sc.counters = reinterpret_cast<unsigned long long *>(scr + pl.partial_bytes + pl.fail_bytes);
    return QMC_OK;
}

int class_maxm(const PackedHeader *h, int c) { return h->class_maxm[c] == 0 ? 0 : (h->class_maxm[c] <= 2 ? 2 : 4); }

/* FP32 evaluation with the sector tables in the kernel's parameter block: the class's sectors are cut into
   groups of at most QMC_PARAM_SECTORS sectors and QMC_PARAM_TERMS terms, one launch per group, each with its own
   work counter and its slice of the class's item range (items of a sector are contiguous). */
int launch_param_groups(const PackedHeader *h, const void *packed_host, int c, int maxm, const EvalArgs &base,
                        const Plan &pl, const Scratch &sc, int sms, int &group_launches, void *stream) {
    const unsigned char *img = static_cast<const unsigned char *>(packed_host);
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(img + h->sectors_off);
    const PackedTermF *tf = reinterpret_cast<const PackedTermF *>(img + h->termsf_off);
    int per_sm = 0;
    int rc = qmc_eval_param_blocks_per_sm(h->dim, c == 1, maxm, pl.block, &per_sm);
    if (rc) return rc;
    if (per_sm < 1) return QMC_ERR_UNSUPPORTED;
    std::unique_ptr<ParamGroup> g(new ParamGroup());
    const int64_t per_sector = (int64_t)base.m * base.chunks;
    int s0 = h->class_begin[c];
    while (s0 < h->class_end[c]) {
        std::memset(g.get(), 0, sizeof(ParamGroup));
        int ns = 0, nt = 0;
        while (s0 + ns < h->class_end[c] && ns < QMC_PARAM_SECTORS && nt + ps[s0 + ns].n_terms <= QMC_PARAM_TERMS) {
            const PackedSector &q = ps[s0 + ns];
            ParamSector &d = g->sec[ns];
            d.kind = q.kind;
            d.sigma = q.sigma;
            d.sing_mask = q.sing_mask;
            d.M = q.M;
            for (int j = 0; j < 6; ++j) {
                d.A[j] = q.A[j];
                d.B[j] = q.B[j];
            }
            d.nU = q.nU;
            d.nF = q.nF;
            d.nG = q.nG;
            d.nH = q.nH;
            d.tbase = nt;
            d.orig_index = q.orig_index;
            d.psec = s0 + ns;
            d.Df = q.Df;
            for (int j = 0; j < 8; ++j) d.gstart[j] = q.gstart[j];
            for (int j = 0; j < 24; ++j) d.hstart[j] = q.hstart[j];
            std::memcpy(&g->terms[nt], tf + q.term0, sizeof(PackedTermF) * q.n_terms);
            nt += q.n_terms;
            ++ns;
        }
        if (ns == 0) return QMC_ERR_UNSUPPORTED;
        if (group_launches >= QMC_MAX_GROUP_LAUNCHES) return QMC_ERR_UNSUPPORTED;
        g->n_sect = ns;
        g->n_terms = nt;
        EvalArgs a = base;
        const int64_t first = (int64_t)(s0 - h->class_begin[c]) * per_sector;
        a.sector_begin = s0;
        a.n_sect = ns;
        a.total_items = (int64_t)ns * per_sector;
        a.partials = base.partials + first * h->n_slots * 2;
        a.part_fails = base.part_fails + first;
        a.counter = sc.counters + 2 * QMC_N_CLASSES + group_launches;
        ++group_launches;
        int64_t grid = (int64_t)sms * per_sm;
        if (grid > a.total_items) grid = a.total_items;
        rc = qmc_launch_eval_param(h->dim, c == 1, maxm, a, *g, (int)grid, pl.block, stream);
        if (rc) return rc;
        s0 += ns;
    }
    return QMC_OK;
}

}  // namespace

extern "C" {

int qmc_eval_partials(const void *packed_host, const void *packed_dev, const qmc_pass *pass,
                      const double *shifts_dev, const double *lambda_dev, void *scratch_dev, size_t scratch_bytes,
                      void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!shifts_dev || !lambda_dev) return QMC_ERR_ARG;
    Plan pl;
    Scratch sc;
    int rc = check_pass(h, packed_dev, pass, scratch_dev, scratch_bytes, pl, sc);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = cuda_status(cudaMemsetAsync(sc.counters, 0,
                                     (2 * QMC_N_CLASSES + QMC_MAX_GROUP_LAUNCHES) * sizeof(unsigned long long), st));
    if (rc) return rc;
    int sms = 0;
    rc = qmc_device_sm_count(&sms);
    if (rc) return rc;
    const size_t smem = sizeof(PackedSector) + (size_t)h->max_terms * sizeof(PackedTerm);
    int group_launches = 0;
    /* FP64 pass: one kernel per class.  Mixed pass: the FP32 kernel takes the sectors marked 1 in
       pass->sector_precision (all when it is null), the FP64 kernel the others; both share the item space. */
    const bool mixed = pass->precision == QMC_PREC_MIXED;
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        if (pl.items[c] == 0) continue;
        const int maxm = class_maxm(h, c);
        for (int prec = 0; prec < 2; ++prec) {
            const int kprec = prec == 0 ? QMC_PREC_FP64 : QMC_PREC_MIXED;
            if (!mixed && prec == 1) continue;
            if (mixed && prec == 0 && !pass->sector_precision) continue;
            EvalArgs a;
            std::memset(&a, 0, sizeof(a));
            a.packed = static_cast<const unsigned char *>(packed_dev);
            a.sectors_off = h->sectors_off;
            a.terms_off = h->terms_off;
            a.termsf_off = h->termsf_off;
            a.sector_begin = h->class_begin[c];
            a.n_sect = h->class_end[c] - h->class_begin[c];
            a.m = pass->n_shifts;
            a.r = pass->transform_r;
            a.P = pl.P;
            a.n_slots = h->n_slots;
            a.n = (uint32_t)pass->lattice.n;
            for (int j = 0; j < QMC_MAX_DIM; ++j) {
                a.z[j] = j < h->dim ? pass->lattice.z[j] : 0;
                a.zstep[j] = (uint32_t)(((uint64_t)pl.block * a.z[j]) % (uint64_t)pass->lattice.n);
            }
            a.invn = 1.0 / (double)pass->lattice.n;
            a.chunks = pl.chunks;
            a.total_items = pl.items[c];
            a.shifts = shifts_dev;
            a.lambda = lambda_dev;
            a.partials = sc.partials + pl.item_off[c] * h->n_slots * 2;
            a.part_fails = sc.pfails + pl.item_off[c];
            a.counter = sc.counters + 2 * c + prec;
            a.eU0 = h->eU0;
            a.eU1 = h->eU1;
            a.eF0 = h->eF0;
            a.eF1 = h->eF1;
            a.smem_bytes = (int)smem;
            a.sector_prec = mixed ? pass->sector_precision : nullptr;
            a.want_prec = prec;
            if (prec == 1 && h->max_terms <= QMC_PARAM_TERMS) {
                /* FP32 with the tables in kernel parameters: groups of consecutive sectors per launch */
                rc = launch_param_groups(h, packed_host, c, maxm, a, pl, sc, sms, group_launches, stream);
                if (rc) return rc;
                continue;
            }
            int per_sm = 0;
            rc = qmc_eval_blocks_per_sm(h->dim, c == 1, maxm, kprec, pl.block, (int)smem, &per_sm);
            if (rc) return rc;
            if (per_sm < 1) return QMC_ERR_UNSUPPORTED;
            int64_t grid = pass->grid > 0 ? pass->grid : (int64_t)sms * per_sm;
            if (grid > pl.items[c]) grid = pl.items[c];
            rc = qmc_launch_eval(h->dim, c == 1, maxm, kprec, a, (int)grid, pl.block, stream);
            if (rc) return rc;
        }
    }
    return QMC_OK;
}

int qmc_probe_precision(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
                        const double *lambda_dev, int64_t n_sample, double *out_dev, void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !packed_dev || !pass || !shift_dev || !lambda_dev || !out_dev || n_sample < 1) return QMC_ERR_ARG;
    Plan pl;
    int rc = make_plan(h, pass, pl);
    if (rc) return rc;
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        const int ns = h->class_end[c] - h->class_begin[c];
        if (ns <= 0) continue;
        ProbeArgs a;
        std::memset(&a, 0, sizeof(a));
        a.packed = static_cast<const unsigned char *>(packed_dev);
        a.sectors_off = h->sectors_off;
        a.terms_off = h->terms_off;
        a.termsf_off = h->termsf_off;
        a.sector_begin = h->class_begin[c];
        a.n_sect = ns;
        a.r = pass->transform_r;
        a.n_slots = h->n_slots;
        a.n = (uint32_t)pass->lattice.n;
        for (int j = 0; j < QMC_MAX_DIM; ++j) a.z[j] = j < h->dim ? pass->lattice.z[j] : 0;
        a.invn = 1.0 / (double)pass->lattice.n;
        a.shift = shift_dev;
        a.lambda = lambda_dev;
        a.n_sample = n_sample;
        a.out = out_dev;
        a.eU0 = h->eU0;
        a.eU1 = h->eU1;
        a.eF0 = h->eF0;
        a.eF1 = h->eF1;
        a.smem_bytes = (int)(sizeof(PackedSector) + 2 * (size_t)h->max_terms * sizeof(PackedTerm));
        rc = qmc_launch_probe(h->dim, c == 1, class_maxm(h, c), a, stream);
        if (rc) return rc;
    }
    return QMC_OK;
}

int qmc_reduce_partials(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const void *scratch_dev,
                        size_t scratch_bytes, double *sums_dev, int64_t *fails_dev, void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!sums_dev || !fails_dev) return QMC_ERR_ARG;
    Plan pl;
    Scratch sc;
    int rc = check_pass(h, packed_dev, pass, const_cast<void *>(scratch_dev), scratch_bytes, pl, sc);
    if (rc) return rc;
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        if (pl.items[c] == 0) continue;
        FinalizeArgs f;
        f.packed = static_cast<const unsigned char *>(packed_dev);
        f.sectors_off = h->sectors_off;
        f.sector_begin = h->class_begin[c];
        f.n_sect = h->class_end[c] - h->class_begin[c];
        f.m = pass->n_shifts;
        f.n_slots = h->n_slots;
        f.chunks = pl.chunks;
        f.partials = sc.partials + pl.item_off[c] * h->n_slots * 2;
        f.part_fails = sc.pfails + pl.item_off[c];
        f.sums = sums_dev;
        f.fails = fails_dev;
        rc = qmc_launch_finalize(f, stream);
        if (rc) return rc;
    }
    return QMC_OK;
}

int qmc_eval_sums(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                  const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, double *sums_dev,
                  int64_t *fails_dev, void *stream) {
    if (!sums_dev || !fails_dev) return QMC_ERR_ARG;
    int rc = qmc_eval_partials(packed_host, packed_dev, pass, shifts_dev, lambda_dev, scratch_dev, scratch_bytes,
                               stream);
    if (rc) return rc;
    return qmc_reduce_partials(packed_host, packed_dev, pass, scratch_dev, scratch_bytes, sums_dev, fails_dev, stream);
}

int qmc_eval_points(const void *packed_host, const void *packed_dev, int32_t sector, const qmc_pass *pass,
                    const double *shift_dev, double lambda, const int64_t *idx_dev, int64_t npts, double *out_dev,
                    int32_t *fails_dev, void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !packed_dev || !pass || !shift_dev || !idx_dev || !out_dev || !fails_dev || npts < 0) return QMC_ERR_ARG;
    if (sector < 0 || sector >= h->n_sectors) return QMC_ERR_ARG;
    Plan pl;
    int rc = make_plan(h, pass, pl);
    if (rc) return rc;
    if (npts == 0) return QMC_OK;
    const PackedSector *ps = sectors_of(packed_host);
    int psec = -1;
    for (int i = 0; i < h->n_sectors; ++i)
        if (ps[i].orig_index == sector) psec = i;
    PointArgs a;
    std::memset(&a, 0, sizeof(a));
    a.packed = static_cast<const unsigned char *>(packed_dev);
    a.sectors_off = h->sectors_off;
    a.terms_off = h->terms_off;
    a.sector = psec;
    a.r = pass->transform_r;
    a.n_slots = h->n_slots;
    a.n = (uint32_t)pass->lattice.n;
    for (int j = 0; j < QMC_MAX_DIM; ++j) a.z[j] = j < h->dim ? pass->lattice.z[j] : 0;
    a.invn = 1.0 / (double)pass->lattice.n;
    a.shift = shift_dev;
    a.lambda = lambda;
    a.idx = idx_dev;
    a.npts = npts;
    a.out = out_dev;
    a.fails = fails_dev;
    a.eU0 = h->eU0;
    a.eU1 = h->eU1;
    a.eF0 = h->eF0;
    a.eF1 = h->eF1;
    a.smem_bytes = (int)(sizeof(PackedSector) + (size_t)ps[psec].n_terms * sizeof(PackedTerm));
    const int cls = ps[psec].kind == 2 ? 1 : 0;
    const int mm = h->class_maxm[cls];
    const int maxm = mm == 0 ? 0 : (mm <= 2 ? 2 : 4);
    return qmc_launch_points(h->dim, cls, maxm, pass->precision, a, stream);
}

int qmc_builtin_lattices(qmc_lattice *out, int32_t cap) {
    for (int i = 0; i < QMC_BUILTIN_LATTICES && i < cap && out; ++i) {
        out[i].n = qmc_builtin_lattice[i].n;
        for (int j = 0; j < QMC_MAX_DIM; ++j) out[i].z[j] = qmc_builtin_lattice[i].z[j];
    }
    return QMC_BUILTIN_LATTICES;
}

int qmc_combine(const void *packed_host, const qmc_pass *pass, const double *sums, double *Q, double *mean,
                double *err) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !pass || !sums || !Q || !mean || !err || pass->n_shifts < 1 || pass->lattice.n < 1) return QMC_ERR_ARG;
    const int m = pass->n_shifts, ns = h->n_slots;
    const int nord = h->order_max - h->order_min + 1;
    const PackedSector *ps = sectors_of(packed_host);
    /* sector-sum orders run from -max_sigma to kmax */
    const int lo = -h->max_sigma;
    const int width = h->kmax - lo + 1;
    const double invn = 1.0 / (double)pass->lattice.n;
    std::vector<double> tr(width), ti(width);
    for (int k = 0; k < m; ++k) {
        std::fill(tr.begin(), tr.end(), 0.0);
        std::fill(ti.begin(), ti.end(), 0.0);
        for (int pi = 0; pi < h->n_sectors; ++pi) {
            const PackedSector &s = ps[pi];
            const double *v = sums + ((size_t)s.orig_index * m + k) * ns * 2;
            /* kind 1: multiply by exp(i pi eF(eps)) = (-1)^{eF0} sum_n (i pi eF1 eps)^n / n! */
            std::vector<double> phr(ns, 0.0), phi(ns, 0.0);
            if (s.kind == 1) {
                double c = (h->eF0 % 2) ? -1.0 : 1.0;
                for (int n = 0; n < ns; ++n) {
                    /* (i pi eF1)^n / n! */
                    const int q = n % 4;
                    const double mag = c;
                    phr[n] = (q == 0) ? mag : (q == 2 ? -mag : 0.0);
                    phi[n] = (q == 1) ? mag : (q == 3 ? -mag : 0.0);
                    c *= M_PI * h->eF1 / (n + 1);
                }
            } else {
                phr[0] = 1.0;
            }
            for (int n = 0; n <= s.M; ++n) {
                double ar = 0.0, ai = 0.0;
                for (int q = 0; q <= n; ++q) {
                    ar += phr[q] * v[2 * (n - q)] - phi[q] * v[2 * (n - q) + 1];
                    ai += phr[q] * v[2 * (n - q) + 1] + phi[q] * v[2 * (n - q)];
                }
                const int order = n - s.sigma;
                if (order < lo || order > h->kmax) continue;
                tr[order - lo] += ar * invn;
                ti[order - lo] += ai * invn;
            }
        }
        for (int o = h->order_min; o <= h->order_max; ++o) {
            double qr = 0.0, qi = 0.0;
            for (int a = lo; a <= h->kmax; ++a) {
                const int pidx = o - a - h->pre_low;
                if (pidx < 0 || pidx >= h->n_pre) continue;
                qr += h->pre[pidx] * tr[a - lo];
                qi += h->pre[pidx] * ti[a - lo];
            }
            Q[((size_t)k * nord + (o - h->order_min)) * 2] = qr;
            Q[((size_t)k * nord + (o - h->order_min)) * 2 + 1] = qi;
        }
    }
    for (int o = 0; o < nord; ++o) {
        double mr = 0.0, mi = 0.0;
        for (int k = 0; k < m; ++k) {
            mr += Q[((size_t)k * nord + o) * 2];
            mi += Q[((size_t)k * nord + o) * 2 + 1];
        }
        mr /= m;
        mi /= m;
        double vr = 0.0, vi = 0.0;
        for (int k = 0; k < m; ++k) {
            const double dr = Q[((size_t)k * nord + o) * 2] - mr, di = Q[((size_t)k * nord + o) * 2 + 1] - mi;
            vr += dr * dr;
            vi += di * di;
        }
        mean[2 * o] = mr;
        mean[2 * o + 1] = mi;
        const double den = m > 1 ? (double)m * (m - 1) : 1.0;
        err[2 * o] = m > 1 ? std::sqrt(vr / den) : INFINITY;
        err[2 * o + 1] = m > 1 ? std::sqrt(vi / den) : INFINITY;
    }
    return QMC_OK;
}

}  // extern "C"

/* ====================================================================== context */
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Integral {
    std::vector<unsigned char> table;
    std::vector<unsigned char> packed;  /* host image; empty until kinematics are set */
    DevBuf dpacked;
    qmc_info info;
};

struct qmc_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    std::map<int32_t, Integral> integrals;
    int32_t next_id = 1;
    DevBuf scratch, sums, fails, shifts, lambda, hpacked, prec, probe;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::mutex mu;
};

namespace {

int dev_reserve(qmc_ctx *c, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return QMC_OK;
    if (b.p) {
        cudaFree(b.p);
        c->used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    bytes = (bytes + 4095) & ~size_t(4095);
    if (c->used + bytes > c->budget) return QMC_ERR_MEMORY;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return QMC_ERR_MEMORY;
    b.bytes = bytes;
    c->used += bytes;
    return QMC_OK;
}

void dev_release(qmc_ctx *c, DevBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        c->used -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

}  // namespace

extern "C" {

int qmc_create(qmc_ctx **out, int32_t device, size_t mem_budget, void *stream) {
    if (!out) return QMC_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) return QMC_ERR_NO_DEVICE;
    if (device < 0 || device >= n) return QMC_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return QMC_ERR_CUDA;
    qmc_ctx *c = new (std::nothrow) qmc_ctx();
    if (!c) return QMC_ERR_MEMORY;
    c->device = device;
    c->budget = mem_budget ? mem_budget : ((size_t)1 << 30);
    c->stream = (cudaStream_t)stream;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        delete c;
        return QMC_ERR_CUDA;
    }
    *out = c;
    return QMC_OK;
}

int qmc_destroy(qmc_ctx *c) {
    if (!c) return QMC_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->integrals) dev_release(c, kv.second.dpacked);
    dev_release(c, c->scratch);
    dev_release(c, c->sums);
    dev_release(c, c->fails);
    dev_release(c, c->shifts);
    dev_release(c, c->lambda);
    dev_release(c, c->hpacked);
    dev_release(c, c->prec);
    dev_release(c, c->probe);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    delete c;
    return QMC_OK;
}

int qmc_load_sectors(qmc_ctx *c, const void *table, size_t bytes, int32_t *id) {
    if (!c || !table || !id) return QMC_ERR_ARG;
    Table t;
    int rc;
    try {
        rc = parse_table(table, bytes, t);
    } catch (...) {
        return QMC_ERR_TABLE;
    }
    if (rc) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    Integral &I = c->integrals[c->next_id];
    I.table.assign(static_cast<const unsigned char *>(table), static_cast<const unsigned char *>(table) + bytes);
    *id = c->next_id++;
    return QMC_OK;
}

int qmc_set_kinematics(qmc_ctx *c, int32_t id, const double *inv, int32_t n_inv, int32_t order_min,
                       int32_t order_max) {
    if (!c) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->integrals.find(id);
    if (it == c->integrals.end()) return QMC_ERR_NOT_FOUND;
    Integral &I = it->second;
    qmc_info info;
    int rc = qmc_prepare(I.table.data(), I.table.size(), inv, n_inv, order_min, order_max, nullptr, 0, &info);
    if (rc) return rc;
    std::vector<unsigned char> img((size_t)info.packed_bytes);
    rc = qmc_prepare(I.table.data(), I.table.size(), inv, n_inv, order_min, order_max, img.data(), img.size(), &info);
    if (rc) return rc;
    cudaSetDevice(c->device);
    rc = dev_reserve(c, I.dpacked, img.size());
    if (rc) return rc;
    rc = cuda_status(cudaMemcpyAsync(I.dpacked.p, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream));
    if (rc) return rc;
    rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    I.packed.swap(img);
    I.info = info;
    return QMC_OK;
}

int qmc_integrate(qmc_ctx *c, int32_t id, const qmc_options *opt, qmc_result *res) {
    if (!c || !opt || !res) return QMC_ERR_ARG;
    std::memset(res, 0, sizeof(*res));
    const auto t0 = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->integrals.find(id);
    if (it == c->integrals.end()) return res->status = QMC_ERR_NOT_FOUND;
    Integral &I = it->second;
    if (I.packed.empty()) return res->status = QMC_ERR_ARG;
    const PackedHeader *h = header_of(I.packed.data());
    const int m = opt->n_shifts > 0 ? opt->n_shifts : 16;
    if (m < 2 || m > 4096) return res->status = QMC_ERR_ARG;
    const int nord = h->order_max - h->order_min + 1;
    res->order_min = h->order_min;
    res->n_orders = nord;
    cudaSetDevice(c->device);
    /* lattice ladder */
    std::vector<qmc_lattice> ladder;
    if (opt->n_lattices > 0) {
        if (!opt->lattices) return res->status = QMC_ERR_ARG;
        ladder.assign(opt->lattices, opt->lattices + opt->n_lattices);
    } else {
        for (int i = std::max(0, opt->ladder_start); i < QMC_BUILTIN_LATTICES; ++i) {
            qmc_lattice L;
            L.n = qmc_builtin_lattice[i].n;
            for (int j = 0; j < QMC_MAX_DIM; ++j) L.z[j] = qmc_builtin_lattice[i].z[j];
            ladder.push_back(L);
        }
    }
    /* shifts (Eq. 18): explicit, or splitmix64 from the seed */
    std::vector<double> shifts;
    if (opt->shifts) shifts.assign(opt->shifts, opt->shifts + (size_t)m * 6);
    else splitmix_shifts(opt->seed, m, shifts);
    int rc = dev_reserve(c, c->shifts, shifts.size() * sizeof(double));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(c->shifts.p, shifts.data(), shifts.size() * sizeof(double),
                                              cudaMemcpyHostToDevice, c->stream));
    const int ns = h->n_sectors;
    std::vector<double> lam(ns, opt->lambda > 0 ? opt->lambda : 0.5);
    std::vector<int> halv(ns, 0);
    const int max_h = opt->max_halvings > 0 ? opt->max_halvings : 6;
    if (!rc) rc = dev_reserve(c, c->lambda, ns * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->sums, (size_t)ns * m * h->n_slots * 2 * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->fails, (size_t)ns * m * sizeof(int64_t));
    if (rc) return res->status = rc;
    std::vector<double> sums((size_t)ns * m * h->n_slots * 2), Q((size_t)m * nord * 2), mean(nord * 2), err(nord * 2);
    std::vector<int64_t> fails((size_t)ns * m);
    const bool mixed = opt->precision == QMC_PREC_MIXED;
    std::vector<int32_t> prec(ns, 1);
    bool probe_due = mixed;
    if (mixed) {
        rc = dev_reserve(c, c->prec, ns * sizeof(int32_t));
        if (!rc) rc = dev_reserve(c, c->probe, (size_t)ns * h->n_slots * 4 * sizeof(double));
        if (rc) return res->status = rc;
    }
    int status = QMC_ERR_NOT_CONVERGED;
    float kernel_ms_total = 0.f;
    for (const qmc_lattice &L : ladder) {
        if (opt->max_n > 0 && L.n > opt->max_n) break;
        qmc_pass pass;
        std::memset(&pass, 0, sizeof(pass));
        pass.lattice = L;
        pass.n_shifts = m;
        pass.transform_r = opt->transform_r > 0 ? opt->transform_r : 3;
        pass.precision = opt->precision;
        pass.block = opt->block;
        pass.points_per_thread = opt->points_per_thread;
        pass.sector_precision = mixed ? (const int32_t *)c->prec.p : nullptr;
        const size_t need = qmc_scratch_bytes(I.packed.data(), &pass);
        if (!need) return res->status = QMC_ERR_ARG;
        rc = dev_reserve(c, c->scratch, need);
        if (rc) return res->status = rc;
        for (;;) {
            rc = cuda_status(cudaMemcpyAsync(c->lambda.p, lam.data(), ns * sizeof(double), cudaMemcpyHostToDevice,
                                             c->stream));
            if (!rc && probe_due) {
                /* FP32 budget: sectors whose FP32 values on the probe sample deviate from FP64 by more than
                   fp32_budget * rel_tol (L1, any order) are evaluated in FP64 */
                const int64_t nsamp = opt->probe_samples > 0 ? opt->probe_samples : 4096;
                const double budget = (opt->fp32_budget > 0 ? opt->fp32_budget : 0.1) * opt->rel_tol;
                std::vector<double> pr((size_t)ns * h->n_slots * 4);
                rc = qmc_probe_precision(I.packed.data(), I.dpacked.p, &pass, (const double *)c->shifts.p,
                                         (const double *)c->lambda.p, nsamp, (double *)c->probe.p, c->stream);
                if (!rc)
                    rc = cuda_status(cudaMemcpyAsync(pr.data(), c->probe.p, pr.size() * sizeof(double),
                                                     cudaMemcpyDeviceToHost, c->stream));
                if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
                if (rc) return res->status = rc;
                res->fp64_reruns = 0;
                for (int s2 = 0; s2 < ns; ++s2) {
                    bool bad = false;
                    for (int o = 0; o < h->n_slots; ++o) {
                        const double *v = &pr[((size_t)s2 * h->n_slots + o) * 4];
                        if (v[1] > budget * v[0] || !std::isfinite(v[1])) bad = true;
                    }
                    prec[s2] = bad ? 0 : 1;
                    res->fp64_reruns += bad;
                }
                rc = cuda_status(cudaMemcpyAsync(c->prec.p, prec.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice,
                                                 c->stream));
                probe_due = false;
            }
            if (!rc) rc = cuda_status(cudaEventRecord(c->ev0, c->stream));
            if (!rc)
                rc = qmc_eval_sums(I.packed.data(), I.dpacked.p, &pass, (const double *)c->shifts.p,
                                   (const double *)c->lambda.p, c->scratch.p, c->scratch.bytes, (double *)c->sums.p,
                                   (int64_t *)c->fails.p, c->stream);
            if (!rc) rc = cuda_status(cudaEventRecord(c->ev1, c->stream));
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(sums.data(), c->sums.p, sums.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost, c->stream));
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(fails.data(), c->fails.p, fails.size() * sizeof(int64_t),
                                                 cudaMemcpyDeviceToHost, c->stream));
            if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
            if (rc) return res->status = rc;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->ev0, c->ev1);
            kernel_ms_total += ms;
            res->passes += 1;
            res->evals += (int64_t)ns * m * L.n;
            /* sign check of Eq. (14): halve lambda of failing sectors and repeat this lattice size */
            bool again = false;
            for (int s = 0; s < ns; ++s) {
                int64_t f = 0;
                for (int k = 0; k < m; ++k) f += fails[(size_t)s * m + k];
                if (f > 0) {
                    res->sign_failures += (int32_t)std::min<int64_t>(f, INT32_MAX);
                    if (halv[s] >= max_h) {
                        res->kernel_ms = kernel_ms_total;
                        return res->status = QMC_ERR_DEFORMATION;
                    }
                    lam[s] *= 0.5;
                    halv[s] += 1;
                    res->lambda_halvings += 1;
                    again = true;
                }
            }
            if (!again) break;
            probe_due = mixed;
        }
        qmc_combine(I.packed.data(), &pass, sums.data(), Q.data(), mean.data(), err.data());
        res->n_final = L.n;
        double vmax = 0.0;
        for (int o = 0; o < nord; ++o) vmax = std::max(vmax, std::hypot(mean[2 * o], mean[2 * o + 1]));
        bool ok = true;
        for (int o = 0; o < nord; ++o) {
            const double e = std::hypot(err[2 * o], err[2 * o + 1]);
            const double v = std::hypot(mean[2 * o], mean[2 * o + 1]);
            const double target = std::max(opt->rel_tol * std::max(v, 1e-6 * vmax), opt->abs_tol);
            ok &= e <= target;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (ok) {
            status = QMC_OK;
            break;
        }
        if (opt->max_seconds > 0 && el > opt->max_seconds) {
            status = QMC_ERR_TIMEOUT;
            break;
        }
    }
    for (int o = 0; o < nord && o < QMC_MAX_ORDERS; ++o) {
        res->value[o][0] = mean[2 * o];
        res->value[o][1] = mean[2 * o + 1];
        res->error[o][0] = err[2 * o];
        res->error[o][1] = err[2 * o + 1];
    }
    res->kernel_ms = kernel_ms_total;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return res->status = status;
}

int qmc_eval_sums_host(qmc_ctx *c, const void *packed_host, const qmc_pass *pass, const double *shifts_host,
                       const double *lambda_host, double *sums_host, int64_t *fails_host) {
    if (!c || !pass || !shifts_host || !lambda_host || !sums_host || !fails_host) return QMC_ERR_ARG;
    const PackedHeader *h = header_of(packed_host);
    if (!h) return QMC_ERR_ARG;
    const size_t need = qmc_scratch_bytes(packed_host, pass);
    if (!need) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    const int m = pass->n_shifts, ns = h->n_sectors;
    const size_t sums_bytes = (size_t)ns * m * h->n_slots * 2 * sizeof(double), fails_bytes = (size_t)ns * m * 8;
    int rc = dev_reserve(c, c->hpacked, (size_t)h->total_bytes);
    if (!rc) rc = dev_reserve(c, c->shifts, (size_t)m * 6 * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->lambda, ns * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->sums, sums_bytes);
    if (!rc) rc = dev_reserve(c, c->fails, fails_bytes);
    if (!rc) rc = dev_reserve(c, c->scratch, need);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    rc = cuda_status(cudaMemcpyAsync(c->hpacked.p, packed_host, (size_t)h->total_bytes, cudaMemcpyHostToDevice, st));
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(c->shifts.p, shifts_host, (size_t)m * 6 * sizeof(double),
                                         cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(c->lambda.p, lambda_host, ns * sizeof(double), cudaMemcpyHostToDevice, st));
    if (!rc)
        rc = qmc_eval_sums(packed_host, c->hpacked.p, pass, (const double *)c->shifts.p, (const double *)c->lambda.p,
                           c->scratch.p, c->scratch.bytes, (double *)c->sums.p, (int64_t *)c->fails.p, st);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(sums_host, c->sums.p, sums_bytes, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(fails_host, c->fails.p, fails_bytes, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    return rc;
}

}  // extern "C"
