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
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
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
/* A run: consecutive packed sectors of one class that the pass evaluates (all of the class unless the pass
   names a subset); each run becomes one job per precision and one reduction job. */
struct Run {
    int cls, sector_begin, n_sect;
    int64_t items, item_off;  /* items of the run; its first item within the pass */
};
struct Plan {
    int block, P;
    int64_t chunks;
    std::vector<Run> runs;
    int64_t total_items;
};

/* Launch shapes chosen by qmc_autotune, per (family, precision, evaluator, lattice-size bucket 2^k >= n); passes
   that leave both block and points_per_thread at 0 use them. */
struct TuneKey {
    uint64_t family;
    int prec, evaluator, log2n;
    bool operator<(const TuneKey &o) const {
        if (family != o.family) return family < o.family;
        if (prec != o.prec) return prec < o.prec;
        if (evaluator != o.evaluator) return evaluator < o.evaluator;
        return log2n < o.log2n;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;

TuneKey tune_key(const PackedHeader *h, const qmc_pass *p) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < p->lattice.n) ++b;
    const int ev = (p->precision == QMC_PREC_MIXED && p->evaluator != QMC_EVAL_TABLE) ? QMC_EVAL_GENERATED : QMC_EVAL_TABLE;
    return TuneKey{h->family, p->precision, ev, b};
}

/* Mixed-precision policy of qmc_integrate and the serving loop: a lattice rung runs in FP32 only when its whole
   pass would cost more than ~1e8 flop in FP64 (about 0.2 ms at the FP64 rate this path reaches on a GB300).
   Below that, the FP32 probe and its extra device round trip cost more than the FP64 pass saves. */
bool fp32_pays(const PackedHeader *h, int m, int64_t n) {
    return (double)h->n_sectors * m * (double)n * h->flops_per_eval > 1e8;
}

int make_plan(const PackedHeader *h, const qmc_pass *p, Plan &pl) {
    if (!h || !p) return QMC_ERR_ARG;
    if (p->lattice.n < 2 || p->lattice.n >= ((int64_t)1 << 31)) return QMC_ERR_ARG;
    if (p->n_shifts < 1 || p->n_shifts > 4096) return QMC_ERR_ARG;
    if (p->transform_r < 0 || p->transform_r > 3) return QMC_ERR_ARG;
    if (p->precision != QMC_PREC_FP64 && p->precision != QMC_PREC_MIXED) return QMC_ERR_ARG;
    if (p->evaluator < QMC_EVAL_AUTO || p->evaluator > QMC_EVAL_GENERATED) return QMC_ERR_ARG;
    int block = p->block, P = p->points_per_thread;
    if (block == 0 && P == 0) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(tune_key(h, p));
        if (it != g_tuned.end()) {
            block = it->second.first;
            P = it->second.second;
        }
    }
    pl.block = block ? block : 128;
    if (pl.block < 32 || pl.block > 256 || pl.block % 32) return QMC_ERR_ARG;
    if (p->precision == QMC_PREC_MIXED && p->evaluator != QMC_EVAL_TABLE && pl.block > qmc_gen_max_block(h->dim))
        return QMC_ERR_ARG;
    pl.P = P ? P : (p->precision == QMC_PREC_MIXED ? 16 : 8);
    if (pl.P < 1 || pl.P > 64) return QMC_ERR_ARG;
    for (int j = 0; j < h->dim; ++j)
        if (p->lattice.z[j] == 0 || (int64_t)p->lattice.z[j] >= p->lattice.n) return QMC_ERR_ARG;
    const int64_t C = (int64_t)pl.block * pl.P;
    pl.chunks = (p->lattice.n + C - 1) / C;
    const PackedSector *ps =
        reinterpret_cast<const PackedSector *>(reinterpret_cast<const unsigned char *>(h) + h->sectors_off);
    int64_t off = 0;
    pl.runs.clear();
    for (int c = 0; c < QMC_N_CLASSES; ++c) {
        int s = h->class_begin[c];
        while (s < h->class_end[c]) {
            if (p->sector_active && !p->sector_active[ps[s].orig_index]) {
                ++s;
                continue;
            }
            int e = s + 1;
            while (e < h->class_end[c] && (!p->sector_active || p->sector_active[ps[e].orig_index])) ++e;
            Run r;
            r.cls = c;
            r.sector_begin = s;
            r.n_sect = e - s;
            r.items = (int64_t)r.n_sect * p->n_shifts * pl.chunks;
            r.item_off = off;
            off += r.items;
            pl.runs.push_back(r);
            s = e;
        }
    }
    pl.total_items = off;
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
        case QMC_ERR_CODEGEN: return "run-time compilation of the generated evaluator failed";
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

namespace {

int class_maxm(const PackedHeader *h, int c) { return h->class_maxm[c] == 0 ? 0 : (h->class_maxm[c] <= 2 ? 2 : 4); }

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

/* Scratch layout of a batch of passes: each pass owns a slice of per-item partials and sign-failure counts (its
   items in (class, sector, shift, chunk) order); the evaluation launches share an array of work counters. */
struct BatchLayout {
    std::vector<Plan> plans;
    std::vector<size_t> partial_off, fail_off;
    size_t counters_off = 0;
    int n_counters = 0;
    size_t total = 0;
};

int batch_layout(const qmc_batch_item *items, int n, BatchLayout &L) {
    if (!items || n < 1) return QMC_ERR_ARG;
    L.plans.resize(n);
    L.partial_off.resize(n);
    L.fail_off.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const PackedHeader *h = header_of(items[i].packed_host);
        int rc = make_plan(h, &items[i].pass, L.plans[i]);
        if (rc) return rc;
        L.partial_off[i] = off;
        off += up256((size_t)L.plans[i].total_items * h->n_slots * 2 * sizeof(double));
        L.fail_off[i] = off;
        off += up256((size_t)L.plans[i].total_items * sizeof(uint32_t));
    }
    size_t runs = 0;
    for (int i = 0; i < n; ++i) runs += L.plans[i].runs.size();
    L.n_counters = (int)(2 * runs + 4); /* at most one launch per (run, precision) */
    L.counters_off = off;
    off += up256((size_t)L.n_counters * sizeof(unsigned long long));
    L.total = off;
    return QMC_OK;
}

int check_items(const qmc_batch_item *items, int n, bool need_eval_inputs, bool need_outputs) {
    for (int i = 0; i < n; ++i) {
        const qmc_batch_item &b = items[i];
        if (!header_of(b.packed_host) || !b.packed_dev || ((uintptr_t)b.packed_dev & 15)) return QMC_ERR_ARG;
        if (need_eval_inputs && (!b.shifts_dev || !b.lambda_dev)) return QMC_ERR_ARG;
        if (need_outputs && (!b.sums_dev || !b.fails_dev)) return QMC_ERR_ARG;
    }
    return QMC_OK;
}

/* gen: kernel handle of a generated evaluator (FP32 jobs of one family), null for the ahead-of-time kernels */
struct LaunchKey {
    int dim, deform, maxm, prec, block, P, r;
    const void *gen;
    bool operator<(const LaunchKey &o) const {
        const int a[7] = {dim, deform, maxm, prec, block, P, r}, b[7] = {o.dim, o.deform, o.maxm, o.prec, o.block, o.P, o.r};
        for (int k = 0; k < 7; ++k)
            if (a[k] != b[k]) return a[k] < b[k];
        return std::less<const void *>()(gen, o.gen);
    }
};

bool use_generated(const qmc_pass &p) { return p.precision == QMC_PREC_MIXED && p.evaluator != QMC_EVAL_TABLE; }
/* FP64 jobs: generated unless the pass asks for the table */
bool use_generated64(const qmc_pass &p, const PackedHeader *) { return p.evaluator != QMC_EVAL_TABLE; }

/* Evaluation launches of a batch: every (pass, class, precision) becomes a job; jobs sharing a kernel
   instantiation and launch shape go into one persistent launch (tables of up to QMC_MAX_JOBS jobs). */
int run_eval(const qmc_batch_item *items, int n, const BatchLayout &L, unsigned char *scr, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(scr + L.counters_off);
    int rc = cuda_status(cudaMemsetAsync(counters, 0, (size_t)L.n_counters * sizeof(unsigned long long), st));
    if (rc) return rc;
    int sms = 0;
    rc = qmc_device_sm_count(&sms);
    if (rc) return rc;
    std::map<LaunchKey, std::vector<Job>> groups;
    std::map<LaunchKey, int> smem_need;
    for (int i = 0; i < n; ++i) {
        const qmc_batch_item &b = items[i];
        const PackedHeader *h = header_of(b.packed_host);
        const Plan &pl = L.plans[i];
        const bool mixed = b.pass.precision == QMC_PREC_MIXED;
        for (const Run &run : pl.runs) {
            const int c = run.cls;
            for (int prec = 0; prec < 2; ++prec) {
                if (!mixed && prec == 1) continue;
                if (mixed && prec == 0 && !b.pass.sector_precision) continue;
                Job J;
                std::memset(&J, 0, sizeof(J));
                J.packed = static_cast<const unsigned char *>(b.packed_dev);
                J.sectors_off = h->sectors_off;
                J.terms_off = h->terms_off;
                J.termsf_off = h->termsf_off;
                J.chunks = pl.chunks;
                J.shifts = b.shifts_dev;
                J.lambda = b.lambda_dev;
                J.sector_prec = mixed ? b.pass.sector_precision : nullptr;
                J.partials = reinterpret_cast<double *>(scr + L.partial_off[i]) + run.item_off * h->n_slots * 2;
                J.part_fails = reinterpret_cast<uint32_t *>(scr + L.fail_off[i]) + run.item_off;
                J.n = (uint32_t)b.pass.lattice.n;
                J.invn = 1.0 / (double)b.pass.lattice.n;
                for (int j = 0; j < QMC_MAX_DIM; ++j) {
                    J.z[j] = j < h->dim ? b.pass.lattice.z[j] : 0;
                    J.zstep[j] = (uint32_t)(((uint64_t)pl.block * J.z[j]) % (uint64_t)b.pass.lattice.n);
                }
                J.sector_begin = run.sector_begin;
                J.n_sect = run.n_sect;
                J.m = b.pass.n_shifts;
                J.n_slots = h->n_slots;
                J.eU0 = h->eU0;
                J.eU1 = h->eU1;
                J.eF0 = h->eF0;
                J.eF1 = h->eF1;
                const void *gen = nullptr;
                if (prec == 1 && use_generated(b.pass)) {
                    rc = qmc_gen_kernel(b.packed_host, QMC_PREC_MIXED, c, &gen);
                    if (rc) return rc;
                } else if (prec == 0 && use_generated64(b.pass, h)) {
                    rc = qmc_gen_kernel(b.packed_host, QMC_PREC_FP64, c, &gen);
                    if (rc) return rc;
                }
                const LaunchKey key{h->dim, c, class_maxm(h, c), prec == 0 ? QMC_PREC_FP64 : QMC_PREC_MIXED, pl.block,
                                    pl.P, b.pass.transform_r, gen};
                groups[key].push_back(J);
                const int need = (int)(sizeof(PackedSector) + (size_t)h->max_terms * sizeof(PackedTerm));
                smem_need[key] = std::max(smem_need[key], need);
            }
        }
    }
    int counter = 0;
    std::unique_ptr<JobTable> jt(new JobTable());
    for (auto &kv : groups) {
        const LaunchKey &k = kv.first;
        const std::vector<Job> &jobs = kv.second;
        for (size_t b0 = 0; b0 < jobs.size(); b0 += QMC_MAX_JOBS) {
            std::memset(jt.get(), 0, sizeof(JobTable));
            const size_t nj = std::min(jobs.size() - b0, (size_t)QMC_MAX_JOBS);
            int64_t total = 0;
            for (size_t q = 0; q < nj; ++q) {
                jt->jobs[q] = jobs[b0 + q];
                jt->jobs[q].item_begin = total;
                total += (int64_t)jt->jobs[q].n_sect * jt->jobs[q].m * jt->jobs[q].chunks;
            }
            jt->n_jobs = (int32_t)nj;
            jt->r = k.r;
            jt->P = k.P;
            jt->want_prec = k.prec == QMC_PREC_FP64 ? 0 : 1;
            jt->total_items = total;
            if (counter >= L.n_counters) return QMC_ERR_UNSUPPORTED;
            jt->counter = counters + counter++;
            jt->smem_bytes = smem_need[k];
            int per_sm = 0;
            rc = k.gen ? qmc_gen_blocks_per_sm(k.gen, k.block, jt->smem_bytes, &per_sm)
                       : qmc_eval_blocks_per_sm(k.dim, k.deform, k.maxm, k.prec, k.block, jt->smem_bytes, &per_sm);
            if (rc) return rc;
            if (per_sm < 1) return QMC_ERR_UNSUPPORTED;
            int64_t grid = (int64_t)sms * per_sm;
            for (int i = 0; i < n; ++i)
                if (items[i].pass.grid > 0) grid = std::min<int64_t>(grid, items[i].pass.grid);
            if (grid > total) grid = total;
            rc = k.gen ? qmc_gen_launch_eval(k.gen, *jt, (int)grid, k.block, stream)
                       : qmc_launch_eval(k.dim, k.deform, k.maxm, k.prec, *jt, (int)grid, k.block, stream);
            if (rc) return rc;
        }
    }
    return QMC_OK;
}

/* Reductions of a batch: one warp per (pass, sector, shift) over that pair's item partials, in fixed order. */
int run_reduce(const qmc_batch_item *items, int n, const BatchLayout &L, const unsigned char *scr, void *stream) {
    std::unique_ptr<FinTable> ft(new FinTable());
    std::memset(ft.get(), 0, sizeof(FinTable));
    int64_t pairs = 0;
    auto flush = [&]() -> int {
        if (ft->n_jobs == 0) return QMC_OK;
        ft->total_pairs = pairs;
        const int rc = qmc_launch_finalize(*ft, stream);
        std::memset(ft.get(), 0, sizeof(FinTable));
        pairs = 0;
        return rc;
    };
    for (int i = 0; i < n; ++i) {
        const qmc_batch_item &b = items[i];
        const PackedHeader *h = header_of(b.packed_host);
        const Plan &pl = L.plans[i];
        for (const Run &run : pl.runs) {
            if (ft->n_jobs == QMC_MAX_JOBS) {
                const int rc = flush();
                if (rc) return rc;
            }
            FinJob &J = ft->jobs[ft->n_jobs++];
            J.packed = static_cast<const unsigned char *>(b.packed_dev);
            J.sectors_off = h->sectors_off;
            J.chunks = pl.chunks;
            J.pair_begin = pairs;
            J.partials = reinterpret_cast<const double *>(scr + L.partial_off[i]) + run.item_off * h->n_slots * 2;
            J.part_fails = reinterpret_cast<const uint32_t *>(scr + L.fail_off[i]) + run.item_off;
            J.sums = b.sums_dev;
            J.fails = b.fails_dev;
            J.sector_begin = run.sector_begin;
            J.n_sect = run.n_sect;
            J.m = b.pass.n_shifts;
            J.n_slots = h->n_slots;
            pairs += (int64_t)J.n_sect * J.m;
        }
    }
    return flush();
}

qmc_batch_item single_item(const void *packed_host, const void *packed_dev, const qmc_pass *pass,
                           const double *shifts_dev, const double *lambda_dev, double *sums_dev, int64_t *fails_dev) {
    qmc_batch_item b;
    std::memset(&b, 0, sizeof(b));
    b.packed_host = packed_host;
    b.packed_dev = packed_dev;
    if (pass) b.pass = *pass;
    b.shifts_dev = shifts_dev;
    b.lambda_dev = lambda_dev;
    b.sums_dev = sums_dev;
    b.fails_dev = fails_dev;
    return b;
}

}  // namespace

extern "C" {

size_t qmc_batch_scratch_bytes(const qmc_batch_item *items, int32_t n) {
    BatchLayout L;
    try {
        if (batch_layout(items, n, L) != QMC_OK) return 0;
    } catch (...) {
        return 0;
    }
    return L.total;
}

size_t qmc_scratch_bytes(const void *packed, const qmc_pass *pass) {
    if (!pass) return 0;
    const qmc_batch_item b = single_item(packed, nullptr, pass, nullptr, nullptr, nullptr, nullptr);
    return qmc_batch_scratch_bytes(&b, 1);
}

int qmc_eval_batch(const qmc_batch_item *items, int32_t n, void *scratch_dev, size_t scratch_bytes, void *stream) {
    try {
        BatchLayout L;
        int rc = batch_layout(items, n, L);
        if (rc) return rc;
        rc = check_items(items, n, true, true);
        if (rc) return rc;
        if (!scratch_dev || ((uintptr_t)scratch_dev & 255)) return QMC_ERR_ARG;
        if (scratch_bytes < L.total) return QMC_ERR_MEMORY;
        unsigned char *scr = static_cast<unsigned char *>(scratch_dev);
        rc = run_eval(items, n, L, scr, stream);
        if (rc) return rc;
        return run_reduce(items, n, L, scr, stream);
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
}

int qmc_eval_partials(const void *packed_host, const void *packed_dev, const qmc_pass *pass,
                      const double *shifts_dev, const double *lambda_dev, void *scratch_dev, size_t scratch_bytes,
                      void *stream) {
    const qmc_batch_item b = single_item(packed_host, packed_dev, pass, shifts_dev, lambda_dev, nullptr, nullptr);
    try {
        BatchLayout L;
        int rc = batch_layout(&b, 1, L);
        if (rc) return rc;
        rc = check_items(&b, 1, true, false);
        if (rc) return rc;
        if (!scratch_dev || ((uintptr_t)scratch_dev & 255)) return QMC_ERR_ARG;
        if (scratch_bytes < L.total) return QMC_ERR_MEMORY;
        return run_eval(&b, 1, L, static_cast<unsigned char *>(scratch_dev), stream);
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
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
    const qmc_batch_item b = single_item(packed_host, packed_dev, pass, nullptr, nullptr, sums_dev, fails_dev);
    try {
        BatchLayout L;
        int rc = batch_layout(&b, 1, L);
        if (rc) return rc;
        rc = check_items(&b, 1, false, true);
        if (rc) return rc;
        if (!scratch_dev || ((uintptr_t)scratch_dev & 255)) return QMC_ERR_ARG;
        if (scratch_bytes < L.total) return QMC_ERR_MEMORY;
        return run_reduce(&b, 1, L, static_cast<const unsigned char *>(scratch_dev), stream);
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
}

int qmc_eval_sums(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                  const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, double *sums_dev,
                  int64_t *fails_dev, void *stream) {
    const qmc_batch_item b = single_item(packed_host, packed_dev, pass, shifts_dev, lambda_dev, sums_dev, fails_dev);
    return qmc_eval_batch(&b, 1, scratch_dev, scratch_bytes, stream);
}

/* ------------------------------------------------------------------ launch-shape autotuner */
static const int k_tune_block[] = {64, 128, 256};
static const int k_tune_P[] = {4, 8, 16, 32};

size_t qmc_autotune_scratch_bytes(const void *packed_host, const qmc_pass *pass) {
    if (!header_of(packed_host) || !pass) return 0;
    size_t need = 0;
    for (int b : k_tune_block)
        for (int P : k_tune_P) {
            qmc_pass q = *pass;
            q.block = b;
            q.points_per_thread = P;
            const size_t s = qmc_scratch_bytes(packed_host, &q);
            if (!s) continue; /* shape not allowed for this pass (generated kernels of large sectors) */
            need = std::max(need, s);
        }
    return need;
}

int qmc_autotune(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                 const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, qmc_tune_result *out,
                 void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !pass || !out) return QMC_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    if (scratch_bytes < qmc_autotune_scratch_bytes(packed_host, pass)) return QMC_ERR_MEMORY;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QMC_ERR_CUDA;
    int rc = QMC_OK;
    float best = -1.f;
    bool warm = false;
    for (int b : k_tune_block)
        for (int P : k_tune_P) {
            if (rc) break;
            qmc_pass q = *pass;
            q.block = b;
            q.points_per_thread = P;
            if (!qmc_scratch_bytes(packed_host, &q)) continue;
            if (!warm) { /* first launch of the kernel (module load, attributes) stays out of the timings */
                rc = qmc_eval_partials(packed_host, packed_dev, &q, shifts_dev, lambda_dev, scratch_dev, scratch_bytes,
                                       stream);
                warm = true;
                if (rc) break;
            }
            rc = cuda_status(cudaEventRecord(e0, st));
            if (!rc)
                rc = qmc_eval_partials(packed_host, packed_dev, &q, shifts_dev, lambda_dev, scratch_dev, scratch_bytes,
                                       stream);
            if (!rc) rc = cuda_status(cudaEventRecord(e1, st));
            if (!rc) rc = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            if (!rc) rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
            if (rc) break;
            const int k = out->n_candidates++;
            out->candidate_block[k] = b;
            out->candidate_points_per_thread[k] = P;
            out->candidate_ms[k] = ms;
            if (best < 0.f || ms < best) {
                best = ms;
                out->block = b;
                out->points_per_thread = P;
                out->ms = ms;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned[tune_key(h, pass)] = {out->block, out->points_per_thread};
    return QMC_OK;
}

int qmc_autotune_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned.clear();
    return QMC_OK;
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

}  // extern "C"

namespace {

/* Eqs. 19-20 with the Gamma prefactor: per-shift totals Q, their mean and standard errors.  invn[s] = 1/n of
   the lattice that produced sector s's sums (table order); only >= 0 restricts the totals to that sector. */
int combine_core(const void *packed_host, int m, const double *invn_of, int only, const double *sums, double *Q,
                 double *mean, double *err) {
    const PackedHeader *h = header_of(packed_host);
    const int ns = h->n_slots;
    const int nord = h->order_max - h->order_min + 1;
    const PackedSector *ps = sectors_of(packed_host);
    /* sector-sum orders run from -max_sigma to kmax */
    const int lo = -h->max_sigma;
    const int width = h->kmax - lo + 1;
    std::vector<double> tr(width), ti(width);
    for (int k = 0; k < m; ++k) {
        std::fill(tr.begin(), tr.end(), 0.0);
        std::fill(ti.begin(), ti.end(), 0.0);
        for (int pi = 0; pi < h->n_sectors; ++pi) {
            const PackedSector &s = ps[pi];
            if (only >= 0 && s.orig_index != only) continue;
            const double invn = invn_of[s.orig_index];
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

}  // namespace

extern "C" {

int qmc_combine(const void *packed_host, const qmc_pass *pass, const double *sums, double *Q, double *mean,
                double *err) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !pass || !sums || !Q || !mean || !err || pass->n_shifts < 1 || pass->lattice.n < 1) return QMC_ERR_ARG;
    std::vector<double> invn(h->n_sectors, 1.0 / (double)pass->lattice.n);
    return combine_core(packed_host, pass->n_shifts, invn.data(), -1, sums, Q, mean, err);
}

int qmc_combine_sectors(const void *packed_host, int32_t n_shifts, const int64_t *n_sector, const double *sums,
                        double *Q, double *mean, double *err) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !n_sector || !sums || !Q || !mean || !err || n_shifts < 1) return QMC_ERR_ARG;
    std::vector<double> invn(h->n_sectors);
    for (int s = 0; s < h->n_sectors; ++s) {
        if (n_sector[s] < 1) return QMC_ERR_ARG;
        invn[s] = 1.0 / (double)n_sector[s];
    }
    return combine_core(packed_host, n_shifts, invn.data(), -1, sums, Q, mean, err);
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

struct Serving;

struct qmc_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    std::map<int32_t, Integral> integrals;
    int32_t next_id = 1;
    DevBuf scratch, sums, fails, shifts, lambda, hpacked, prec, probe;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::mutex mu;
    Serving *serving = nullptr;
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

namespace {

/* ------------------------------------------------------------------ integration to a requested accuracy
 * State of one integration (qmc_integrate, or one serving request).  Every sector s has its own rung r_s on the
 * lattice ladder, deformation parameter lambda_s (halved on sign failures, Eq. 14) and precision flag; sums
 * holds the latest per-(sector, shift) sums, each from its own lattice.  A step evaluates the active sectors
 * (one pass per distinct rung, sector_active masks), then:
 *   sign failures -> halve lambda of the failing sectors, which alone are evaluated again;
 *   otherwise the per-shift totals over all sectors (Eqs. 19-20, qmc_combine_sectors) give value and error;
 *   converged (every order meets the target) -> done;
 *   else lock-step (lock_step != 0): every sector moves one rung up, as in a plain ladder;
 *        per-sector (lock_step = 0, the default): for each order still above target, sectors are taken in order of
 *        variance contribution per cost of their next rung until they hold enough of the variance for one
 *        doubling of n (which removes at least 3/4 of a QMC sector variance) to bring the order to its target,
 *        and at most 90 % of it; only those move up. */
struct IntegState {
    const unsigned char *packed = nullptr;
    const PackedHeader *h = nullptr;
    qmc_options opt;
    int m = 0, ns = 0, nord = 0, max_h = 6;
    bool mixed = false, adaptive = false, probe_due = false;
    std::vector<qmc_lattice> ladder;
    std::vector<double> shifts, lam, sums;
    std::vector<int64_t> fails;
    std::vector<int> rung, halv;
    std::vector<char> active;
    std::vector<int32_t> prec;
    std::vector<double> flops;                  /* per sector (table order) */
    std::vector<std::vector<int32_t>> masks;    /* host masks of the current passes */
    int probe_item = -1;
    std::chrono::steady_clock::time_point t0;

    int init(const unsigned char *packed_host, const qmc_options &o, std::chrono::steady_clock::time_point start,
             qmc_result &res) {
        packed = packed_host;
        h = header_of(packed);
        opt = o;
        t0 = start;
        m = o.n_shifts > 0 ? o.n_shifts : 16;
        if (m < 2 || m > 4096) return QMC_ERR_ARG;
        if (o.rel_tol < 0 || o.abs_tol < 0) return QMC_ERR_ARG;
        ns = h->n_sectors;
        nord = h->order_max - h->order_min + 1;
        res.order_min = h->order_min;
        res.n_orders = nord;
        max_h = o.max_halvings > 0 ? o.max_halvings : 6;
        if (o.n_lattices > 0) {
            if (!o.lattices) return QMC_ERR_ARG;
            ladder.assign(o.lattices, o.lattices + o.n_lattices);
        } else {
            for (int i = std::max(0, o.ladder_start); i < QMC_BUILTIN_LATTICES; ++i) {
                qmc_lattice L;
                L.n = qmc_builtin_lattice[i].n;
                for (int j = 0; j < QMC_MAX_DIM; ++j) L.z[j] = qmc_builtin_lattice[i].z[j];
                ladder.push_back(L);
            }
        }
        while (!ladder.empty() && o.max_n > 0 && ladder.back().n > o.max_n) ladder.pop_back();
        if (ladder.empty()) return QMC_ERR_NOT_CONVERGED;
        /* shifts (Eq. 18): explicit, or splitmix64 from the seed */
        if (o.shifts) shifts.assign(o.shifts, o.shifts + (size_t)m * 6);
        else splitmix_shifts(o.seed, m, shifts);
        mixed = o.precision == QMC_PREC_MIXED;
        adaptive = o.lock_step == 0;
        probe_due = mixed;
        rung.assign(ns, 0);
        halv.assign(ns, 0);
        active.assign(ns, 1);
        lam.assign(ns, o.lambda > 0 ? o.lambda : 0.5);
        prec.assign(ns, 1);
        sums.assign((size_t)ns * m * h->n_slots * 2, 0.0);
        fails.assign((size_t)ns * m, 0);
        flops.assign(ns, 0.0);
        const PackedSector *ps = sectors_of(packed);
        for (int pi = 0; pi < ns; ++pi) flops[ps[pi].orig_index] = std::max(ps[pi].flops, 1.0);
        return QMC_OK;
    }

    int64_t probe_samples() const { return opt.probe_samples > 0 ? opt.probe_samples : 4096; }

    /* passes of the next evaluation: one per distinct rung among the active sectors */
    void passes(std::vector<qmc_pass> &out, const int32_t *prec_dev) {
        out.clear();
        masks.clear();
        probe_item = -1;
        std::vector<int> rs;
        for (int s = 0; s < ns; ++s)
            if (active[s] && std::find(rs.begin(), rs.end(), rung[s]) == rs.end()) rs.push_back(rung[s]);
        std::sort(rs.begin(), rs.end());
        for (int r : rs) {
            std::vector<int32_t> mk(ns, 0);
            double fl = 0.0;
            int cnt = 0;
            for (int s = 0; s < ns; ++s)
                if (active[s] && rung[s] == r) {
                    mk[s] = 1;
                    fl += flops[s];
                    ++cnt;
                }
            qmc_pass p;
            std::memset(&p, 0, sizeof(p));
            p.lattice = ladder[r];
            p.n_shifts = m;
            p.transform_r = opt.transform_r > 0 ? opt.transform_r : 3;
            p.block = opt.block;
            p.points_per_thread = opt.points_per_thread;
            p.evaluator = opt.evaluator;
            /* mixed policy: FP32 only where this pass would cost more than ~1e8 flop in FP64 */
            const bool use32 = mixed && fl * m * (double)ladder[r].n > 1e8;
            p.precision = use32 ? QMC_PREC_MIXED : QMC_PREC_FP64;
            p.sector_precision = use32 ? prec_dev : nullptr;
            if (use32 && probe_due && probe_item < 0) probe_item = (int)out.size();
            masks.push_back(cnt == ns ? std::vector<int32_t>() : mk);
            out.push_back(p);
        }
        for (size_t k = 0; k < out.size(); ++k) out[k].sector_active = masks[k].empty() ? nullptr : masks[k].data();
    }

    void set_precision(const std::vector<double> &pr, qmc_result &res) {
        const double budget = (opt.fp32_budget > 0 ? opt.fp32_budget : 0.1) * opt.rel_tol;
        res.fp64_reruns = 0;
        for (int s = 0; s < ns; ++s) {
            bool bad = false;
            for (int o = 0; o < h->n_slots; ++o) {
                const double *v = &pr[((size_t)s * h->n_slots + o) * 4];
                if (v[1] > budget * v[0] || !std::isfinite(v[1])) bad = true;
            }
            prec[s] = bad ? 0 : 1;
            res.fp64_reruns += bad;
        }
        probe_due = false;
    }

    void count(const std::vector<qmc_pass> &ps, qmc_result &res) const {
        res.passes += 1;
        for (const qmc_pass &p : ps) {
            int cnt = 0;
            for (int s = 0; s < ns; ++s) cnt += p.sector_active ? (p.sector_active[s] != 0) : 1;
            res.evals += (int64_t)cnt * m * p.lattice.n;
        }
    }

    /* after an evaluation: returns QMC_PENDING to continue, or the final status */
    int step(qmc_result &res) {
        /* sign check of Eq. (14) on the sectors just evaluated */
        bool again = false;
        for (int s = 0; s < ns; ++s) {
            if (!active[s]) continue;
            int64_t f = 0;
            for (int k = 0; k < m; ++k) f += fails[(size_t)s * m + k];
            if (f > 0) {
                res.sign_failures += (int32_t)std::min<int64_t>(f, INT32_MAX);
                if (halv[s] >= max_h) return QMC_ERR_DEFORMATION;
                lam[s] *= 0.5;
                halv[s] += 1;
                res.lambda_halvings += 1;
                again = true;
            } else {
                active[s] = 0;
            }
        }
        if (again) {
            probe_due = mixed;
            return QMC_PENDING;
        }
        std::vector<int64_t> nvec(ns);
        int64_t nmax = 0;
        for (int s = 0; s < ns; ++s) {
            nvec[s] = ladder[rung[s]].n;
            nmax = std::max(nmax, nvec[s]);
        }
        std::vector<double> Q((size_t)m * nord * 2), mean(nord * 2), err(nord * 2);
        qmc_combine_sectors(packed, m, nvec.data(), sums.data(), Q.data(), mean.data(), err.data());
        res.n_final = nmax;
        for (int o = 0; o < nord && o < QMC_MAX_ORDERS; ++o) {
            res.value[o][0] = mean[2 * o];
            res.value[o][1] = mean[2 * o + 1];
            res.error[o][0] = err[2 * o];
            res.error[o][1] = err[2 * o + 1];
        }
        double vmax = 0.0;
        for (int o = 0; o < nord; ++o) vmax = std::max(vmax, std::hypot(mean[2 * o], mean[2 * o + 1]));
        std::vector<double> tau(nord), e(nord);
        bool ok = true;
        for (int o = 0; o < nord; ++o) {
            e[o] = std::hypot(err[2 * o], err[2 * o + 1]);
            tau[o] = std::max(opt.rel_tol * std::max(std::hypot(mean[2 * o], mean[2 * o + 1]), 1e-6 * vmax), opt.abs_tol);
            ok &= e[o] <= tau[o];
        }
        if (ok) return QMC_OK;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (opt.max_seconds > 0 && el > opt.max_seconds) return QMC_ERR_TIMEOUT;
        if (!adaptive) {
            for (int s = 0; s < ns; ++s)
                if (rung[s] + 1 >= (int)ladder.size()) return QMC_ERR_NOT_CONVERGED;
            for (int s = 0; s < ns; ++s) {
                rung[s] += 1;
                active[s] = 1;
            }
            return QMC_PENDING;
        }
        /* per-sector allocation: error contribution of each sector per order */
        std::vector<double> Qs((size_t)m * nord * 2), ms(nord * 2), es(nord * 2);
        std::vector<double> invn(ns);
        for (int s = 0; s < ns; ++s) invn[s] = 1.0 / (double)nvec[s];
        std::vector<double> e2((size_t)ns * nord, 0.0);
        for (int s = 0; s < ns; ++s) {
            combine_core(packed, m, invn.data(), s, sums.data(), Qs.data(), ms.data(), es.data());
            for (int o = 0; o < nord; ++o) e2[(size_t)s * nord + o] = es[2 * o] * es[2 * o] + es[2 * o + 1] * es[2 * o + 1];
        }
        std::vector<char> pick(ns, 0);
        for (int o = 0; o < nord; ++o) {
            if (e[o] <= tau[o]) continue;
            double tot = 0.0;
            for (int s = 0; s < ns; ++s) tot += e2[(size_t)s * nord + o];
            if (tot <= 0.0) continue;
            /* share of this order's variance the step must remove; one doubling removes >= 3/4 of a sector's, so
               the picked sectors must hold >= 4/3 of that share (with a margin), but never the last 10 %: sectors
               that barely contribute stay on their lattice until their share grows */
            const double need_frac = 1.0 - (tau[o] * tau[o]) / (e[o] * e[o]);
            const double need = std::min(0.9, 1.2 * need_frac / 0.75) * tot;
            std::vector<std::pair<double, int>> order;
            for (int s = 0; s < ns; ++s) {
                if (rung[s] + 1 >= (int)ladder.size()) continue;
                const double cost = flops[s] * (double)ladder[rung[s] + 1].n;
                order.push_back({e2[(size_t)s * nord + o] / cost, s});
            }
            std::sort(order.begin(), order.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
                return a.first > b.first || (a.first == b.first && a.second < b.second);
            });
            double got = 0.0;
            for (const auto &pr : order) {
                if (got >= need) break;
                pick[pr.second] = 1;
                got += e2[(size_t)pr.second * nord + o];
            }
        }
        bool any = false;
        for (int s = 0; s < ns; ++s)
            if (pick[s]) {
                rung[s] += 1;
                active[s] = 1;
                any = true;
            }
        return any ? QMC_PENDING : QMC_ERR_NOT_CONVERGED;
    }
};

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

void serving_shutdown(qmc_ctx *c);

int qmc_destroy(qmc_ctx *c) {
    if (!c) return QMC_ERR_ARG;
    serving_shutdown(c);
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
    cudaSetDevice(c->device);
    IntegState st;
    int rc = st.init(I.packed.data(), *opt, t0, *res);
    if (rc) return res->status = rc;
    const int ns = st.ns, m = st.m;
    const PackedHeader *h = st.h;
    rc = dev_reserve(c, c->shifts, st.shifts.size() * sizeof(double));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(c->shifts.p, st.shifts.data(), st.shifts.size() * sizeof(double),
                                              cudaMemcpyHostToDevice, c->stream));
    if (!rc) rc = dev_reserve(c, c->lambda, ns * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->sums, st.sums.size() * sizeof(double));
    if (!rc) rc = dev_reserve(c, c->fails, st.fails.size() * sizeof(int64_t));
    if (!rc && st.mixed) rc = dev_reserve(c, c->prec, ns * sizeof(int32_t));
    if (!rc && st.mixed) rc = dev_reserve(c, c->probe, (size_t)ns * h->n_slots * 4 * sizeof(double));
    if (rc) return res->status = rc;
    float kernel_ms_total = 0.f;
    std::vector<qmc_pass> passes;
    std::vector<qmc_batch_item> items;
    int status = QMC_PENDING;
    while (status == QMC_PENDING) {
        st.passes(passes, (const int32_t *)c->prec.p);
        rc = cuda_status(cudaMemcpyAsync(c->lambda.p, st.lam.data(), ns * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream));
        if (!rc && st.probe_item >= 0) {
            /* FP32 budget of Sec. II's cancellation-prone sectors: the probe decides which sectors stay in FP32 */
            std::vector<double> pr((size_t)ns * h->n_slots * 4);
            rc = qmc_probe_precision(st.packed, I.dpacked.p, &passes[st.probe_item], (const double *)c->shifts.p,
                                     (const double *)c->lambda.p, st.probe_samples(), (double *)c->probe.p, c->stream);
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(pr.data(), c->probe.p, pr.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost, c->stream));
            if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
            if (!rc) {
                st.set_precision(pr, *res);
                rc = cuda_status(cudaMemcpyAsync(c->prec.p, st.prec.data(), ns * sizeof(int32_t),
                                                 cudaMemcpyHostToDevice, c->stream));
            }
        }
        if (rc) return res->status = rc;
        items.assign(passes.size(), qmc_batch_item());
        for (size_t k = 0; k < passes.size(); ++k) {
            std::memset(&items[k], 0, sizeof(qmc_batch_item));
            items[k].packed_host = st.packed;
            items[k].packed_dev = I.dpacked.p;
            items[k].pass = passes[k];
            items[k].shifts_dev = (const double *)c->shifts.p;
            items[k].lambda_dev = (const double *)c->lambda.p;
            items[k].sums_dev = (double *)c->sums.p;
            items[k].fails_dev = (int64_t *)c->fails.p;
        }
        const size_t need = qmc_batch_scratch_bytes(items.data(), (int32_t)items.size());
        if (!need) return res->status = QMC_ERR_ARG;
        rc = dev_reserve(c, c->scratch, need);
        if (!rc) rc = cuda_status(cudaEventRecord(c->ev0, c->stream));
        if (!rc) rc = qmc_eval_batch(items.data(), (int32_t)items.size(), c->scratch.p, c->scratch.bytes, c->stream);
        if (!rc) rc = cuda_status(cudaEventRecord(c->ev1, c->stream));
        if (!rc)
            rc = cuda_status(cudaMemcpyAsync(st.sums.data(), c->sums.p, st.sums.size() * sizeof(double),
                                             cudaMemcpyDeviceToHost, c->stream));
        if (!rc)
            rc = cuda_status(cudaMemcpyAsync(st.fails.data(), c->fails.p, st.fails.size() * sizeof(int64_t),
                                             cudaMemcpyDeviceToHost, c->stream));
        if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
        if (rc) return res->status = rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        kernel_ms_total += ms;
        st.count(passes, *res);
        status = st.step(*res);
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

/* ====================================================================== serving: continuous batching */
/*
 * Requests (an integral at a kinematic point, with options) are queued by qmc_submit.  A scheduler thread admits
 * them while the context's device-memory budget allows their tables, shift sums and first-pass scratch, and then
 * runs rounds: in each round every active request contributes the pass at its current lattice size to one
 * qmc_eval_batch (persistent launches shared by all requests of the same sector class), the per-shift sums come
 * back, and each request independently halves lambda of failing sectors, checks its convergence and either
 * finishes, retries the same size, or moves to the next lattice size.  Requests that arrive while others are
 * running join at the next round.  A request's passes are computed exactly as they would be alone, so its
 * result does not depend on what else is in the batch.
 */
namespace {

enum { REQ_QUEUED = 0, REQ_ACTIVE = 1, REQ_DONE = 2 };

struct Request {
    int64_t id = 0;
    int32_t integral_id = 0;
    std::vector<unsigned char> table;
    std::vector<double> inv;
    int32_t omin = 0, omax = 0;
    qmc_options opt;
    std::vector<unsigned char> packed;
    qmc_info info;
    DevBuf dpacked, dshifts, dlambda, dsums, dfails, dprec, dprobe;
    std::vector<double> shifts_copy;          /* the caller's explicit shifts / lattices, copied at submission */
    std::vector<qmc_lattice> lattices_copy;
    IntegState st;                 /* the same integration state machine as qmc_integrate */
    std::vector<qmc_pass> passes;  /* passes of the current round */
    qmc_result res;
    std::chrono::steady_clock::time_point t_submit, t_admit;
    bool cancelled = false;
    int state = REQ_QUEUED;
};

}  // namespace

struct Serving {
    std::thread th;
    cudaStream_t stream = nullptr; /* the loop's own stream: rounds never wait for, or block, other context calls */
    DevBuf scratch;                /* the loop's own scratch (counted in the context's budget) */
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> compiling; /* admitted; waiting for their family's generated code */
    std::vector<std::shared_ptr<Request>> active;
    std::map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_id = 1;
    qmc_serving_stats stats;
};

namespace {

void release_request(qmc_ctx *c, Request &r) {
    for (DevBuf *b : {&r.dpacked, &r.dshifts, &r.dlambda, &r.dsums, &r.dfails, &r.dprec, &r.dprobe}) dev_release(c, *b);
}

void finish(Serving *S, qmc_ctx *c, Request &r, int status) {
    release_request(c, r);
    if (status != QMC_OK && r.res.n_final == 0 && !r.st.ladder.empty()) r.res.n_final = r.st.ladder[0].n;
    r.res.status = status;
    r.res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
    r.res.queued_seconds = std::chrono::duration<double>(r.t_admit - r.t_submit).count();
    std::lock_guard<std::mutex> g(S->mu);
    r.state = REQ_DONE;
    S->stats.completed += 1;
}

/* host preparation and device buffers of a newly admitted request (called with the context mutex held) */
int admit(Serving *S, qmc_ctx *c, Request &r) {
    int rc = qmc_prepare(r.table.data(), r.table.size(), r.inv.data(), (int32_t)r.inv.size(), r.omin, r.omax, nullptr,
                         0, &r.info);
    if (rc) return rc;
    r.packed.assign((size_t)r.info.packed_bytes, 0);
    rc = qmc_prepare(r.table.data(), r.table.size(), r.inv.data(), (int32_t)r.inv.size(), r.omin, r.omax,
                     r.packed.data(), r.packed.size(), &r.info);
    if (rc) return rc;
    if (!r.shifts_copy.empty()) r.opt.shifts = r.shifts_copy.data();
    if (!r.lattices_copy.empty()) r.opt.lattices = r.lattices_copy.data();
    rc = r.st.init(r.packed.data(), r.opt, r.t_submit, r.res);
    if (rc) return rc;
    const PackedHeader *h = r.st.h;
    const int ns = h->n_sectors;
    rc = dev_reserve(c, r.dpacked, r.packed.size());
    if (!rc) rc = dev_reserve(c, r.dshifts, r.st.shifts.size() * sizeof(double));
    if (!rc) rc = dev_reserve(c, r.dlambda, ns * sizeof(double));
    if (!rc) rc = dev_reserve(c, r.dsums, r.st.sums.size() * sizeof(double));
    if (!rc) rc = dev_reserve(c, r.dfails, r.st.fails.size() * sizeof(int64_t));
    if (!rc) rc = dev_reserve(c, r.dprec, ns * sizeof(int32_t));
    if (!rc) rc = dev_reserve(c, r.dprobe, (size_t)ns * h->n_slots * 4 * sizeof(double));
    if (rc) return rc;
    rc = cuda_status(cudaMemcpyAsync(r.dpacked.p, r.packed.data(), r.packed.size(), cudaMemcpyHostToDevice, S->stream));
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(r.dshifts.p, r.st.shifts.data(), r.st.shifts.size() * sizeof(double),
                                         cudaMemcpyHostToDevice, S->stream));
    return rc;
}

/* generated evaluators the request's passes may use: compiled in the background; QMC_OK once all are loaded */
int gen_ready(const Request &r) {
    int rc = QMC_OK;
    if (r.opt.precision == QMC_PREC_MIXED) rc = qmc_gen_compile(r.packed.data(), QMC_PREC_MIXED, 2, nullptr);
    if (rc == QMC_OK) rc = qmc_gen_compile(r.packed.data(), QMC_PREC_FP64, 2, nullptr);
    return rc;
}

/* FP32 budget check of a mixed-precision request before the first FP32 pass (as in qmc_integrate); lambda
   must already be on the device */
int probe(Serving *S, Request &r) {
    const PackedHeader *h = r.st.h;
    std::vector<double> pr((size_t)h->n_sectors * h->n_slots * 4);
    int rc = qmc_probe_precision(r.packed.data(), r.dpacked.p, &r.passes[r.st.probe_item], (const double *)r.dshifts.p,
                                 (const double *)r.dlambda.p, r.st.probe_samples(), (double *)r.dprobe.p, S->stream);
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(pr.data(), r.dprobe.p, pr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                         S->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(S->stream));
    if (rc) return rc;
    r.st.set_precision(pr, r.res);
    return cuda_status(cudaMemcpyAsync(r.dprec.p, r.st.prec.data(), r.st.ns * sizeof(int32_t), cudaMemcpyHostToDevice,
                                       S->stream));
}

void serve_loop(qmc_ctx *c) {
    Serving *S = c->serving;
    cudaSetDevice(c->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> fresh, cancelled;
        /* lock order: the context mutex is never taken while the serving mutex is held */
        size_t in_use;
        {
            std::lock_guard<std::mutex> g(c->mu);
            in_use = c->used;
        }
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto ready = [&] { return S->stop || !S->queue.empty() || !S->active.empty(); };
            if (S->compiling.empty()) S->cv.wait(lk, ready);
            else S->cv.wait_for(lk, std::chrono::milliseconds(2), ready);
            if (S->stop) return;
            /* cancelled requests leave at the round boundary (finished below, outside this lock) */
            for (auto it = S->active.begin(); it != S->active.end();) {
                if ((*it)->cancelled) {
                    cancelled.push_back(*it);
                    it = S->active.erase(it);
                } else {
                    ++it;
                }
            }
            /* admission: requests are taken in arrival order while the budget keeps room for their tables and
               sums plus a first-pass share of scratch; at least one request always runs */
            while (!S->queue.empty()) {
                auto r = S->queue.front();
                if (r->cancelled) {
                    S->queue.pop_front();
                    r->state = REQ_DONE;
                    r->res.status = QMC_ERR_CANCELLED;
                    S->stats.completed += 1;
                    continue;
                }
                const size_t est = 2 * r->table.size() + ((size_t)8 << 20);
                if (!S->active.empty() && in_use + est > c->budget) break;
                S->queue.pop_front();
                fresh.push_back(r);
                in_use += est;
                if (S->active.size() + fresh.size() >= QMC_MAX_JOBS / 4) break;
            }
        }
        /* device buffers of cancelled and newly admitted requests: the context mutex guards the budget */
        {
            std::lock_guard<std::mutex> g(c->mu);
            for (auto &r : cancelled) finish(S, c, *r, QMC_ERR_CANCELLED);
            for (auto &r : fresh) {
                r->t_admit = std::chrono::steady_clock::now();
                const int rc = admit(S, c, *r);
                if (rc) {
                    finish(S, c, *r, rc);
                    r.reset();
                }
            }
        }
        /* requests whose family's generated evaluator is still compiling (in the background) wait aside */
        {
            std::vector<std::shared_ptr<Request>> still;
            for (auto &r : S->compiling) {
                const int rc = r->cancelled ? QMC_ERR_CANCELLED : gen_ready(*r);
                if (rc == QMC_PENDING) {
                    still.push_back(r);
                } else if (rc) {
                    std::lock_guard<std::mutex> g(c->mu);
                    finish(S, c, *r, rc);
                } else {
                    fresh.push_back(r);
                }
            }
            S->compiling.swap(still);
        }
        for (auto &r : fresh) {
            if (!r) continue;
            if (r->opt.evaluator != QMC_EVAL_TABLE &&
                std::find(S->compiling.begin(), S->compiling.end(), r) == S->compiling.end()) {
                const int g = gen_ready(*r);
                if (g == QMC_PENDING) {
                    S->compiling.push_back(r);
                    continue;
                }
                if (g) {
                    std::lock_guard<std::mutex> lk2(c->mu);
                    finish(S, c, *r, g);
                    continue;
                }
            }
            std::lock_guard<std::mutex> g2(S->mu);
            r->state = REQ_ACTIVE;
            S->active.push_back(r);
            S->stats.peak_active = std::max<int64_t>(S->stats.peak_active, (int64_t)S->active.size());
        }
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::lock_guard<std::mutex> g2(S->mu);
            batch = S->active;
        }
        if (batch.empty()) continue;
        /* this round: one step of every active request (its passes: one per lattice rung among the sectors it
           evaluates), all in shared launches; no context lock is held meanwhile */
        int rc = QMC_OK;
        for (auto &r : batch) {
            r->st.passes(r->passes, (const int32_t *)r->dprec.p);
            rc = cuda_status(cudaMemcpyAsync(r->dlambda.p, r->st.lam.data(), r->st.lam.size() * sizeof(double),
                                             cudaMemcpyHostToDevice, S->stream));
            if (!rc && r->st.probe_item >= 0) rc = probe(S, *r);
            if (rc) break;
        }
        std::vector<qmc_batch_item> items;
        std::vector<size_t> first(batch.size() + 1, 0); /* items of batch[i]: [first[i], first[i + 1]) */
        for (size_t i = 0; i < batch.size() && !rc; ++i) {
            Request &r = *batch[i];
            for (const qmc_pass &ps : r.passes) {
                qmc_batch_item b;
                std::memset(&b, 0, sizeof(b));
                b.packed_host = r.packed.data();
                b.packed_dev = r.dpacked.p;
                b.pass = ps;
                b.shifts_dev = (const double *)r.dshifts.p;
                b.lambda_dev = (const double *)r.dlambda.p;
                b.sums_dev = (double *)r.dsums.p;
                b.fails_dev = (int64_t *)r.dfails.p;
                items.push_back(b);
            }
            first[i + 1] = items.size();
        }
        size_t need = rc ? 0 : qmc_batch_scratch_bytes(items.data(), (int32_t)items.size());
        if (!rc && !need) rc = QMC_ERR_ARG;
        if (!rc) {
            std::lock_guard<std::mutex> g(c->mu);
            /* the round shrinks (later requests wait) when its scratch would not fit the budget */
            while (batch.size() > 1 && c->used - S->scratch.bytes + ((need + 4095) & ~size_t(4095)) > c->budget) {
                batch.pop_back();
                items.resize(first[batch.size()]);
                need = qmc_batch_scratch_bytes(items.data(), (int32_t)items.size());
            }
            rc = dev_reserve(c, S->scratch, need);
        }
        if (!rc) rc = qmc_eval_batch(items.data(), (int32_t)items.size(), S->scratch.p, S->scratch.bytes, S->stream);
        for (size_t i = 0; i < batch.size() && !rc; ++i) {
            IntegState &st = batch[i]->st;
            rc = cuda_status(cudaMemcpyAsync(st.sums.data(), batch[i]->dsums.p, st.sums.size() * sizeof(double),
                                             cudaMemcpyDeviceToHost, S->stream));
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(st.fails.data(), batch[i]->dfails.p, st.fails.size() * sizeof(int64_t),
                                                 cudaMemcpyDeviceToHost, S->stream));
        }
        if (!rc) rc = cuda_status(cudaStreamSynchronize(S->stream));
        {
            std::lock_guard<std::mutex> g2(S->mu);
            S->stats.rounds += 1;
            S->stats.batched_passes += (int64_t)items.size();
        }
        std::vector<std::shared_ptr<Request>> done;
        {
            std::lock_guard<std::mutex> g(c->mu);
            for (auto &rp : batch) {
                Request &r = *rp;
                if (rc) {
                    finish(S, c, r, rc);
                    done.push_back(rp);
                    continue;
                }
                r.st.count(r.passes, r.res);
                const int st = r.st.step(r.res);
                if (st != QMC_PENDING) {
                    finish(S, c, r, st);
                    done.push_back(rp);
                }
            }
        }
        std::lock_guard<std::mutex> g2(S->mu);
        for (auto &d : done) S->active.erase(std::remove(S->active.begin(), S->active.end(), d), S->active.end());
    }
}

}  // namespace

void serving_shutdown(qmc_ctx *c) {
    if (!c->serving) return;
    {
        std::lock_guard<std::mutex> g(c->serving->mu);
        c->serving->stop = true;
    }
    c->serving->cv.notify_all();
    if (c->serving->th.joinable()) c->serving->th.join();
    cudaSetDevice(c->device);
    if (c->serving->stream) cudaStreamSynchronize(c->serving->stream);
    for (auto &kv : c->serving->all) release_request(c, *kv.second);
    dev_release(c, c->serving->scratch);
    if (c->serving->stream) cudaStreamDestroy(c->serving->stream);
    delete c->serving;
    c->serving = nullptr;
}

extern "C" {

int qmc_submit(qmc_ctx *c, int32_t integral_id, const double *invariants, int32_t n_invariants, int32_t order_min,
               int32_t order_max, const qmc_options *opt, int64_t *request_id) {
    if (!c || !opt || !request_id || (n_invariants > 0 && !invariants)) return QMC_ERR_ARG;
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> g(c->mu);
        auto it = c->integrals.find(integral_id);
        if (it == c->integrals.end()) return QMC_ERR_NOT_FOUND;
        r->table = it->second.table;
    }
    r->integral_id = integral_id;
    r->inv.assign(invariants, invariants + n_invariants);
    r->omin = order_min;
    r->omax = order_max;
    r->opt = *opt;
    std::memset(&r->res, 0, sizeof(r->res));
    const int m = opt->n_shifts > 0 ? opt->n_shifts : 16;
    if (m < 2 || m > 4096 || opt->rel_tol < 0) return QMC_ERR_ARG;
    if (opt->n_lattices > 0 && !opt->lattices) return QMC_ERR_ARG;
    if (opt->n_lattices <= 0 && std::max(0, opt->ladder_start) >= QMC_BUILTIN_LATTICES) return QMC_ERR_ARG;
    if (opt->shifts) r->opt.shifts = nullptr; /* copied below: the caller's array need not outlive the call */
    if (opt->shifts) r->shifts_copy.assign(opt->shifts, opt->shifts + (size_t)m * 6);
    if (opt->n_lattices > 0) {
        r->lattices_copy.assign(opt->lattices, opt->lattices + opt->n_lattices);
        r->opt.lattices = nullptr;
    }
    r->t_submit = std::chrono::steady_clock::now();
    r->t_admit = r->t_submit;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (!c->serving) {
            Serving *S = new Serving();
            std::memset(&S->stats, 0, sizeof(qmc_serving_stats));
            cudaSetDevice(c->device);
            if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
                delete S;
                return QMC_ERR_CUDA;
            }
            c->serving = S;
            S->th = std::thread(serve_loop, c);
        }
    }
    Serving *S = c->serving;
    {
        std::lock_guard<std::mutex> g(S->mu);
        r->id = S->next_id++;
        S->queue.push_back(r);
        S->all[r->id] = r;
        S->stats.submitted += 1;
    }
    S->cv.notify_all();
    *request_id = r->id;
    return QMC_OK;
}

int qmc_poll(qmc_ctx *c, int64_t request_id, qmc_result *out) {
    if (!c || !out) return QMC_ERR_ARG;
    if (!c->serving) return QMC_ERR_NOT_FOUND;
    Serving *S = c->serving;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(request_id);
    if (it == S->all.end()) return QMC_ERR_NOT_FOUND;
    if (it->second->state != REQ_DONE) return QMC_PENDING;
    *out = it->second->res;
    return out->status;
}

int qmc_cancel(qmc_ctx *c, int64_t request_id) {
    if (!c || !c->serving) return QMC_ERR_NOT_FOUND;
    Serving *S = c->serving;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(request_id);
    if (it == S->all.end()) return QMC_ERR_NOT_FOUND;
    it->second->cancelled = true;
    S->cv.notify_all();
    return QMC_OK;
}

int qmc_serving_stats_get(qmc_ctx *c, qmc_serving_stats *out) {
    if (!c || !out) return QMC_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    if (!c->serving) return QMC_OK;
    Serving *S = c->serving;
    int64_t used;
    {
        std::lock_guard<std::mutex> g(c->mu);
        used = (int64_t)c->used;
    }
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->stats;
    out->queued = (int64_t)S->queue.size();
    out->active = (int64_t)S->active.size();
    out->device_bytes = used;
    return QMC_OK;
}

}  // extern "C"
