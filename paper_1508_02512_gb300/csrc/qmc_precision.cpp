/*
 * Per-sector precision of a mixed pass (qmc_choose_precision): FP32, FP32 with FP64 islands at a level, or FP64,
 * from the FP32/FP64 probe with island bins (qmc_probe_islands) and the current estimate of the integral.
 *
 * The paper evaluates in one precision; the FP32 path, its error budget and the islands are this library's.  The
 * islands follow the remark after Eq. 12 of Li, Wang, Yan, Zhao, Chin. Phys. C 40 (2016) 033103: the subtraction
 * of Eq. 11 cancels near the faces t_j = 0, which is where FP32 loses its digits.
 */
#include <algorithm>
#include <cmath>
#include <limits>
#include <new>
#include <vector>

#include "qmc_host_internal.h"

namespace qmci {

void order_totals(const void *packed_host, int m, const int64_t *n_sector, const double *sums, std::vector<double> &Tr,
                  std::vector<double> &Ti) {
    const PackedHeader *h = header_of(packed_host);
    const PackedSector *ps = sectors_of(packed_host);
    const int ns = h->n_sectors, sl = h->n_slots;
    std::vector<int> sig(ns, 0);
    for (int pi = 0; pi < ns; ++pi) sig[ps[pi].orig_index] = ps[pi].sigma;
    int maxsig = 0;
    for (int s = 0; s < ns; ++s) maxsig = std::max(maxsig, sig[s]);
    Tr.assign(sl + maxsig, 0.0);
    Ti.assign(sl + maxsig, 0.0);
    for (int s = 0; s < ns; ++s) {
        const double inv = 1.0 / ((double)m * (double)n_sector[s]);
        for (int o = 0; o < sl; ++o) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < m; ++k) {
                re += sums[(((size_t)s * m + k) * sl + o) * 2];
                im += sums[(((size_t)s * m + k) * sl + o) * 2 + 1];
            }
            Tr[o - sig[s] + maxsig] += re * inv;
            Ti[o - sig[s] + maxsig] += im * inv;
        }
    }
}

bool choose_precision(const void *packed_host, const double *probe, const double *bins, int64_t n_sample,
                      const std::vector<double> &Tr, const std::vector<double> &Ti, double budget, int32_t *codes,
                      int32_t *n_fp64, int32_t *n_islands) {
    const PackedHeader *h = header_of(packed_host);
    const PackedSector *ps = sectors_of(packed_host);
    const int ns = h->n_sectors, sl = h->n_slots;
    std::vector<int> sig(ns, 0);
    std::vector<double> flops(ns, 1.0);
    std::vector<char> fp64_only(ns, 0);
    for (int pi = 0; pi < ns; ++pi) {
        const int s = ps[pi].orig_index;
        sig[s] = ps[pi].sigma;
        flops[s] = std::max(ps[pi].flops, 1.0);
        fp64_only[s] = ps[pi].taylor != 0;
    }
    int maxsig = 0;
    for (int s = 0; s < ns; ++s) maxsig = std::max(maxsig, sig[s]);
    const int K = sl + maxsig; /* order index k + maxsig, k = slot - sigma */
    std::vector<double> lim(K, 0.0);
    double tmax = 0.0;
    const bool have = (int)Tr.size() == K && (int)Ti.size() == K;
    if (have)
        for (int k = 0; k < K; ++k) tmax = std::max(tmax, std::hypot(Tr[k], Ti[k]));
    for (int k = 0; k < K && tmax > 0.0; ++k) lim[k] = budget * std::max(std::hypot(Tr[k], Ti[k]), 1e-6 * tmax);
    const double per = 1.0 / (double)std::max<int64_t>(n_sample, 1);
    const int per_bin = QMC_ISLAND_BIN_WORDS(sl);
    /* options: 0 = FP32, 1 + L = islands at level L, NOPT - 1 = FP64.  Per option and slot, over its FP32 bins:
       st = {mean |e|, |mean e|, 0, sum |e|^2 / n^2} (e = v32 - v64, n = the sample size) */
    const int NOPT = QMC_ISLAND_LEVELS + 2;
    std::vector<double> cost((size_t)ns * NOPT), st((size_t)ns * NOPT * sl * 4, 0.0), own((size_t)ns * sl);
    std::vector<char> ok((size_t)ns * NOPT, 1);
    auto S = [&](int s, int q, int o) { return &st[(((size_t)s * NOPT + q) * sl + o) * 4]; };
    for (int s = 0; s < ns; ++s) {
        const double *bs = bins + (size_t)s * QMC_ISLAND_BINS * per_bin;
        for (int o = 0; o < sl; ++o) own[(size_t)s * sl + o] = probe[((size_t)s * sl + o) * 4] * per;
        for (int q = 0; q < NOPT; ++q) {
            const int top = q == NOPT - 1 ? -1 : (q == 0 ? QMC_ISLAND_BINS - 1 : q - 1); /* FP32 bins 0..top */
            double island = 0.0;
            for (int b = top + 1; b < QMC_ISLAND_BINS; ++b) island += bs[b * per_bin] * per;
            cost[(size_t)s * NOPT + q] = flops[s] * (q == NOPT - 1 ? QMC_FP64_COST : 1.0 + QMC_FP64_COST * island);
            for (int o = 0; o < sl; ++o) {
                double *e = S(s, q, o);
                for (int b = 0; b <= top; ++b)
                    for (int j = 0; j < 4; ++j) e[j] += bs[b * per_bin + 1 + 4 * o + j];
                e[0] *= per;
                e[1] = std::hypot(e[1], e[2]) * per;
                e[2] = 0.0;
                e[3] *= per * per;
                for (int j = 0; j < 4; ++j)
                    if (!std::isfinite(e[j])) ok[(size_t)s * NOPT + q] = 0;
            }
        }
        if (fp64_only[s])
            for (int q = 0; q < NOPT - 1; ++q) ok[(size_t)s * NOPT + q] = 0;
    }
    /* the bias bound of summed statistics: the signed mean with three standard errors, capped by the mean |e| */
    auto bound = [](double a, double r, double i, double v) {
        return std::min(a, std::hypot(r, i) + 3.0 * std::sqrt(v));
    };
    std::vector<int> pick(ns, NOPT - 1);
    if (tmax <= 0.0) {
        /* no estimate of the integral yet: each sector is held to budget * mean |v64| of its own, per slot */
        for (int s = 0; s < ns; ++s) {
            double best = std::numeric_limits<double>::infinity();
            for (int q = 0; q < NOPT; ++q) {
                if (!ok[(size_t)s * NOPT + q]) continue;
                bool fits = true;
                for (int o = 0; o < sl && fits; ++o) {
                    const double *e = S(s, q, o);
                    fits = bound(e[0], e[1], e[2], e[3]) <= budget * own[(size_t)s * sl + o];
                }
                if (fits && cost[(size_t)s * NOPT + q] < best) {
                    best = cost[(size_t)s * NOPT + q];
                    pick[s] = q;
                }
            }
        }
    } else {
        /* per order k, the sectors' statistics add up: bound_k = min(sum mean|e|, sum |mean e| + 3 sqrt(sum var))
           <= lim_k (the sectors' biases are added without cancelling one another; their sampling variances add).
           Every term falls when a sector moves to FP64, so the greedy cannot stall.  Greedy: every sector
           starts at its cheapest option; while an order is over its limit, take the change of one sector's option
           with the largest reduction of the violated orders' excess (relative to their limits) per unit of extra
           cost, among changes that push no order over its limit */
        std::vector<double> tot((size_t)K * 4, 0.0);
        for (int s = 0; s < ns; ++s) {
            double best = std::numeric_limits<double>::infinity();
            for (int q = 0; q < NOPT; ++q)
                if (ok[(size_t)s * NOPT + q] && cost[(size_t)s * NOPT + q] < best) {
                    best = cost[(size_t)s * NOPT + q];
                    pick[s] = q;
                }
            for (int o = 0; o < sl; ++o)
                for (int j = 0; j < 4; ++j) tot[(size_t)(o - sig[s] + maxsig) * 4 + j] += S(s, pick[s], o)[j];
        }
        auto bound_k = [&](int k) { const double *t = &tot[(size_t)k * 4]; return bound(t[0], t[1], t[2], t[3]); };
        for (int guard = 0; guard < 4 * ns * NOPT; ++guard) {
            bool over = false;
            for (int k = 0; k < K; ++k) over |= bound_k(k) > lim[k];
            if (!over) break;
            int bs = -1, bq = -1;
            double bratio = -1.0;
            for (int s = 0; s < ns; ++s) {
                const double c0 = cost[(size_t)s * NOPT + pick[s]];
                for (int q = 0; q < NOPT; ++q) {
                    if (q == pick[s] || !ok[(size_t)s * NOPT + q]) continue;
                    double gain = 0.0;
                    bool worse = false, moved = false;
                    for (int o = 0; o < sl && !worse; ++o) {
                        const double *e0 = S(s, pick[s], o), *e1 = S(s, q, o);
                        if (e0[0] == e1[0] && e0[1] == e1[1] && e0[2] == e1[2] && e0[3] == e1[3]) continue;
                        moved = true;
                        const int k = o - sig[s] + maxsig;
                        const double *t = &tot[(size_t)k * 4];
                        const double before = bound(t[0], t[1], t[2], t[3]);
                        const double after = bound(t[0] - e0[0] + e1[0], t[1] - e0[1] + e1[1], t[2] - e0[2] + e1[2],
                                                   std::max(t[3] - e0[3] + e1[3], 0.0));
                        /* relative slack: the updated sums round differently from the ones they replace */
                        const double slack = 1e-12 * (t[0] + e1[0]);
                        if (after > std::max(before, lim[k]) + slack) worse = true;
                        else if (before > lim[k] && after < before - slack)
                            gain += (before - std::max(after, lim[k])) / std::max(lim[k], 1e-300);
                    }
                    if (worse || !moved || gain <= 0.0) continue;
                    const double dc = cost[(size_t)s * NOPT + q] - c0;
                    const double ratio = dc <= 0.0 ? std::numeric_limits<double>::infinity() : gain / dc;
                    if (ratio > bratio) {
                        bratio = ratio;
                        bs = s;
                        bq = q;
                    }
                }
            }
            if (bs < 0) break; /* no single change helps: the step below settles it */
            for (int o = 0; o < sl; ++o) {
                const int k = o - sig[bs] + maxsig;
                for (int j = 0; j < 4; ++j) tot[(size_t)k * 4 + j] += S(bs, bq, o)[j] - S(bs, pick[bs], o)[j];
                tot[(size_t)k * 4 + 3] = std::max(tot[(size_t)k * 4 + 3], 0.0);
            }
            pick[bs] = bq;
        }
        /* still over a limit (no single change helped, or the step bound ran out): the sectors with error in such
           an order take FP64 */
        std::vector<char> over(K, 0);
        for (int k = 0; k < K; ++k) over[k] = bound_k(k) > lim[k];
        for (int s = 0; s < ns; ++s)
            for (int o = 0; o < sl; ++o)
                if (over[o - sig[s] + maxsig] && S(s, pick[s], o)[0] > 0.0) pick[s] = NOPT - 1;
    }
    int32_t f64 = 0, isl = 0;
    for (int s = 0; s < ns; ++s) {
        const int q = pick[s];
        codes[s] = q == NOPT - 1 ? 0 : (q == 0 ? 1 : 2 + (q - 1));
        f64 += q == NOPT - 1;
        isl += q > 0 && q < NOPT - 1;
    }
    if (n_fp64) *n_fp64 = f64;
    if (n_islands) *n_islands = isl;
    return tmax > 0.0;
}

}  // namespace qmci

int qmc_choose_precision(const void *packed_host, int32_t n_shifts, const int64_t *n_sector, const double *sums,
                         const double *probe, const double *bins, int64_t n_sample, double rel_tol,
                         double fp32_budget, int32_t *codes, int32_t *counts) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !probe || !bins || !codes || n_sample < 1 || rel_tol < 0 || fp32_budget < 0) return QMC_ERR_ARG;
    if (sums && (!n_sector || n_shifts < 1)) return QMC_ERR_ARG;
    try {
        std::vector<double> Tr, Ti;
        if (sums) {
            for (int s = 0; s < h->n_sectors; ++s)
                if (n_sector[s] < 1) return QMC_ERR_ARG;
            qmci::order_totals(packed_host, n_shifts, n_sector, sums, Tr, Ti);
        }
        const double budget = (fp32_budget > 0 ? fp32_budget : 0.1) * rel_tol;
        int32_t f64 = 0, isl = 0;
        qmci::choose_precision(packed_host, probe, bins, n_sample, Tr, Ti, budget, codes, &f64, &isl);
        if (counts) {
            counts[0] = f64;
            counts[1] = isl;
        }
        return QMC_OK;
    } catch (const std::bad_alloc &) {
        return QMC_ERR_MEMORY;
    }
}
