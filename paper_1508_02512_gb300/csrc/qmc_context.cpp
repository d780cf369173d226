/*
 * Contexts (qmc_create ...): device memory under a budget, loaded integrals, the integrate-to-accuracy state
 * machine shared by qmc_integrate and the serving loop (per-sector lattices, lambda halving, the FP32 probe),
 * and the serving loop itself (continuous batching of requests in shared launches).
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103:
 * Sec. II Eq. 14 (sign check of the deformation), Sec. III Eqs. 18-20 (shifts, estimator, error).
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
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lattice_table.h"
#include "qmc_host_internal.h"

/* the serving loop's admission takes its load estimates times this factor before comparing them with limits */
#define QMC_SHED_MARGIN 1.25

namespace {

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
    /* qmc_integrate's abort flag (mapped pinned host memory, allocated on first use): set at the time limit */
    volatile int32_t *abort_host = nullptr;
    int32_t *abort_dev = nullptr;
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
    std::vector<char> fp64_only;                /* per sector: class 2 (alpha <= -2) runs in FP64 always */
    std::vector<std::vector<int32_t>> masks;    /* host masks of the current passes */
    int probe_item = -1;
    std::vector<double> Tr, Ti;                 /* order_totals(): per order, summed over sectors */
    std::vector<double> probe_pr;               /* the last probe's sums, and its points per sector */
    int64_t probe_n = 0;                        /* points per sector of the last probe */
    bool prec_provisional = false;
    bool prec_changed = false;                  /* prec changed outside set_precision: copy it to the device */
    std::vector<char> forced64;                 /* sectors whose FP32 sums came out non-finite: FP64 from then on */
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
        fp64_only.assign(ns, 0);
        Tr.clear();
        Ti.clear();
        probe_pr.clear();
        probe_n = 0;
        prec_provisional = false;
        prec_changed = false;
        forced64.assign(ns, 0);
        const PackedSector *ps = sectors_of(packed);
        for (int pi = 0; pi < ns; ++pi) {
            flops[ps[pi].orig_index] = std::max(ps[pi].flops, 1.0);
            fp64_only[ps[pi].orig_index] = ps[pi].taylor != 0;
        }
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
            /* the probe samples the largest lattice among the FP32 passes */
            if (use32 && probe_due && (probe_item < 0 || p.lattice.n > out[probe_item].lattice.n))
                probe_item = (int)out.size();
            masks.push_back(cnt == ns ? std::vector<int32_t>() : mk);
            out.push_back(p);
        }
        for (size_t k = 0; k < out.size(); ++k) out[k].sector_active = masks[k].empty() ? nullptr : masks[k].data();
    }

    /* the current estimate of each eps order, summed over sectors (qmci::order_totals); called where every
       sector's sums belong to its rung */
    void order_totals() {
        std::vector<int64_t> nv(ns);
        for (int s = 0; s < ns; ++s) nv[s] = ladder[rung[s]].n;
        qmci::order_totals(packed, m, nv.data(), sums.data(), Tr, Ti);
    }

    /* Precision of each sector (qmc_choose_precision's rule) from the probe with island bins: pr holds the probe's
       n_sectors x n_slots x 4 sums, then n_sectors x QMC_ISLAND_BINS x QMC_ISLAND_BIN_WORDS(n_slots) bins, over
       n_samp points per sector.  Before the first evaluation (no totals) the decision is provisional:
       revisit_precision takes it again on the same probe once totals exist. */
    void set_precision(const std::vector<double> &pr, int64_t n_samp, qmc_result &res) {
        const double budget = (opt.fp32_budget > 0 ? opt.fp32_budget : 0.1) * opt.rel_tol;
        const bool totals = qmci::choose_precision(packed, pr.data(), pr.data() + (size_t)ns * h->n_slots * 4, n_samp,
                                                   Tr, Ti, budget, prec.data(), nullptr, nullptr);
        for (int s = 0; s < ns; ++s)
            if (forced64[s]) prec[s] = 0;
        count_precision(res);
        probe_due = false;
        prec_provisional = !totals;
        if (&pr != &probe_pr) probe_pr = pr;
        probe_n = n_samp;
    }

    void count_precision(qmc_result &res) const {
        res.fp64_reruns = res.island_sectors = 0;
        for (int s = 0; s < ns; ++s) {
            res.fp64_reruns += prec[s] == 0;
            res.island_sectors += prec[s] >= 2;
        }
    }

    /* true when the precision was taken again or a sector was moved to FP64 (the caller copies prec to the device
       before the next pass) */
    bool revisit_precision(qmc_result &res) {
        const bool changed = prec_changed;
        prec_changed = false;
        if (prec_provisional && !probe_pr.empty()) {
            double tmax = 0.0;
            for (size_t k = 0; k < Tr.size(); ++k) tmax = std::max(tmax, std::hypot(Tr[k], Ti[k]));
            if (tmax > 0.0) {
                set_precision(probe_pr, probe_n, res);
                return true;
            }
        }
        return changed;
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
        /* non-finite sums of a sector just evaluated (an FP32 overflow at points the probe did not sample, or a
           singular point): in a mixed integration the sector runs in FP64 from now on and this step is evaluated
           again; in FP64 the integration stops */
        bool redo = false;
        const size_t per_sector = (size_t)m * h->n_slots * 2;
        for (int s = 0; s < ns; ++s) {
            if (!active[s]) continue;
            bool finite = true;
            for (size_t q = 0; q < per_sector && finite; ++q) finite = std::isfinite(sums[(size_t)s * per_sector + q]);
            if (finite) continue;
            res.nonfinite_sectors += 1;
            if (!mixed || prec[s] == 0) return QMC_ERR_NONFINITE;
            forced64[s] = 1;
            prec[s] = 0;
            prec_changed = true;
            redo = true;
        }
        if (redo) {
            count_precision(res);
            return QMC_PENDING;
        }
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
        if (mixed) order_totals();
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
            qmci::combine_core(packed, m, invn.data(), s, sums.data(), Qs.data(), ms.data(), es.data());
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
    if (c->abort_host) cudaFreeHost((void *)c->abort_host);
    delete c;
    return QMC_OK;
}

int qmc_load_sectors(qmc_ctx *c, const void *table, size_t bytes, int32_t *id) {
    if (!c || !table || !id) return QMC_ERR_ARG;
    const int rc = qmci::validate_table(table, bytes);
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

namespace {

/* sets *flag at `deadline` unless disarmed first (destruction disarms and joins) */
struct DeadlineTimer {
    std::mutex mu;
    std::condition_variable cv;
    bool done = false;
    std::thread th;
    DeadlineTimer(volatile int32_t *flag, std::chrono::steady_clock::time_point deadline) {
        th = std::thread([this, flag, deadline] {
            std::unique_lock<std::mutex> lk(mu);
            if (!cv.wait_until(lk, deadline, [this] { return done; })) *flag = 1;
        });
    }
    ~DeadlineTimer() {
        {
            std::lock_guard<std::mutex> g(mu);
            done = true;
        }
        cv.notify_all();
        th.join();
    }
};

}  // namespace

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
    const size_t probe_words = (size_t)ns * h->n_slots * 4;
    const size_t bin_words = (size_t)ns * QMC_ISLAND_BINS * QMC_ISLAND_BIN_WORDS(h->n_slots);
    if (!rc && st.mixed) rc = dev_reserve(c, c->probe, (probe_words + bin_words) * sizeof(double));
    if (rc) return res->status = rc;
    /* a time limit stops a running pass: the kernels read the abort flag at every work item */
    std::unique_ptr<DeadlineTimer> timer;
    if (opt->max_seconds > 0) {
        if (!c->abort_host) {
            void *f = nullptr;
            if (cudaHostAlloc(&f, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess ||
                cudaHostGetDevicePointer((void **)&c->abort_dev, f, 0) != cudaSuccess) {
                if (f) cudaFreeHost(f);
                c->abort_dev = nullptr;
                return res->status = QMC_ERR_CUDA;
            }
            c->abort_host = static_cast<volatile int32_t *>(f);
        }
        *c->abort_host = 0;
        const auto limit = std::chrono::duration_cast<std::chrono::steady_clock::duration>(
            std::chrono::duration<double>(opt->max_seconds));
        timer.reset(new DeadlineTimer(c->abort_host, t0 + limit));
    }
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
            std::vector<double> pr(probe_words + bin_words);
            rc = qmc_probe_islands(st.packed, I.dpacked.p, &passes[st.probe_item], (const double *)c->shifts.p,
                                   (const double *)c->lambda.p, st.probe_samples(), (double *)c->probe.p,
                                   (double *)c->probe.p + probe_words, c->stream);
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(pr.data(), c->probe.p, pr.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost, c->stream));
            if (!rc) rc = cuda_status(cudaStreamSynchronize(c->stream));
            if (!rc) {
                st.set_precision(pr, std::min<int64_t>(st.probe_samples(), passes[st.probe_item].lattice.n), *res);
                rc = cuda_status(cudaMemcpyAsync(c->prec.p, st.prec.data(), ns * sizeof(int32_t),
                                                 cudaMemcpyHostToDevice, c->stream));
            }
        } else if (!rc && st.revisit_precision(*res)) {
            rc = cuda_status(cudaMemcpyAsync(c->prec.p, st.prec.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice,
                                             c->stream));
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
            items[k].abort_flag = timer ? c->abort_dev : nullptr;
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
        if (timer && *c->abort_host) { /* the pass was stopped at the time limit: its sums are incomplete */
            status = QMC_ERR_TIMEOUT;
            break;
        }
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
    double sec_used = 0.0;         /* loop seconds charged to it so far: its share of each round's time */
    bool cancelled = false;
    int state = REQ_QUEUED;
    int abort_slot = -1;           /* its abort flag in Serving::abort_host while it runs, or -1 */
};

}  // namespace

/* abort flags of running requests: mapped pinned host memory, read by the kernels at every work item */
#define QMC_ABORT_SLOTS 1024

struct Serving {
    std::thread th;
    volatile int32_t *abort_host = nullptr; /* QMC_ABORT_SLOTS flags; a running request owns one */
    int32_t *abort_dev = nullptr;           /* the same flags as the device sees them */
    std::vector<char> slot_used;
    /* watchdog: sets the abort flag of a running request whose time limit passes during a round */
    std::thread wd;
    std::mutex wmu;
    std::condition_variable wcv;
    bool wstop = false;
    std::vector<std::pair<std::chrono::steady_clock::time_point, int>> armed; /* (deadline, slot) */
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
    /* load estimate for shedding: per integral id, a moving average of the loop seconds its completed requests
       were charged */
    std::map<int32_t, double> sec_per_request;
};

namespace {

void release_request(qmc_ctx *c, Request &r) {
    for (DevBuf *b : {&r.dpacked, &r.dshifts, &r.dlambda, &r.dsums, &r.dfails, &r.dprec, &r.dprobe}) dev_release(c, *b);
}

void finish(Serving *S, qmc_ctx *c, Request &r, int status) {
    release_request(c, r);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (r.abort_slot >= 0) {
            S->abort_host[r.abort_slot] = 0;
            S->slot_used[r.abort_slot] = 0;
            r.abort_slot = -1;
        }
    }
    if (status != QMC_OK && r.res.n_final == 0 && !r.st.ladder.empty()) r.res.n_final = r.st.ladder[0].n;
    r.res.status = status;
    r.res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
    r.res.queued_seconds = std::chrono::duration<double>(r.t_admit - r.t_submit).count();
    std::lock_guard<std::mutex> g(S->mu);
    r.state = REQ_DONE;
    S->stats.completed += 1;
    if (status == QMC_OK && r.sec_used > 0.0) {
        auto it = S->sec_per_request.find(r.integral_id);
        if (it == S->sec_per_request.end()) S->sec_per_request[r.integral_id] = r.sec_used;
        else it->second = 0.7 * it->second + 0.3 * r.sec_used;
    }
}

/* seconds of device work a queued request still needs by the loop's estimate (0 when it has no history) */
double est_seconds(const Serving *S, int32_t integral_id, double used) {
    auto it = S->sec_per_request.find(integral_id);
    if (it == S->sec_per_request.end()) return 0.0;
    return std::max(0.0, it->second - used);
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
    if (!rc)
        rc = dev_reserve(c, r.dprobe,
                         ((size_t)ns * h->n_slots * 4 + (size_t)ns * QMC_ISLAND_BINS * QMC_ISLAND_BIN_WORDS(h->n_slots))
                             * sizeof(double));
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
    const size_t probe_words = (size_t)h->n_sectors * h->n_slots * 4;
    std::vector<double> pr(probe_words + (size_t)h->n_sectors * QMC_ISLAND_BINS * QMC_ISLAND_BIN_WORDS(h->n_slots));
    int rc = qmc_probe_islands(r.packed.data(), r.dpacked.p, &r.passes[r.st.probe_item], (const double *)r.dshifts.p,
                               (const double *)r.dlambda.p, r.st.probe_samples(), (double *)r.dprobe.p,
                               (double *)r.dprobe.p + probe_words, S->stream);
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(pr.data(), r.dprobe.p, pr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                         S->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(S->stream));
    if (rc) return rc;
    r.st.set_precision(pr, std::min<int64_t>(r.st.probe_samples(), r.passes[r.st.probe_item].lattice.n), r.res);
    return cuda_status(cudaMemcpyAsync(r.dprec.p, r.st.prec.data(), r.st.ns * sizeof(int32_t), cudaMemcpyHostToDevice,
                                       S->stream));
}

/* sets the abort flag of each armed slot when its deadline passes (the serving loop arms the running round's
   requests that have a time limit, and disarms them when the round is over) */
void watchdog(Serving *S) {
    std::unique_lock<std::mutex> lk(S->wmu);
    while (!S->wstop) {
        if (S->armed.empty()) {
            S->wcv.wait(lk);
            continue;
        }
        auto next = S->armed.front().first;
        for (const auto &a : S->armed) next = std::min(next, a.first);
        S->wcv.wait_until(lk, next);
        const auto now = std::chrono::steady_clock::now();
        for (auto it = S->armed.begin(); it != S->armed.end();) {
            if (it->first <= now) {
                S->abort_host[it->second] = 1;
                it = S->armed.erase(it);
            } else {
                ++it;
            }
        }
    }
}

void serve_loop(qmc_ctx *c) {
    Serving *S = c->serving;
    cudaSetDevice(c->device);
    std::chrono::steady_clock::time_point t_iter;
    for (;;) {
        std::vector<std::shared_ptr<Request>> fresh, cancelled, expired;
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
            t_iter = std::chrono::steady_clock::now();
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
               sums plus a first-pass share of scratch; at least one request always runs.  With load estimates
               (est_seconds), a round advances every active request together, so an admitted request ends no
               earlier than the work of all requests running beside it: a request with a time limit is shed when
               its own work on top of the work ahead (the active, compiling and just admitted requests'
               remaining) would end past its limit, and the queue waits while admitting its head would end the
               work ahead past the tightest limit among those running.  Both compare with a margin of
               QMC_SHED_MARGIN on the estimates. */
            const auto now = std::chrono::steady_clock::now();
            auto left = [&](const Request &q) {
                return q.opt.max_seconds > 0
                           ? q.opt.max_seconds - std::chrono::duration<double>(now - q.t_submit).count()
                           : std::numeric_limits<double>::infinity();
            };
            double ahead = 0.0, tight = std::numeric_limits<double>::infinity();
            for (const auto &a : S->active) {
                ahead += est_seconds(S, a->integral_id, a->sec_used);
                tight = std::min(tight, left(*a));
            }
            for (const auto &a : S->compiling) {
                ahead += est_seconds(S, a->integral_id, 0.0);
                tight = std::min(tight, left(*a));
            }
            while (!S->queue.empty()) {
                auto r = S->queue.front();
                if (r->cancelled) {
                    S->queue.pop_front();
                    r->state = REQ_DONE;
                    r->res.status = QMC_ERR_CANCELLED;
                    S->stats.completed += 1;
                    continue;
                }
                const double mine = left(*r);
                if (mine < 0.0) {
                    /* its deadline passed in the queue: it leaves without work (finished below, outside this
                       lock), which keeps an overloaded loop's device time for requests that can still finish */
                    S->queue.pop_front();
                    r->t_admit = now;
                    expired.push_back(r);
                    continue;
                }
                const double own = est_seconds(S, r->integral_id, 0.0);
                const double end = QMC_SHED_MARGIN * (ahead + own);
                if (own > 0.0 && end > mine) {
                    S->queue.pop_front();
                    r->t_admit = now;
                    expired.push_back(r);
                    S->stats.shed += 1;
                    continue;
                }
                const bool running = !S->active.empty() || !fresh.empty();
                if (running && own > 0.0 && end > tight) break;
                const size_t est = 2 * r->table.size() + ((size_t)8 << 20);
                if (running && in_use + est > c->budget) break;
                S->queue.pop_front();
                fresh.push_back(r);
                in_use += est;
                ahead += own;
                tight = std::min(tight, mine);
                if (S->active.size() + fresh.size() >= QMC_MAX_JOBS / 4) break;
            }
        }
        /* device buffers of cancelled and newly admitted requests: the context mutex guards the budget */
        {
            std::lock_guard<std::mutex> g(c->mu);
            for (auto &r : cancelled) finish(S, c, *r, QMC_ERR_CANCELLED);
            for (auto &r : expired) finish(S, c, *r, QMC_ERR_TIMEOUT);
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
            /* its abort flag (none when all slots are taken: it then stops at round boundaries only) */
            for (int k = 0; k < QMC_ABORT_SLOTS && r->abort_slot < 0; ++k)
                if (!S->slot_used[k]) {
                    S->slot_used[k] = 1;
                    S->abort_host[k] = r->cancelled ? 1 : 0;
                    r->abort_slot = k;
                }
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
            else if (!rc && r->st.revisit_precision(r->res))
                rc = cuda_status(cudaMemcpyAsync(r->dprec.p, r->st.prec.data(), r->st.ns * sizeof(int32_t),
                                                 cudaMemcpyHostToDevice, S->stream));
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
                b.abort_flag = r.abort_slot >= 0 ? S->abort_dev + r.abort_slot : nullptr;
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
        /* time limits of the round's requests: past one, the watchdog stops that request's remaining work items
           (armed before the launch: the copies back below go to pageable memory and block until the round ends) */
        {
            std::lock_guard<std::mutex> gw(S->wmu);
            S->armed.clear();
            for (auto &r : batch)
                if (r->opt.max_seconds > 0 && r->abort_slot >= 0)
                    S->armed.push_back({r->t_submit + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                                          std::chrono::duration<double>(r->opt.max_seconds)),
                                        r->abort_slot});
        }
        S->wcv.notify_all();
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
            std::lock_guard<std::mutex> gw(S->wmu);
            S->armed.clear();
        }
        /* the round's time (the whole iteration: admission, preparation, probes, the batch, the copies back) is
           charged to its requests in proportion to their evaluations' algorithmic flop, FP64 evaluations
           weighted by QMC_FP64_COST */
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_iter).count();
        std::vector<double> wv(batch.size(), 0.0);
        double round_work = 0.0;
        for (size_t i = 0; i < batch.size() && !rc; ++i) {
            Request &r = *batch[i];
            const PackedSector *ps = sectors_of(r.packed.data());
            std::vector<double> fl(r.st.ns, 0.0);
            for (int pi = 0; pi < r.st.ns; ++pi) fl[ps[pi].orig_index] = ps[pi].flops;
            for (const qmc_pass &p : r.passes)
                for (int s = 0; s < r.st.ns; ++s)
                    if (!p.sector_active || p.sector_active[s]) {
                        const bool f32 = p.precision == QMC_PREC_MIXED && r.st.prec[s] != 0;
                        wv[i] += fl[s] * (double)r.st.m * (double)p.lattice.n * (f32 ? 1.0 : QMC_FP64_COST);
                    }
            round_work += wv[i];
        }
        if (!rc && round_work > 0.0)
            for (size_t i = 0; i < batch.size(); ++i) batch[i]->sec_used += sec * wv[i] / round_work;
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
                /* stopped within the round (cancelled, or its time limit passed): its sums are incomplete */
                if (r.abort_slot >= 0 && S->abort_host[r.abort_slot]) {
                    bool cancelled;
                    {
                        std::lock_guard<std::mutex> g3(S->mu);
                        cancelled = r.cancelled;
                    }
                    finish(S, c, r, cancelled ? QMC_ERR_CANCELLED : QMC_ERR_TIMEOUT);
                    done.push_back(rp);
                    continue;
                }
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
    {
        std::lock_guard<std::mutex> g(c->serving->wmu);
        c->serving->wstop = true;
    }
    c->serving->wcv.notify_all();
    if (c->serving->wd.joinable()) c->serving->wd.join();
    cudaSetDevice(c->device);
    if (c->serving->stream) cudaStreamSynchronize(c->serving->stream);
    for (auto &kv : c->serving->all) release_request(c, *kv.second);
    dev_release(c, c->serving->scratch);
    if (c->serving->stream) cudaStreamDestroy(c->serving->stream);
    if (c->serving->abort_host) cudaFreeHost((void *)c->serving->abort_host);
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
            void *flags = nullptr;
            if (cudaHostAlloc(&flags, QMC_ABORT_SLOTS * sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess ||
                cudaHostGetDevicePointer((void **)&S->abort_dev, flags, 0) != cudaSuccess) {
                if (flags) cudaFreeHost(flags);
                cudaStreamDestroy(S->stream);
                delete S;
                return QMC_ERR_CUDA;
            }
            S->abort_host = static_cast<volatile int32_t *>(flags);
            for (int k = 0; k < QMC_ABORT_SLOTS; ++k) S->abort_host[k] = 0;
            S->slot_used.assign(QMC_ABORT_SLOTS, 0);
            c->serving = S;
            S->wd = std::thread(watchdog, S);
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
    /* a running request stops within the round: the kernels skip its remaining work items */
    if (it->second->abort_slot >= 0) S->abort_host[it->second->abort_slot] = 1;
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
