/*
 * Passes of the hot path on the device: launch planning (runs of sectors, items, chunks), batches of passes in
 * shared persistent launches (job tables), the fixed-order reductions, the FP32/FP64 precision probe, sampled
 * per-point values, the launch-shape autotuner, and the combination of per-(sector, shift) sums into Laurent
 * coefficients with errors.
 *
 * Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals", Chin. Phys. C 40 (2016) 033103:
 * Sec. III (Eqs. 16-21), the shifted rank-1 lattice estimator.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lattice_table.h"
#include "qmc_host_internal.h"

namespace {

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

}  // namespace

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
                /* class 2 (endpoint exponents alpha <= -2): FP64 whatever the pass's precision */
                const bool fp64_only = c == 2;
                if ((!mixed || fp64_only) && prec == 1) continue;
                if (mixed && !fp64_only && prec == 0 && !b.pass.sector_precision) continue;
                Job J;
                std::memset(&J, 0, sizeof(J));
                J.packed = static_cast<const unsigned char *>(b.packed_dev);
                J.sectors_off = h->sectors_off;
                J.terms_off = h->terms_off;
                J.termsf_off = h->termsf_off;
                J.chunks = pl.chunks;
                J.shifts = b.shifts_dev;
                J.lambda = b.lambda_dev;
                J.sector_prec = (mixed && !fp64_only) ? b.pass.sector_precision : nullptr;
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
                J.abort = b.abort_flag;
                J.eU0 = h->eU0;
                J.eU1 = h->eU1;
                J.eF0 = h->eF0;
                J.eF1 = h->eF1;
                const void *gen = nullptr;
                if (prec == 1 && use_generated(b.pass)) {
                    rc = qmc_gen_kernel(b.packed_host, QMC_PREC_MIXED, c, &gen);
                    if (rc) return rc;
                } else if (prec == 0 && !fp64_only && use_generated64(b.pass, h)) {
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
    /* Launch order: the map orders keys by (dim, class, series length) and then precision, so the FP64 launch
       of a mixed pass's items precedes their FP32 launch.  Sectors with FP64 islands rely on it: the FP64 kernel
       writes an item's island partial, the FP32 kernel then adds the rest to it. */
    static_assert(QMC_PREC_FP64 < QMC_PREC_MIXED, "FP64 launches must sort before FP32 launches");
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

namespace {

int probe(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
          const double *lambda_dev, int64_t n_sample, double *out_dev, double *bins_dev, void *stream) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !packed_dev || !pass || !shift_dev || !lambda_dev || !out_dev || n_sample < 1) return QMC_ERR_ARG;
    Plan pl;
    int rc = make_plan(h, pass, pl);
    if (rc) return rc;
    for (int c = 0; c < 2; ++c) { /* class 2 always runs in FP64: nothing to probe */
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
        a.bins = bins_dev;
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

}  // namespace

int qmc_probe_precision(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
                        const double *lambda_dev, int64_t n_sample, double *out_dev, void *stream) {
    return probe(packed_host, packed_dev, pass, shift_dev, lambda_dev, n_sample, out_dev, nullptr, stream);
}

int qmc_probe_islands(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
                      const double *lambda_dev, int64_t n_sample, double *out_dev, double *bins_dev, void *stream) {
    if (!bins_dev) return QMC_ERR_ARG;
    return probe(packed_host, packed_dev, pass, shift_dev, lambda_dev, n_sample, out_dev, bins_dev, stream);
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
    const int cls = ps[psec].taylor ? 2 : (ps[psec].kind == 2 ? 1 : 0);
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

namespace qmci {

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

}  // namespace qmci

extern "C" {

int qmc_combine(const void *packed_host, const qmc_pass *pass, const double *sums, double *Q, double *mean,
                double *err) {
    const PackedHeader *h = header_of(packed_host);
    if (!h || !pass || !sums || !Q || !mean || !err || pass->n_shifts < 1 || pass->lattice.n < 1) return QMC_ERR_ARG;
    std::vector<double> invn(h->n_sectors, 1.0 / (double)pass->lattice.n);
    return qmci::combine_core(packed_host, pass->n_shifts, invn.data(), -1, sums, Q, mean, err);
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
    return qmci::combine_core(packed_host, n_shifts, invn.data(), -1, sums, Q, mean, err);
}

}  // extern "C"
