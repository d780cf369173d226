/*
 * qmcfi -- quasi-Monte Carlo evaluation of sector-decomposed Feynman integrals on one GB300 GPU (sm_103a).
 *
 * Method: Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals",
 * Chin. Phys. C 40 (2016) 033103.  The library evaluates the eps-expansion coefficients of every sector
 * integral of Sec. II, Eq. (9) -- with the endpoint subtraction of Eqs. (10)-(12) and, for sectors whose
 * F polynomial changes sign, the contour deformation of Eq. (14) with its Jacobian -- at the points of a
 * randomly shifted rank-1 lattice (Sec. III, Eqs. 17-18) after a periodising transform (Eq. 21), and sums
 * them into per-shift estimates whose spread gives the error (Eqs. 19-20).
 *
 * Conventions
 *   - Every function returns an int status: QMC_OK (0), QMC_PENDING (1), or a negative QMC_ERR_* code;
 *     qmc_strerror() names it.  No C++ exception crosses this interface.
 *   - Inputs are borrowed: the library copies what it keeps.  Outputs are caller-owned.  Pointers documented
 *     as "device" must point to memory of the current CUDA device; all others are host pointers.
 *   - Functions taking a `stream` (a cudaStream_t passed as void*, NULL = legacy default stream) are
 *     asynchronous: they enqueue work and return; the caller synchronises before reading device outputs.
 *   - A sector table is the binary format written by paper_1508_02512_gb300/tables.py (see qmc_prepare).
 *   - Series slots: for a sector with sigma singular variables, slot n of its per-shift sums holds the
 *     coefficient of eps^(n - sigma) of the sector integral; slots beyond the sector's order range are zero.
 */
#ifndef QMCFI_H
#define QMCFI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMC_OK 0
#define QMC_PENDING 1
#define QMC_ERR_ARG (-1)          /* bad argument (null pointer, size out of range, ...) */
#define QMC_ERR_TABLE (-2)        /* malformed or inconsistent sector table */
#define QMC_ERR_UNSUPPORTED (-3)  /* valid but outside what the kernels implement (dim > 6, exponent > 15, ...) */
#define QMC_ERR_KINEMATICS (-4)   /* kinematics make a leading coefficient vanish */
#define QMC_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define QMC_ERR_MEMORY (-6)       /* device memory budget or capacity exceeded */
#define QMC_ERR_DEFORMATION (-7)  /* Im F(z) > 0 persists after the lambda-halving cap */
#define QMC_ERR_TIMEOUT (-8)      /* max_seconds reached before the requested accuracy */
#define QMC_ERR_CANCELLED (-9)
#define QMC_ERR_NOT_FOUND (-10)   /* unknown integral or request id */
#define QMC_ERR_NO_DEVICE (-11)   /* no usable CUDA device */
#define QMC_ERR_NOT_CONVERGED (-12) /* lattice ladder exhausted before the requested accuracy */
#define QMC_ERR_CODEGEN (-13)     /* run-time compilation of a generated evaluator failed (NVRTC) */
#define QMC_ERR_NONFINITE (-14)   /* a sector's FP64 sums are not finite (overflow or a singular point) */

#define QMC_MAX_DIM 6             /* sector dimension (7 propagators) */
#define QMC_MAX_SLOTS 5           /* series slots per sector */
#define QMC_MAX_ORDERS 8          /* Laurent orders of a result */

enum { QMC_PREC_FP64 = 0, QMC_PREC_MIXED = 1 };

/* Polynomial evaluator of a pass:
 *   QMC_EVAL_AUTO (0)      = QMC_EVAL_GENERATED
 *   QMC_EVAL_TABLE         the kernels walk each sector's staged term table and decode its exponents per point
 *   QMC_EVAL_GENERATED     straight-line code generated for the family of sector tables (same exponents) and
 *                          compiled at run time with NVRTC on first use (qmc_gen_compile), in each precision
 *                          the pass evaluates in; the coefficients are still read from the staged table, so
 *                          kinematic points of one family share it. */
enum { QMC_EVAL_AUTO = 0, QMC_EVAL_TABLE = 1, QMC_EVAL_GENERATED = 2 };

/* A rank-1 lattice (Eq. 17): prime size n and generating vector z (a dim-d sector uses z[0..d-1]). */
typedef struct {
    int64_t n;
    uint32_t z[QMC_MAX_DIM];
} qmc_lattice;

/* Summary of a prepared integral (filled by qmc_prepare). */
typedef struct {
    int32_t n_sectors, dim, loops, n_invariants;
    int32_t order_min, order_max;  /* Laurent orders of the integral the preparation serves */
    int32_t kmax;                  /* highest eps order needed from each sector integral */
    int32_t n_slots;               /* series slots per sector in every output (<= QMC_MAX_SLOTS) */
    int32_t n_deformed, n_negative, max_sigma, max_terms;
    int32_t pre_low;               /* lowest eps power of Gamma(N_nu - L D/2) / prod Gamma(nu_j) */
    int32_t n_pre;
    double pre[QMC_MAX_ORDERS + 4]; /* its coefficients for eps^pre_low, eps^(pre_low+1), ... */
    int64_t packed_bytes;          /* size of the packed device image */
    double flops_per_eval;         /* algorithmic FP work per (sector, shift, point), mean over sectors */
    double transcendentals_per_eval;
} qmc_info;

/* Per-sector description inside a packed image. */
typedef struct {
    int32_t kind;      /* 0: F > 0 on the cube; 1: F < 0 (real, phase exp(i pi eF(eps)) applied on the host);
                          2: deformed (Eq. 14) */
    int32_t sigma;     /* number of variables with exponent alpha <= -1 (Eqs. 10-12) */
    int32_t n_slots;   /* slots this sector fills */
    int32_t n_terms;   /* polynomial terms staged in shared memory (U, F, dF, d2F) */
    double flops;      /* algorithmic FP work per point */
} qmc_sector_desc;

/* One pass of the hot path over one integral: every sector x shift x lattice point. */
typedef struct {
    qmc_lattice lattice;
    int32_t n_shifts;          /* m random shifts, 1..4096 */
    int32_t transform_r;       /* periodising transform order 0..3 (Eq. 21 is r = 1) */
    int32_t precision;         /* QMC_PREC_FP64 or QMC_PREC_MIXED */
    int32_t block;             /* threads per block: 0 = default (128), else 32..256 and a multiple of 32; at most
                                  128 for generated FP32 evaluators of 5- and 6-dimensional sectors */
    int32_t points_per_thread; /* 0 = default, else 1..64 */
    int32_t grid;              /* blocks of the persistent kernel: 0 = one wave on the device */
    int32_t evaluator;         /* QMC_EVAL_* of the FP32 evaluation */
    int32_t reserved;
    const int32_t *sector_precision; /* QMC_PREC_MIXED only: device array, one entry per sector (table order):
                                        1 = evaluate in FP32; 2 + L (0 <= L < QMC_ISLAND_LEVELS) = FP32 except
                                        at the sector's island points of level L, which run in FP64 (see
                                        qmc_probe_islands); anything else = FP64.  NULL = every sector FP32 */
    const int32_t *sector_active;    /* HOST array, one entry per sector (table order): nonzero = evaluate this
                                        sector; NULL = every sector.  The pass writes sums/fails of the evaluated
                                        sectors only and leaves the others' entries as they were, so passes of
                                        different lattice sizes can fill one output (per-sector lattices). */
} qmc_pass;

/* One pass of one prepared integral, as an element of a batch (qmc_eval_batch). */
typedef struct {
    const void *packed_host;   /* image from qmc_prepare, host copy */
    const void *packed_dev;    /* the same image in device memory (16-byte aligned) */
    qmc_pass pass;
    const double *shifts_dev;  /* pass.n_shifts x 6 */
    const double *lambda_dev;  /* one per sector */
    double *sums_dev;          /* outputs as in qmc_eval_sums */
    int64_t *fails_dev;
    const volatile int32_t *abort_flag; /* NULL, or a device-visible int32 (e.g. mapped pinned host memory) that the
                                           kernels read at every work item: once nonzero, the pass's remaining
                                           items are skipped (their partials become zero) and its sums are
                                           meaningless.  Stops a long pass early (cancellation, time limits). */
} qmc_batch_item;

/* Text for a status code (static storage). */
const char *qmc_strerror(int status);

/* Library version (major * 10000 + minor * 100 + patch). */
int qmc_version(void);

/*
 * qmc_prepare -- host only; no CUDA call.
 * Parses and validates a sector table (Sec. II, Eq. 9: per sector the exponents A_j + B_j eps, a constant
 * Jacobian factor D and the polynomials Ut, Ft with coefficients linear in the kinematic invariants; tables of
 * the iterated and of the geometric decomposition have the same form), evaluates the coefficients at
 * `invariants` (n_invariants values in the table's invariant order), classifies every sector by the signs of
 * Ft's coefficients (kind 0/1/2), derives for deformed sectors the gradient and Hessian polynomials of Ft that
 * Eq. (14) and its Jacobian need, computes the Gamma prefactor series of Eq. (2), and writes the packed image
 * that the kernels read (relocatable: offsets only; copy it to device memory as is).
 *   order_min..order_max: Laurent orders of the integral the image must serve (order_max - order_min < 8).
 *   packed: output buffer of packed_capacity bytes, or NULL to query info->packed_bytes only.
 * Sectors with an exponent A_j = -2 or -3 (Taylor subtraction of Eq. 11 with p = 1, 2) are taken when F~ keeps
 * one sign on the cube (no deformation) and at most two variables have A_j <= -1: they form a third class that
 * always runs in FP64 (table evaluator, truncated power series of U~ and F~ in the expanded variables).
 * Errors: QMC_ERR_ARG, QMC_ERR_TABLE, QMC_ERR_UNSUPPORTED (among others: A_j <= -4, A_j <= -2 in a deformed
 * sector or beside more than one other singular variable), QMC_ERR_KINEMATICS, QMC_ERR_MEMORY (capacity).
 */
int qmc_prepare(const void *table, size_t table_bytes, const double *invariants, int32_t n_invariants,
                int32_t order_min, int32_t order_max, void *packed, size_t packed_capacity, qmc_info *info);

/* Description of sector `sector` (table order) of a packed image (host pointer).  QMC_ERR_ARG if out of range. */
int qmc_sector_desc_get(const void *packed, int32_t sector, qmc_sector_desc *out);

/* Bytes of device scratch that qmc_eval_sums needs for `pass` on this image (per-item partial sums, fail
 * counters and work counters).  Returns 0 for invalid arguments. */
size_t qmc_scratch_bytes(const void *packed, const qmc_pass *pass);

/*
 * qmc_eval_sums -- the hot path (Sec. III, Eqs. 16-18), asynchronous on `stream`.
 * For every sector s, shift k and slot n:
 *   sums[((s * n_shifts) + k) * n_slots + n] = sum_{i < lattice.n} w(x_i) I_s(t(x_i)) coefficient n,
 *   x_i = {i z / n + Delta_k},  stored as (re, im) double pairs,
 *   fails[s * n_shifts + k] = number of points of deformed sectors with Im F(z) > 0 (Eq. 14 sign check).
 * packed_host / packed_dev: the same image in host and device memory.  shifts_dev: n_shifts x 6 doubles in
 * [0,1).  lambda_dev: one deformation parameter per sector (table order).  scratch_dev: at least
 * qmc_scratch_bytes() bytes, 256-byte aligned, owned by the caller; contents need no initialisation and are
 * overwritten.  Sums are deterministic: independent of grid size and scheduling for fixed block and
 * points_per_thread.  Errors: QMC_ERR_ARG, QMC_ERR_UNSUPPORTED, QMC_ERR_MEMORY (scratch too small), QMC_ERR_CUDA.
 */
int qmc_eval_sums(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                  const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, double *sums_dev,
                  int64_t *fails_dev, void *stream);

/*
 * qmc_eval_batch -- many passes (different integrals, kinematic points, lattices or shifts) in shared launches,
 * asynchronous on `stream`: every (pass, sector class, precision) becomes a job, and jobs that use the same kernel
 * instantiation go into one persistent launch whose blocks take work items across all of them (continuous
 * batching for the serving loop).  Each pass's results are identical, bit for bit, to running it alone with
 * qmc_eval_sums (per-item work and reduction order do not depend on the batch).  scratch: at least
 * qmc_batch_scratch_bytes(items, n) bytes, 256-byte aligned.  The paper evaluates one integral at a time; the
 * batching is this library's (Sec. III, Eqs. 16-18 per pass).
 */
size_t qmc_batch_scratch_bytes(const qmc_batch_item *items, int32_t n);
int qmc_eval_batch(const qmc_batch_item *items, int32_t n, void *scratch_dev, size_t scratch_bytes, void *stream);

/* The two launches of qmc_eval_sums, exposed separately (same arguments and semantics): qmc_eval_partials runs
 * the evaluation kernel and leaves one partial sum per work item and slot in the scratch buffer;
 * qmc_reduce_partials sums them per (sector, shift) in a fixed order into sums/fails.  The scratch buffer must
 * not be reused between the two calls. */
int qmc_eval_partials(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                      const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, void *stream);
int qmc_reduce_partials(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const void *scratch_dev,
                        size_t scratch_bytes, double *sums_dev, int64_t *fails_dev, void *stream);

/*
 * qmc_probe_precision -- FP32-versus-FP64 discrepancy per sector (the mixed-precision budget check),
 * asynchronous on `stream`.  For each sector s, a strided sample of n_sample lattice points i = k * (n / n_sample)
 * of the shift shift_dev[0..5] is evaluated by both the FP32 and the FP64 device code; per slot it writes
 *   out[(s * n_slots + slot) * 4 + {0,1,2,3}] = sum |v64|, sum |v32 - v64|, sum (v32 - v64) re, im.
 * The FP32 values come from the table evaluator whatever pass->evaluator says (the generated evaluator performs
 * the same products and FMAs, summed in another order).
 * The paper evaluates in one precision; the split into an FP32 path, FP64 islands near the singular faces and
 * FP64 sectors under an error budget is this library's (Sec. II, after Eq. 12, motivates FP64 where cancellation
 * is large).
 */
int qmc_probe_precision(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
                        const double *lambda_dev, int64_t n_sample, double *out_dev, void *stream);

/*
 * FP64 islands.  The subtraction of Eq. 11 cancels near the faces t_j = 0 of a sector's singular variables (the
 * remark after Eq. 12): that is where FP32 loses the digits a sector's error budget needs.  A mixed pass can keep
 * such a sector in FP32 and evaluate only its island points in FP64.  A lattice point is an island at level L
 * when prod_{j singular} (k_j + 1) / n < 10^-(L+1), k_j = floor(n x_j) the integer part of its shifted lattice
 * coordinate; the product is taken in FP32, each factor and product correctly rounded, floored at 1e-30 after
 * each factor.  Its island bin is the number of levels it is an island at (0 .. QMC_ISLAND_LEVELS).
 *
 * qmc_probe_islands -- qmc_probe_precision's sample and output, and in addition, per sector and island bin,
 * the sample points in the bin and per slot sums over them of e = v32 - v64:
 *   bins_dev[(s * QMC_ISLAND_BINS + b) * (1 + 4 n_slots) + 0]                    = points of sector s in bin b
 *   bins_dev[(s * QMC_ISLAND_BINS + b) * (1 + 4 n_slots) + 1 + 4 slot + {0..3}] = sum |e|, sum e (re, im),
 *                                                                                 sum |e|^2 in that slot
 * With islands at level L the FP32 points are those of bins 0..L.  bins_dev must not be NULL (QMC_ERR_ARG).
 * Each sector's sample is spread over a cluster of blocks and reduced in a fixed order (deterministic).
 */
#define QMC_ISLAND_LEVELS 6
#define QMC_ISLAND_BINS (QMC_ISLAND_LEVELS + 1)
#define QMC_ISLAND_BIN_WORDS(n_slots) (1 + 4 * (n_slots)) /* doubles per (sector, bin) of bins_dev */
int qmc_probe_islands(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shift_dev,
                      const double *lambda_dev, int64_t n_sample, double *out_dev, double *bins_dev, void *stream);

/*
 * qmc_choose_precision -- per-sector precision codes for a mixed pass (qmc_pass.sector_precision), as qmc_integrate
 * and the serving loop choose them.  Host-only: all arrays are host memory.
 *   probe, bins: qmc_probe_islands' outputs (copied to the host), n_sample points per sector.
 *   sums, n_sector, n_shifts: the current sums (qmc_eval_sums layout) and each sector's lattice size (table
 *     order), for the estimate T_k of each eps order summed over sectors before the Gamma prefactor; sums = NULL
 *     when no estimate exists yet.
 *   codes: out, one per sector: 1 = FP32, 2 + L = FP32 with FP64 islands at level L, 0 = FP64.
 *   counts: out (may be NULL): [0] sectors in FP64, [1] sectors with islands.
 * Options per sector: FP32 (every bin in FP32), islands at level L (bins 0..L in FP32; the points of the other
 * bins cost FP64) and FP64.  Per option and slot the FP32 bins give mean |e|, |mean e| and sum |e|^2 / n^2
 * (e = v32 - v64, n = n_sample); cost = the sector's flop per point with FP64 evaluations counted 30 times.  The
 * FP32 error budget is (fp32_budget > 0 ? fp32_budget : 0.1) * rel_tol.  Per order k the chosen options'
 * statistics add up over the sectors whose slot falls in that order, and the order's FP32 bias bound
 * min(sum mean |e|, sum |mean e| + 3 sqrt(sum |e|^2 / n^2)) -- each sector's signed mean (no cancellation
 * between sectors) with three standard errors, capped by the mean |e| -- may not exceed budget * |T_k|
 * (floor 1e-6 max_k |T_k|).  Every sector starts at its cheapest option; while an order is over its limit, the
 * change of one sector's option with the largest reduction of the excess per extra cost is taken; what no single
 * change can fix goes to FP64.  Without an estimate, each sector takes its cheapest option whose own bound is
 * within budget times its own mean |v64| in every slot.  An option with a non-finite FP32 error is never taken;
 * sectors with endpoint exponents alpha <= -2 always take FP64.
 * Errors: QMC_ERR_ARG for a NULL required pointer, n_sample < 1, negative rel_tol/fp32_budget, or sums without
 * n_sector / n_shifts >= 1 / positive sizes.
 */
int qmc_choose_precision(const void *packed_host, int32_t n_shifts, const int64_t *n_sector, const double *sums,
                         const double *probe, const double *bins, int64_t n_sample, double rel_tol,
                         double fp32_budget, int32_t *codes, int32_t *counts);

/*
 * Generated evaluators (the paper evaluates a fixed, hand-written integrand per sector; this is the
 * library's way of getting the same straight-line arithmetic for any table).  A family = the sector tables
 * with identical exponent structure (same topology and kinematic class, any kinematic point).
 * precision: QMC_PREC_MIXED for the FP32 evaluator (coefficients as hi + lo float pairs), QMC_PREC_FP64 for
 *   the FP64 one (one FMA per term on the FP64 coefficients).
 * qmc_gen_source: writes the CUDA source generated for the family of `packed_host` (an image from qmc_prepare)
 *   into buf (cap bytes, NUL-terminated); *len receives the size needed (call with buf = NULL to query).
 *   Host only.  Errors: QMC_ERR_ARG, QMC_ERR_MEMORY (cap too small).
 * qmc_gen_compile: compiles that source with NVRTC for sm_103a.  load = 0: compile only (no CUDA device needed;
 *   nothing cached).  load = 1: compile unless the family is cached (waiting for a compilation of the same
 *   family already under way), load the module and keep it for the life of the process (the FP32 passes of
 *   QMC_EVAL_GENERATED do this on first use; call it beforehand to keep compilation out of a timed region).
 *   load = 2: the same in a background thread (current device): returns QMC_PENDING while it runs, QMC_OK once
 *   the module is loaded (the serving loop uses this so that other requests keep running meanwhile).
 *   info (may be NULL) receives the family key, compilation time (of the cached compilation when cached = 1),
 *   source and cubin sizes; cached = 1: the module was already loaded in this process, 2: its cubin came from
 *   the disk cache.  A failed compilation is remembered: later calls return its status.
 *   Disk cache (optional): with the environment variable QMC_GEN_CACHE_DIR naming a writable directory, cubins
 *   are stored there and reused by later processes (file name: family, precision, generator version, embedded
 *   device sources and NVRTC version; written atomically).
 *   Errors: QMC_ERR_ARG, QMC_ERR_CODEGEN (NVRTC failed; its log goes to stderr), QMC_ERR_CUDA (load failed).
 */
typedef struct {
    uint64_t family;
    double compile_ms;
    int64_t source_bytes, cubin_bytes;
    int32_t cached;  /* 0: compiled now, 1: loaded earlier in this process, 2: read from the disk cache */
    int32_t reserved;
} qmc_gen_info;

int qmc_gen_source(const void *packed_host, int32_t precision, char *buf, size_t cap, size_t *len);
int qmc_gen_compile(const void *packed_host, int32_t precision, int32_t load, qmc_gen_info *info);

/*
 * Launch-shape autotuner (the paper fixes no launch shape; this is the library's).  qmc_autotune runs the
 * evaluation launch of `pass` (qmc_eval_partials semantics, synchronous on `stream`) once per candidate shape,
 * block in {64, 128, 256} threads (those the pass allows) x points_per_thread in {4, 8, 16, 32}, times each
 * with CUDA events (one untimed launch first), returns the timings and the fastest shape in *out, and records
 * that shape for the family of the image, the pass's precision and evaluator and the lattice-size bucket
 * (smallest 2^k >= n).
 * From then on, in this process, passes of that key whose block and points_per_thread are both 0 use the
 * recorded shape: qmc_scratch_bytes, qmc_eval_sums, qmc_integrate and the serving loop included.  Results
 * depend on the shape only through the summation order.  pass->block/points_per_thread are ignored.
 * scratch: at least qmc_autotune_scratch_bytes(packed_host, pass) bytes (the largest candidate's need).
 * qmc_autotune_clear forgets every recorded shape.
 * Errors: QMC_ERR_ARG, QMC_ERR_MEMORY (scratch too small), QMC_ERR_CUDA, and those of qmc_eval_partials.
 */
typedef struct {
    int32_t block, points_per_thread;  /* the fastest candidate */
    float ms;                          /* its evaluation-launch time */
    int32_t n_candidates;
    int32_t candidate_block[16], candidate_points_per_thread[16];
    float candidate_ms[16];
} qmc_tune_result;

size_t qmc_autotune_scratch_bytes(const void *packed_host, const qmc_pass *pass);
int qmc_autotune(const void *packed_host, const void *packed_dev, const qmc_pass *pass, const double *shifts_dev,
                 const double *lambda_dev, void *scratch_dev, size_t scratch_bytes, qmc_tune_result *out,
                 void *stream);
int qmc_autotune_clear(void);

/*
 * qmc_eval_sums_noalloc -- qmc_eval_sums without a caller-provided scratch buffer, for callers that cannot
 * allocate device memory (e.g. an application whose own pool allocator holds all device memory, or a
 * latency-critical loop that forbids allocation after start-up).  The paper has no counterpart: this is a
 * deployment convenience.  Same inputs, outputs and results as qmc_eval_sums; the scratch is a fixed 32 MiB
 * array inside the library that every GPU loading the library holds until exit.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with the device current), so make it before any
 * stream capture.  The address is kept per device ordinal for the primary context: it does not survive
 * cudaDeviceReset or a switch to another context on that device.  Calls share the array: calls that overlap on
 * the GPU race; calls in one stream are ordered.
 * Allocates nothing (no cudaMalloc/cudaFree).  Code is loaded on first use, though: with the default evaluator
 * (QMC_EVAL_AUTO = generated) the first pass of a family of sector tables in a process compiles that family's
 * evaluator with NVRTC and loads the module onto the device, which needs device memory.  Callers that cannot
 * allow this during their allocation-free phase warm up at start-up (qmc_gen_compile with load = 1 for each
 * precision the passes use, or one call of this function) or set pass->evaluator = QMC_EVAL_TABLE.
 * Returns QMC_ERR_MEMORY, without touching sums or fails, when the pass needs more scratch than 32 MiB
 * (qmc_scratch_bytes() > 33554432), QMC_ERR_ARG for invalid passes.
 */
int qmc_eval_sums_noalloc(const void *packed_host, const void *packed_dev, const qmc_pass *pass,
                          const double *shifts_dev, const double *lambda_dev, double *sums_dev, int64_t *fails_dev,
                          void *stream);

/*
 * qmc_eval_points -- per-point values of one sector (for sampled checks), asynchronous on `stream`.
 * For each j < npts: out[j * n_slots + n] = w(x) I_s(t(x)) coefficient n at x = {idx[j] z / n + Delta},
 * Delta = shift_dev[0..5], computed by the same device code as qmc_eval_sums.  idx_dev: npts int64 lattice
 * indices in [0, lattice.n).  out_dev: npts x n_slots (re, im) pairs.  fails_dev: npts int32 flags.
 */
int qmc_eval_points(const void *packed_host, const void *packed_dev, int32_t sector, const qmc_pass *pass,
                    const double *shift_dev, double lambda, const int64_t *idx_dev, int64_t npts, double *out_dev,
                    int32_t *fails_dev, void *stream);

/* Built-in lattice ladder (largest prime below 2^k, k = 10..26, fast-CBC vectors).  Copies up to `cap`
 * entries into `out` and returns how many exist. */
int qmc_builtin_lattices(qmc_lattice *out, int32_t cap);

/* Combine per-shift sector sums of one pass into the Laurent coefficients of the integral (Sec. III,
 * Eqs. 16-20; host only).  sums: as written by qmc_eval_sums (host copy).  Q: n_shifts x n_orders (re, im)
 * per-shift estimates, n_orders = order_max - order_min + 1 of the image; mean/err: n_orders (re, im) each;
 * err holds the standard errors of the real and imaginary parts. */
int qmc_combine(const void *packed_host, const qmc_pass *pass, const double *sums, double *Q, double *mean,
                double *err);

/* qmc_combine for sums whose sectors come from lattices of different sizes (passes with sector_active):
 * n_sector[s] = lattice size that produced sector s's sums (table order).  Each sector's estimate of Eq. 19 is
 * still unbiased per shift, so the per-shift totals and Eq. 20 keep their meaning.  Host only. */
int qmc_combine_sectors(const void *packed_host, int32_t n_shifts, const int64_t *n_sector, const double *sums,
                        double *Q, double *mean, double *err);

/* ------------------------------------------------------------------ integrate to a requested accuracy */

typedef struct qmc_ctx qmc_ctx;

typedef struct {
    double rel_tol;          /* stop when every order meets err <= rel_tol * max(|value|, 1e-6 * max |value|) */
    double abs_tol;          /* ... or err <= abs_tol */
    int32_t precision;       /* QMC_PREC_FP64 / QMC_PREC_MIXED */
    int32_t n_shifts;        /* m (default 16) */
    uint64_t seed;           /* shifts: splitmix64 from this state, 6 draws per shift */
    double lambda;           /* initial deformation parameter (Eq. 14); halved per failing sector */
    int32_t max_halvings;    /* cap on lambda halvings per sector (default 6) */
    int32_t transform_r;     /* default 3 */
    int32_t ladder_start;    /* index into the built-in ladder where the loop starts (0 = 2^10) */
    int32_t n_lattices;      /* > 0: use `lattices` instead of the built-in ladder */
    const qmc_lattice *lattices;
    const double *shifts;    /* optional n_shifts x 6 host array overriding the seed */
    int64_t max_n;           /* stop the ladder above this lattice size (0 = no limit) */
    double max_seconds;      /* 0 = no limit; else the time limit (QMC_ERR_TIMEOUT), which also stops a running
                                pass: the kernels skip its remaining work items once a timer sets an abort flag */
    int32_t block, points_per_thread; /* launch shape (0 = default) */
    int64_t probe_samples;   /* QMC_PREC_MIXED: points per sector of the FP32/FP64 probe (0 = 4096) */
    double fp32_budget;      /* QMC_PREC_MIXED (0 = 0.1): the FP32 error budget is fp32_budget * rel_tol of the
                                integral.  Per eps order, the probe's mean |v32 - v64| per point of the sectors kept
                                in FP32 may add up to that fraction of the current estimate of the order (summed
                                over sectors, before the Gamma prefactor); sectors take the budget in order of their
                                share of it and the rest run in FP64.  Before any estimate exists (the probe precedes
                                the first FP32 pass), a sector runs in FP64 when its sum|v32-v64| exceeds
                                fp32_budget * rel_tol * sum|v64| in any order; after the first evaluation the
                                decision is taken again on the same probe with the estimates. */
    int32_t evaluator;       /* QMC_EVAL_* of the FP32 evaluation (passes and probe) */
    int32_t lock_step;       /* 0 (default): each sector has its own lattice size, and after each step only the
                                sectors that carry most of the remaining error per unit of cost move up the ladder
                                (the per-shift totals stay valid estimates, qmc_combine_sectors); nonzero: all
                                sectors climb the ladder together */
} qmc_options;

typedef struct {
    int32_t status;
    int32_t order_min, n_orders;
    double value[QMC_MAX_ORDERS][2];  /* Laurent coefficients (re, im), order_min + k */
    double error[QMC_MAX_ORDERS][2];  /* standard errors of re and im (Eq. 20) */
    int64_t n_final;                  /* largest lattice size any sector reached */
    int64_t evals;                    /* sector x shift x point evaluations, all passes */
    double seconds;                   /* wall time of qmc_integrate */
    double kernel_ms;                 /* device time of the evaluation kernels, all passes */
    int32_t passes, lambda_halvings, fp64_reruns, sign_failures;
    double queued_seconds;            /* serving: time between qmc_submit and admission */
    int32_t island_sectors;           /* mixed: sectors in FP32 with FP64 islands (fp64_reruns: sectors in FP64) */
    int32_t nonfinite_sectors;        /* sectors whose sums came out NaN or infinite: a mixed integration runs them
                                         again in FP64 (counted in fp64_reruns too); in FP64 the integration stops
                                         with QMC_ERR_NONFINITE */
} qmc_result;

typedef struct {
    int64_t submitted, completed, queued, active, peak_active;
    int64_t rounds;                   /* batched rounds run by the scheduler */
    int64_t batched_passes;           /* passes run, summed over rounds */
    int64_t device_bytes;             /* device memory held by the context */
    int64_t shed;                     /* requests turned away before running: their deadline could not be met */
} qmc_serving_stats;

/* Context: owns a CUDA stream binding, the device copies of loaded integrals and its scratch.
 * device: CUDA ordinal; mem_budget: bytes of device memory the context may hold (0 = 1 GiB);
 * stream: cudaStream_t to launch on (NULL = the legacy default stream). */
int qmc_create(qmc_ctx **out, int32_t device, size_t mem_budget, void *stream);
int qmc_destroy(qmc_ctx *ctx);

/* Copies a sector table into the context; returns its id. */
int qmc_load_sectors(qmc_ctx *ctx, const void *table, size_t table_bytes, int32_t *integral_id);

/* Evaluates the table at a kinematic point for Laurent orders order_min..order_max and uploads the packed
 * image (qmc_prepare semantics). */
int qmc_set_kinematics(qmc_ctx *ctx, int32_t integral_id, const double *invariants, int32_t n_invariants,
                       int32_t order_min, int32_t order_max);

/* One pass with host buffers (blocking): copies the packed image, shifts and per-sector lambda from host memory to
 * context-owned device buffers, runs qmc_eval_sums on the context's stream and copies sums and fails back to the
 * host (layouts as in qmc_eval_sums).  Pinned host memory makes the copies asynchronous DMA. */
int qmc_eval_sums_host(qmc_ctx *ctx, const void *packed_host, const qmc_pass *pass, const double *shifts_host,
                       const double *lambda_host, double *sums_host, int64_t *fails_host);

/* Blocking: integrates to the requested accuracy (Sec. III: shifted rank-1 lattice rules of growing size, Eqs.
 * 19-20 for the value and its error).  Each step evaluates the sectors that need it (all shifts): lambda of
 * sectors failing the sign check of Eq. (14) is halved and they are re-run; otherwise, unless opt->lock_step,
 * only the sectors holding most of the remaining variance per unit of cost move to the next lattice size
 * (per-sector lattices; the paper lets all sectors climb together, as lock_step does).  Mixed precision runs a
 * step in FP32 only where its FP64 cost would exceed ~1e8 flop, after the FP32/FP64 probe of
 * qmc_probe_precision.  Stops when every order meets the tolerance, or at max_n, max_seconds or the end of the
 * ladder.  Returns the status also stored in out->status. */
int qmc_integrate(qmc_ctx *ctx, int32_t integral_id, const qmc_options *opt, qmc_result *out);

/* ------------------------------------------------------------------ serving (continuous batching) */
/* Queue an integration request: the integral `integral_id` (loaded with qmc_load_sectors) at the kinematic point
 * `invariants`, Laurent orders order_min..order_max, options as for qmc_integrate.  A scheduler thread of the
 * context admits requests while its device-memory budget has room and runs batched rounds: each active request
 * contributes the pass at its current lattice size to shared launches (qmc_eval_batch); requests that arrive
 * meanwhile join at the next round.  A request's result is the same, bit for bit, as qmc_integrate with the same
 * options would give alone.  opt->max_seconds counts from submission: a request whose limit passes while it
 * is still queued finishes with QMC_ERR_TIMEOUT without running, and so does one that cannot finish in time by
 * the loop's estimate (counted in qmc_serving_stats.shed).  The estimate: each round's measured time is charged
 * to its requests by their share of its evaluations; a completed request's charge, averaged per integral, is the
 * cost of the next one; the work ahead of a queued request is the remaining cost of the running ones (requests
 * running together share every round, so one ends no earlier than their summed cost); all taken with a margin of
 * 1.25.  A queued request also waits while admitting it would, by the same estimate, end a running request past
 * its limit.  The paper
 * has no serving loop; this is the library's deployment layer. */
int qmc_submit(qmc_ctx *ctx, int32_t integral_id, const double *invariants, int32_t n_invariants, int32_t order_min,
               int32_t order_max, const qmc_options *opt, int64_t *request_id);

/* QMC_PENDING while the request is queued or running; otherwise fills `out` and returns its final status.
 * out->seconds is the time from submission to completion, out->queued_seconds the wait before admission. */
int qmc_poll(qmc_ctx *ctx, int64_t request_id, qmc_result *out);

/* Marks a request cancelled; it leaves at the next round boundary with status QMC_ERR_CANCELLED. */
int qmc_cancel(qmc_ctx *ctx, int64_t request_id);

/* Counters of the serving loop. */
int qmc_serving_stats_get(qmc_ctx *ctx, qmc_serving_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* QMCFI_H */
