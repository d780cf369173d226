/*
 * Packed device image of a prepared integral, shared by the host runtime (qmc_prepare.cpp, qmc_pass.cpp, qmc_context.cpp) and the kernels
 * (qmc_kernels.cu).  One contiguous, relocatable buffer (offsets only):
 *
 *   PackedHeader                      kinematics-independent data, prefactor series, launch classes
 *   PackedSector[n_sectors]           sectors sorted by class (undeformed first, then deformed)
 *   PackedTerm[n_terms_total]         per sector: Ut terms, Ft terms, dFt/dt_j terms (j = 0..dim-1),
 *                                     d2Ft/dt_j dt_k terms (j <= k, row-major upper triangle)
 *
 *   PackedTermF[n_terms_total]        the same terms for the FP32 path: the coefficient as a float pair
 *                                     hi + lo (hi = fl32(c), lo = fl32(c - hi)) and the same exponents
 *
 * A term is one monomial c * prod_j t_j^{e_j}: 8 bytes of coefficient (already evaluated at the kinematic
 * point) and 8 exponent bytes, 16 bytes in all, so that a block stages a sector into shared memory with
 * 16-byte vector copies and every thread of a warp reads the same term (a shared-memory broadcast).
 */
#pragma once
#include <stdint.h>

#include "../../include/qmcfi.h"

#define QMC_PACK_MAGIC 0x31504d51u /* "QMP1" */
#define QMC_MAX_EXP 15             /* largest exponent of one variable in one term */
#define QMC_MAX_SECTOR_TERMS 3072  /* terms staged per sector (48 KiB of shared memory) */
#define QMC_N_CLASSES 3            /* 0: undeformed sectors, 1: deformed sectors, 2: undeformed sectors with an
                                      endpoint exponent alpha <= -2 (Taylor subtraction of Eq. 11 with p > 0) */
/* Sectors of class 2: every variable with alpha_j <= -1 is expanded at t_j = 0 to order p_j = -alpha_j - 1 */
#define QMC_TAYLOR_MAX_P 2         /* alpha_j >= -3 */
#define QMC_TAYLOR_MAX_Z 2         /* variables with alpha_j <= -1 in such a sector */
#define QMC_TAYLOR_EXTRA 10        /* Taylor terms of a remainder taken from its own series */
#define QMC_TAYLOR_SMALL_T 0.02    /* below it a variable's remainder comes from that series */
#define QMC_TAYLOR_Q (QMC_TAYLOR_MAX_P + QMC_TAYLOR_EXTRA + 1) /* orders per expanded variable */

struct PackedHeader {
    uint32_t magic;
    int32_t n_sectors;
    int32_t dim, loops, n_nu, n_props;
    int32_t eU0, eU1, eF0, eF1;           /* U^{eU0 + eU1 eps} / F^{eF0 + eF1 eps} */
    int32_t order_min, order_max, kmax, n_slots;
    int32_t pre_low, n_pre;
    double pre[QMC_MAX_ORDERS + 4];
    int32_t class_begin[QMC_N_CLASSES], class_end[QMC_N_CLASSES], class_maxm[QMC_N_CLASSES];
    int32_t max_terms, n_terms_total;
    int64_t sectors_off, terms_off, total_bytes;
    double flops_per_eval, transc_per_eval;
    int32_t n_deformed, n_negative, max_sigma, reserved;
    int64_t termsf_off;
    uint64_t family;                      /* hash of everything the generated evaluators depend on (exponents) */
    int64_t reserved2;
};

struct PackedSector {
    int32_t kind;       /* 0: F > 0, 1: F < 0 (kernel uses |F|), 2: deformed */
    int32_t sigma;      /* number of singular variables (A_j == -1) */
    int32_t sing_mask;  /* bit j set when A_j == -1 */
    int32_t M;          /* series computed to eps^M before the 1/eps pole factors; slots 0..M */
    int32_t A[8], B[8];
    int32_t nU, nF, nG, nH;
    int32_t term0;      /* index of the sector's first term in the term array */
    int32_t n_terms;    /* nU + nF + nG + nH */
    int32_t orig_index; /* position of the sector in the table (outputs are indexed by it) */
    int32_t taylor;     /* 1: some alpha_j <= -2 (class 2) */
    int16_t gstart[8];  /* gradient polynomial j: terms [gstart[j], gstart[j+1]) of the G block */
    int16_t hstart[24]; /* Hessian polynomial p (j <= k): terms [hstart[p], hstart[p+1]) of the H block */
    double D;
    double flops, transc;
    float Df;           /* D rounded to FP32 (the FP32 path must not convert FP64 values per point) */
    float pad;
};

struct PackedTerm {
    double c;
    uint8_t e[8];
};

struct PackedTermF {
    float hi, lo;
    uint8_t e[8];
};

static_assert(sizeof(PackedTerm) == 16, "term must be 16 bytes");
static_assert(sizeof(PackedTermF) == 16, "FP32 term must be 16 bytes");
static_assert(sizeof(PackedSector) % 16 == 0, "sector record must be 16-byte aligned");
static_assert(sizeof(PackedHeader) % 16 == 0, "header must be 16-byte aligned");

/* One evaluation job: one pass of one prepared integral over one sector class (a contiguous range of its packed
   sectors), every shift and every lattice point.  An evaluation launch covers a table of jobs that share the
   kernel instantiation (sector dimension, deformation, series length, precision): a single integral's pass, or
   the passes of many requests at once (continuous batching).  Items of a job are numbered (sector, shift, chunk),
   chunk = blockDim * P consecutive lattice indices; item_begin places them in the launch's item space. */
struct Job {
    const unsigned char *packed;  /* device image */
    int64_t sectors_off, terms_off, termsf_off;
    int64_t chunks;               /* chunks per (sector, shift) */
    int64_t item_begin;           /* first item of this job in the launch */
    const double *shifts;         /* m x 6 */
    const double *lambda;         /* per sector, table order */
    const int32_t *sector_prec;   /* mixed passes: per sector (table order), 1 = FP32; null = all of want_prec */
    double *partials;             /* this job's items x n_slots x 2 */
    uint32_t *part_fails;         /* this job's items */
    double invn;
    uint32_t n;                   /* lattice size */
    uint32_t z[QMC_MAX_DIM];
    uint32_t zstep[QMC_MAX_DIM];  /* (blockDim * z_j) mod n */
    int32_t sector_begin, n_sect, m, n_slots;
    int32_t eU0, eU1, eF0, eF1;
    const volatile int32_t *abort; /* null, or nonzero once the pass is stopped: its remaining items are skipped */
};

#define QMC_MAX_JOBS 96

/* Kernel parameter block of an evaluation launch (read from the constant bank). */
struct JobTable {
    int32_t n_jobs, r, P, want_prec;
    int64_t total_items;
    unsigned long long *counter;  /* work counter of this launch (zeroed before it) */
    int32_t smem_bytes, pad;
    Job jobs[QMC_MAX_JOBS];
};

/* Reduction of one job's partials into its per-(sector, shift) sums. */
struct FinJob {
    const unsigned char *packed;
    int64_t sectors_off, chunks, pair_begin;
    const double *partials;
    const uint32_t *part_fails;
    double *sums;                 /* n_sectors(table order) x m x n_slots x 2 */
    int64_t *fails;               /* n_sectors x m */
    int32_t sector_begin, n_sect, m, n_slots;
};

struct FinTable {
    int32_t n_jobs, pad;
    int64_t total_pairs;
    FinJob jobs[QMC_MAX_JOBS];
};

static_assert(sizeof(JobTable) < 32000, "job table must fit the kernel parameter limit");
static_assert(sizeof(FinTable) < 32000, "finalize table must fit the kernel parameter limit");

/* blocks per sector of the precision probe (a thread-block cluster; portable size) */
#define QMC_PROBE_CLUSTER 8

/* Precision probe: a strided sample of each sector's lattice points for one shift, in FP32 and FP64. */
struct ProbeArgs {
    const unsigned char *packed;
    int64_t sectors_off, terms_off, termsf_off;
    int32_t sector_begin, n_sect;
    int32_t r, n_slots;
    uint32_t n;
    uint32_t z[QMC_MAX_DIM];
    double invn;
    const double *shift;          /* 6 doubles */
    const double *lambda;         /* per sector, table order */
    int64_t n_sample;             /* sample points per sector */
    double *out;                  /* n_sectors(table order) x n_slots x 4: sum|v64|, sum|v32-v64|, sum(v32-v64) re, im */
    double *bins;                 /* null, or n_sectors(table order) x QMC_ISLAND_BINS x (1 + 4 n_slots): per island
                                     bin, the points in it and per slot, over them, sum |e|, sum e (re, im) and
                                     sum |e|^2, e = v32 - v64 */
    int32_t eU0, eU1, eF0, eF1;
    int32_t smem_bytes;
};

struct PointArgs {
    const unsigned char *packed;
    int64_t sectors_off, terms_off;
    int32_t sector;               /* packed index */
    int32_t r, n_slots;
    uint32_t n;
    uint32_t z[QMC_MAX_DIM];
    double invn;
    const double *shift;
    double lambda;
    const int64_t *idx;
    int64_t npts;
    double *out;
    int32_t *fails;
    int32_t eU0, eU1, eF0, eF1;
    int32_t smem_bytes;
};

/* Launchers implemented in qmc_kernels.cu (C++ linkage, internal). */
int qmc_launch_eval(int dim, int deform, int maxm, int precision, const JobTable &t, int grid, int block,
                    void *stream);
int qmc_launch_finalize(const FinTable &t, void *stream);
int qmc_launch_points(int dim, int deform, int maxm, int precision, const PointArgs &a, void *stream);
int qmc_device_sm_count(int *sms);
int qmc_eval_blocks_per_sm(int dim, int deform, int maxm, int precision, int block, int smem_bytes, int *out);
int qmc_launch_probe(int dim, int deform, int maxm, const ProbeArgs &a, void *stream);

/* Generated evaluators (qmc_jit.cpp): the evaluation kernel (QMC_PREC_FP64 or _MIXED = FP32) of a family's
   module for sector class cls
   (compiled and loaded on first use), its occupancy and launch.  Kernel handles are cudaKernel_t values passed
   as const void *. */
int qmc_gen_kernel(const void *packed_host, int precision, int cls, const void **eval_kernel);
uint64_t qmc_family_key(const void *packed_host); /* computed from the image, not read from its header */
int qmc_gen_max_block(int dim);                  /* largest block of a generated kernel for sectors of this dimension */
int qmc_gen_blocks_per_sm(const void *kernel, int block, int smem_bytes, int *out);
int qmc_gen_launch_eval(const void *kernel, const JobTable &t, int grid, int block, void *stream);
