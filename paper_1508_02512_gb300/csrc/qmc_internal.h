/*
 * Packed device image of a prepared integral, shared by the host runtime (qmc_host.cpp) and the kernels
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
#define QMC_N_CLASSES 2            /* 0: undeformed sectors, 1: deformed sectors */

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
    int32_t reserved;
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

/* Per-launch arguments of the evaluation kernels (passed by value). */
struct EvalArgs {
    const unsigned char *packed;  /* device image */
    int64_t sectors_off, terms_off;
    int32_t sector_begin;         /* first packed sector of the class */
    int32_t n_sect;               /* sectors in the class */
    int32_t m;                    /* shifts */
    int32_t r;                    /* transform order */
    int32_t P;                    /* points per thread */
    int32_t n_slots;              /* partial/sum stride */
    uint32_t n;                   /* lattice size */
    uint32_t z[QMC_MAX_DIM];
    uint32_t zstep[QMC_MAX_DIM];  /* (blockDim * z_j) mod n */
    double invn;
    int64_t chunks;               /* chunks per (sector, shift) */
    int64_t total_items;          /* n_sect * m * chunks */
    const double *shifts;         /* m x 6 */
    const double *lambda;         /* per sector, table order */
    double *partials;             /* total_items x n_slots x 2 */
    uint32_t *part_fails;         /* total_items */
    unsigned long long *counter;  /* work counter (zeroed before launch) */
    int32_t eU0, eU1, eF0, eF1;
    int32_t smem_bytes;
    int64_t termsf_off;
    const int32_t *sector_prec;   /* per sector (table order): 0 FP64, 1 FP32; null = all of want_prec */
    int32_t want_prec;            /* items of sectors with another precision are skipped */
};

/* FP32 kernel with its tables in kernel parameters (constant bank): a group of sectors per launch. */
#define QMC_PARAM_SECTORS 16
#define QMC_PARAM_TERMS 1600
#define QMC_MAX_GROUP_LAUNCHES 1024

struct ParamSector {
    int32_t kind, sigma, sing_mask, M;
    int32_t A[6], B[6];
    int32_t nU, nF, nG, nH;
    int32_t tbase;      /* first term of the sector in ParamGroup::terms */
    int32_t orig_index;
    int32_t psec;       /* packed index */
    float Df;
    int16_t gstart[8];
    int16_t hstart[24];
};

struct ParamGroup {
    int32_t n_sect, n_terms, pad0, pad1;
    ParamSector sec[QMC_PARAM_SECTORS];
    PackedTermF terms[QMC_PARAM_TERMS];
};

static_assert(sizeof(ParamSector) % 16 == 0, "param sector must be 16-byte aligned");

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
    int32_t eU0, eU1, eF0, eF1;
    int32_t smem_bytes;
};

struct FinalizeArgs {
    const unsigned char *packed;
    int64_t sectors_off;
    int32_t sector_begin, n_sect, m, n_slots;
    int64_t chunks;
    const double *partials;
    const uint32_t *part_fails;
    double *sums;                 /* n_sectors(table order) x m x n_slots x 2 */
    int64_t *fails;               /* n_sectors x m */
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
int qmc_launch_eval(int dim, int deform, int maxm, int precision, const EvalArgs &a, int grid, int block,
                    void *stream);
int qmc_launch_finalize(const FinalizeArgs &a, void *stream);
int qmc_launch_points(int dim, int deform, int maxm, int precision, const PointArgs &a, void *stream);
int qmc_device_sm_count(int *sms);
int qmc_eval_blocks_per_sm(int dim, int deform, int maxm, int precision, int block, int smem_bytes, int *out);
int qmc_launch_probe(int dim, int deform, int maxm, const ProbeArgs &a, void *stream);
int qmc_launch_eval_param(int dim, int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                          void *stream);
int qmc_eval_param_blocks_per_sm(int dim, int deform, int maxm, int block, int *out);
