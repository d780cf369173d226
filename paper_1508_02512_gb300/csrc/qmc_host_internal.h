/*
 * Declarations shared by the host translation units of the qmcfi library (qmc_prepare.cpp, qmc_pass.cpp,
 * qmc_context.cpp): access to a packed image and helpers with one definition.
 */
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "qmc_internal.h"

/* the image's header, or NULL when the buffer does not start with one */
inline const PackedHeader *header_of(const void *packed) {
    const PackedHeader *h = static_cast<const PackedHeader *>(packed);
    return (h && h->magic == QMC_PACK_MAGIC) ? h : nullptr;
}
inline const PackedSector *sectors_of(const void *packed) {
    const PackedHeader *h = header_of(packed);
    return reinterpret_cast<const PackedSector *>(static_cast<const unsigned char *>(packed) + h->sectors_off);
}
inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA; }

/* cost of an FP64 evaluation per algorithmic flop relative to FP32 (the generated kernels' measured rates differ by
   20-33x): for the choice of each sector's precision, and for charging a serving round's time to its requests */
#define QMC_FP64_COST 30.0

namespace qmci {
/* per eps order k of the sector sums (slot - sigma, offset by the largest sigma), summed over sectors before the
   Gamma prefactor; n_sector[s] is the lattice size of sector s's sums (table order) */
void order_totals(const void *packed_host, int m, const int64_t *n_sector, const double *sums, std::vector<double> &Tr,
                  std::vector<double> &Ti);

/* qmc_choose_precision's rule on order totals (empty: no estimate yet); returns whether totals were used */
bool choose_precision(const void *packed_host, const double *probe, const double *bins, int64_t n_sample,
                      const std::vector<double> &Tr, const std::vector<double> &Ti, double budget, int32_t *codes,
                      int32_t *n_fp64, int32_t *n_islands);

/* QMC_OK when the blob is a well-formed sector table, else the status qmc_prepare would return */
int validate_table(const void *blob, size_t bytes);

/* Eqs. 19-20 with the Gamma prefactor: per-shift totals Q, their mean and standard errors.  invn_of[s] = 1/n of
   the lattice that produced sector s's sums (table order); only >= 0 restricts the totals to that sector. */
int combine_core(const void *packed_host, int m, const double *invn_of, int only, const double *sums, double *Q,
                 double *mean, double *err);
}  // namespace qmci
