/*
 * Declarations shared by the host translation units of the qmcfi library (qmc_prepare.cpp, qmc_pass.cpp,
 * qmc_context.cpp): access to a packed image and helpers with one definition.
 */
#pragma once
#include <cuda_runtime.h>

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

namespace qmci {
/* QMC_OK when the blob is a well-formed sector table, else the status qmc_prepare would return */
int validate_table(const void *blob, size_t bytes);

/* Eqs. 19-20 with the Gamma prefactor: per-shift totals Q, their mean and standard errors.  invn_of[s] = 1/n of
   the lattice that produced sector s's sums (table order); only >= 0 restricts the totals to that sector. */
int combine_core(const void *packed_host, int m, const double *invn_of, int only, const double *sums, double *Q,
                 double *mean, double *err);
}  // namespace qmci
