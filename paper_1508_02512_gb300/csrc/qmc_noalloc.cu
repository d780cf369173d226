/*
 * qmc_eval_sums_noalloc: the evaluation pass of qmc_eval_sums for callers that cannot allocate device memory.
 *
 * Some callers cannot call cudaMalloc: a host application that has reserved all device memory for its own pool
 * allocator (a further cudaMalloc fails or fragments that pool), or a latency-critical loop whose deployment
 * forbids device allocation after start-up.  qmc_eval_sums asks the caller for a scratch buffer; this variant
 * needs none.  Its scratch (per-item partial sums, sign-failure counts and work counters) lives in the
 * file-scope array below, which every GPU that loads this library holds until the process exits.
 *
 * The array's name is, in host code, a host-side stand-in, not a device address: its device address is taken
 * once per device with cudaGetSymbolAddress (with that device current) on the first call made on that device,
 * so that first call should come before any stream capture.  The address is cached per device ordinal and
 * belongs to the context that was current then (the runtime's primary context): it goes stale after
 * cudaDeviceReset, or when the caller makes another context current on that device, so only the primary
 * context is supported and the library must not outlive a reset of its device.  All calls share the array, so two calls whose
 * work overlaps on the GPU (different streams, or different host threads) race on it; calls in one stream
 * are serialised by the stream.  The work counters are cleared by every call; partials are overwritten.
 */
#include <cuda_runtime.h>

#include <mutex>

#include "qmc_internal.h"

#define QMC_NOALLOC_SCRATCH_BYTES (32u << 20) /* 32 MiB */
#define QMC_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char qmc_noalloc_scratch[QMC_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
void *g_addr[QMC_NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" int qmc_eval_sums_noalloc(const void *packed_host, const void *packed_dev, const qmc_pass *pass,
                                     const double *shifts_dev, const double *lambda_dev, double *sums_dev,
                                     int64_t *fails_dev, void *stream) {
    const size_t need = qmc_scratch_bytes(packed_host, pass);
    if (need == 0) return QMC_ERR_ARG;
    if (need > QMC_NOALLOC_SCRATCH_BYTES) return QMC_ERR_MEMORY; /* pass too large for the fixed scratch */
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_NO_DEVICE;
    if (dev < 0 || dev >= QMC_NOALLOC_MAX_DEVICES) return QMC_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, qmc_noalloc_scratch) != cudaSuccess || !p) return QMC_ERR_CUDA;
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    return qmc_eval_sums(packed_host, packed_dev, pass, shifts_dev, lambda_dev, scratch, QMC_NOALLOC_SCRATCH_BYTES,
                         sums_dev, fails_dev, stream);
}
