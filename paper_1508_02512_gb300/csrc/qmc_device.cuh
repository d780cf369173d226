#pragma once
/* Host launchers of the ahead-of-time kernels (one instantiation per sector dimension, deformation and series
 * length); the device code is in qmc_dev.cuh. */
#include <cuda_runtime.h>

#include "qmc_dev.cuh"

/* ------------------------------------------------------------------ dispatch */
template <int S, bool DEF, int MAXM>
static int launch_eval_t(const JobTable &t, int grid, int block, cudaStream_t st) {
    auto k = qmc_eval_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    k<<<grid, block, t.smem_bytes, st>>>(t);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int occupancy_t(int block, int smem, int *out) {
    auto k = qmc_eval_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return QMC_ERR_CUDA;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, block, smem) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int launch_eval_f32_t(const JobTable &t, int grid, int block, cudaStream_t st) {
    auto k = qmc_eval_kernel_f32<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    k<<<grid, block, t.smem_bytes, st>>>(t);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int occupancy_f32_t(int block, int smem, int *out) {
    auto k = qmc_eval_kernel_f32<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return QMC_ERR_CUDA;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, block, smem) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int launch_probe_t(const ProbeArgs &a, cudaStream_t st) {
    auto k = qmc_probe_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    if (a.n_sect < 1) return QMC_OK;
    /* one cluster of QMC_PROBE_CLUSTER blocks per sector where the device can place such clusters with this
       shared memory; otherwise one block per sector (the kernel reads its cluster shape) */
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = QMC_PROBE_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)a.n_sect * QMC_PROBE_CLUSTER);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = (size_t)a.smem_bytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        clusters = 0;
    }
    if (clusters < 1) {
        cfg.gridDim = dim3((unsigned)a.n_sect);
        cfg.numAttrs = 0;
    }
    return cudaLaunchKernelEx(&cfg, k, a) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, bool DEF, int MAXM>
static int launch_points_t(const PointArgs &a, cudaStream_t st) {
    auto k = qmc_points_kernel<S, DEF, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    const int block = 128;
    long long g = (a.npts + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    k<<<(int)g, block, a.smem_bytes, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

/* class 2 (endpoint exponents alpha <= -2): FP64 only */
template <int S, int MAXM>
static int launch_eval_taylor_t(const JobTable &t, int grid, int block, cudaStream_t st) {
    auto k = qmc_eval_kernel_taylor<S, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    k<<<grid, block, t.smem_bytes, st>>>(t);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, int MAXM>
static int occupancy_taylor_t(int block, int smem, int *out) {
    auto k = qmc_eval_kernel_taylor<S, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return QMC_ERR_CUDA;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, block, smem) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int S, int MAXM>
static int launch_points_taylor_t(const PointArgs &a, cudaStream_t st) {
    auto k = qmc_points_kernel_taylor<S, MAXM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes) != cudaSuccess)
        return QMC_ERR_CUDA;
    const int block = 128;
    long long g = (a.npts + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    k<<<(int)g, block, a.smem_bytes, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}
