/*
 * Dispatch of the evaluation kernels by sector dimension, and the deterministic reduction kernel.
 * The templates live in qmc_device.cuh; each qmc_kern_d<N>.cu instantiates one sector dimension.
 */
#include "qmc_device.cuh"

int qmc_launch_eval_d1(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d1(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d1(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d1(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d2(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d2(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d2(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d2(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d3(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d3(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d3(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d3(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d4(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d4(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d4(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d4(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d5(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d5(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d5(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d5(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d6(int deform, int maxm, int precision, const EvalArgs &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d6(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d6(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d6(int deform, int maxm, const PointArgs &a, cudaStream_t st);

int qmc_launch_eval_param_d1(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d1(int deform, int maxm, int block, int *out);
int qmc_launch_eval_param_d2(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d2(int deform, int maxm, int block, int *out);
int qmc_launch_eval_param_d3(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d3(int deform, int maxm, int block, int *out);
int qmc_launch_eval_param_d4(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d4(int deform, int maxm, int block, int *out);
int qmc_launch_eval_param_d5(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d5(int deform, int maxm, int block, int *out);
int qmc_launch_eval_param_d6(int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                              cudaStream_t st);
int qmc_occupancy_param_d6(int deform, int maxm, int block, int *out);

/* ------------------------------------------------------------------ K4: deterministic per-(sector, shift) sums */
__global__ void __launch_bounds__(128) qmc_finalize_kernel(FinalizeArgs a) {
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long pairs = (long long)a.n_sect * a.m;
    if (wg >= pairs) return;
    const int ls = (int)(wg / a.m), shift = (int)(wg % a.m);
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(a.packed + a.sectors_off) + a.sector_begin + ls;
    const int orig = ps->orig_index;
    const long long base = wg * a.chunks;
    double s[2 * QMC_MAX_SLOTS], c[2 * QMC_MAX_SLOTS];
#pragma unroll
    for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q) s[q] = c[q] = 0.0;
    unsigned long long f = 0;
    for (long long k = lane; k < a.chunks; k += 32) {
        const double *p = a.partials + (base + k) * a.n_slots * 2;
#pragma unroll
        for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q)
            if (q < 2 * a.n_slots) kahan_add(s[q], c[q], p[q]);
        f += a.part_fails[base + k];
    }
#pragma unroll
    for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q) {
        double v = s[q] - c[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0 && q < 2 * a.n_slots) a.sums[((long long)orig * a.m + shift) * a.n_slots * 2 + q] = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
    if (lane == 0) a.fails[(long long)orig * a.m + shift] = (int64_t)f;
}

int qmc_launch_eval(int dim, int deform, int maxm, int precision, const EvalArgs &a, int grid, int block,
                    void *stream) {
    if (precision != QMC_PREC_FP64 && precision != QMC_PREC_MIXED) return QMC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    switch (dim) {
        case 1: return qmc_launch_eval_d1(deform, maxm, precision, a, grid, block, st);
        case 2: return qmc_launch_eval_d2(deform, maxm, precision, a, grid, block, st);
        case 3: return qmc_launch_eval_d3(deform, maxm, precision, a, grid, block, st);
        case 4: return qmc_launch_eval_d4(deform, maxm, precision, a, grid, block, st);
        case 5: return qmc_launch_eval_d5(deform, maxm, precision, a, grid, block, st);
        case 6: return qmc_launch_eval_d6(deform, maxm, precision, a, grid, block, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_eval_blocks_per_sm(int dim, int deform, int maxm, int precision, int block, int smem_bytes, int *out) {
    if (precision != QMC_PREC_FP64 && precision != QMC_PREC_MIXED) return QMC_ERR_UNSUPPORTED;
    switch (dim) {
        case 1: return qmc_occupancy_d1(deform, maxm, precision, block, smem_bytes, out);
        case 2: return qmc_occupancy_d2(deform, maxm, precision, block, smem_bytes, out);
        case 3: return qmc_occupancy_d3(deform, maxm, precision, block, smem_bytes, out);
        case 4: return qmc_occupancy_d4(deform, maxm, precision, block, smem_bytes, out);
        case 5: return qmc_occupancy_d5(deform, maxm, precision, block, smem_bytes, out);
        case 6: return qmc_occupancy_d6(deform, maxm, precision, block, smem_bytes, out);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_probe(int dim, int deform, int maxm, const ProbeArgs &a, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dim) {
        case 1: return qmc_launch_probe_d1(deform, maxm, a, st);
        case 2: return qmc_launch_probe_d2(deform, maxm, a, st);
        case 3: return qmc_launch_probe_d3(deform, maxm, a, st);
        case 4: return qmc_launch_probe_d4(deform, maxm, a, st);
        case 5: return qmc_launch_probe_d5(deform, maxm, a, st);
        case 6: return qmc_launch_probe_d6(deform, maxm, a, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_points(int dim, int deform, int maxm, int precision, const PointArgs &a, void *stream) {
    if (precision != QMC_PREC_FP64) return QMC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    switch (dim) {
        case 1: return qmc_launch_points_d1(deform, maxm, a, st);
        case 2: return qmc_launch_points_d2(deform, maxm, a, st);
        case 3: return qmc_launch_points_d3(deform, maxm, a, st);
        case 4: return qmc_launch_points_d4(deform, maxm, a, st);
        case 5: return qmc_launch_points_d5(deform, maxm, a, st);
        case 6: return qmc_launch_points_d6(deform, maxm, a, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_eval_param(int dim, int deform, int maxm, const EvalArgs &a, const ParamGroup &g, int grid, int block,
                          void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dim) {
        case 1: return qmc_launch_eval_param_d1(deform, maxm, a, g, grid, block, st);
        case 2: return qmc_launch_eval_param_d2(deform, maxm, a, g, grid, block, st);
        case 3: return qmc_launch_eval_param_d3(deform, maxm, a, g, grid, block, st);
        case 4: return qmc_launch_eval_param_d4(deform, maxm, a, g, grid, block, st);
        case 5: return qmc_launch_eval_param_d5(deform, maxm, a, g, grid, block, st);
        case 6: return qmc_launch_eval_param_d6(deform, maxm, a, g, grid, block, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_eval_param_blocks_per_sm(int dim, int deform, int maxm, int block, int *out) {
    switch (dim) {
        case 1: return qmc_occupancy_param_d1(deform, maxm, block, out);
        case 2: return qmc_occupancy_param_d2(deform, maxm, block, out);
        case 3: return qmc_occupancy_param_d3(deform, maxm, block, out);
        case 4: return qmc_occupancy_param_d4(deform, maxm, block, out);
        case 5: return qmc_occupancy_param_d5(deform, maxm, block, out);
        case 6: return qmc_occupancy_param_d6(deform, maxm, block, out);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_finalize(const FinalizeArgs &a, void *stream) {
    const long long pairs = (long long)a.n_sect * a.m;
    if (pairs == 0) return QMC_OK;
    const int block = 128;
    const long long grid = (pairs * 32 + block - 1) / block;
    qmc_finalize_kernel<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int qmc_device_sm_count(int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_NO_DEVICE;
    return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}
