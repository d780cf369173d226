/*
 * Dispatch of the evaluation kernels by sector dimension, and the deterministic reduction kernel.
 * The templates live in qmc_device.cuh; each qmc_kern_d<N>.cu instantiates one sector dimension.
 */
#include "qmc_device.cuh"

int qmc_launch_eval_d1(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d1(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d1(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d1(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d2(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d2(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d2(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d2(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d3(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d3(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d3(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d3(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d4(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d4(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d4(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d4(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d5(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d5(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d5(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d5(int deform, int maxm, const PointArgs &a, cudaStream_t st);
int qmc_launch_eval_d6(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st);
int qmc_occupancy_d6(int deform, int maxm, int precision, int block, int smem, int *out);
int qmc_launch_probe_d6(int deform, int maxm, const ProbeArgs &a, cudaStream_t st);
int qmc_launch_points_d6(int deform, int maxm, const PointArgs &a, cudaStream_t st);


/* ------------------------------------------------------------------ K4: deterministic per-(sector, shift) sums */
/* one warp per (job, sector, shift): lanes take that pair's item partials in a fixed strided order (Kahan), then
   a fixed shuffle tree; results do not depend on which block produced which partial */
__global__ void __launch_bounds__(128) qmc_finalize_kernel(const __grid_constant__ FinTable ft) {
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= ft.total_pairs) return;
    int lo = 0, hi = ft.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ft.jobs[mid].pair_begin <= wg) lo = mid;
        else hi = mid - 1;
    }
    const FinJob &J = ft.jobs[lo];
    const long long pr = wg - J.pair_begin;
    const int ls = (int)(pr / J.m), shift = (int)(pr % J.m);
    const PackedSector *ps = reinterpret_cast<const PackedSector *>(J.packed + J.sectors_off) + J.sector_begin + ls;
    const int orig = ps->orig_index;
    const long long base = pr * J.chunks;
    double s[2 * QMC_MAX_SLOTS], c[2 * QMC_MAX_SLOTS];
#pragma unroll
    for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q) s[q] = c[q] = 0.0;
    unsigned long long f = 0;
    for (long long k = lane; k < J.chunks; k += 32) {
        const double *p = J.partials + (base + k) * J.n_slots * 2;
#pragma unroll
        for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q)
            if (q < 2 * J.n_slots) kahan_add(s[q], c[q], p[q]);
        f += J.part_fails[base + k];
    }
#pragma unroll
    for (int q = 0; q < 2 * QMC_MAX_SLOTS; ++q) {
        double v = s[q] - c[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0 && q < 2 * J.n_slots) J.sums[((long long)orig * J.m + shift) * J.n_slots * 2 + q] = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
    if (lane == 0) J.fails[(long long)orig * J.m + shift] = (int64_t)f;
}

int qmc_launch_eval(int dim, int deform, int maxm, int precision, const JobTable &a, int grid, int block,
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

int qmc_launch_finalize(const FinTable &t, void *stream) {
    if (t.total_pairs == 0) return QMC_OK;
    const int block = 128;
    const long long grid = (t.total_pairs * 32 + block - 1) / block;
    qmc_finalize_kernel<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(t);
    return cudaPeekAtLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int qmc_device_sm_count(int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_NO_DEVICE;
    return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}
