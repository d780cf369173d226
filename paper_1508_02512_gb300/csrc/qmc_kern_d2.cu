/* Instantiations of the evaluation kernels for 2-dimensional sectors (one translation unit per sector
 * dimension so that the library builds in parallel). */
#include "qmc_device.cuh"

int qmc_launch_eval_d2(int deform, int maxm, int precision, const JobTable &a, int grid, int block, cudaStream_t st) {
    if (precision == QMC_PREC_MIXED) {
        switch (deform * 10 + maxm) {
        case 0: return launch_eval_f32_t<2, false, 0>(a, grid, block, st);
        case 2: return launch_eval_f32_t<2, false, 2>(a, grid, block, st);
        case 4: return launch_eval_f32_t<2, false, 4>(a, grid, block, st);
        case 10: return launch_eval_f32_t<2, true, 0>(a, grid, block, st);
        case 12: return launch_eval_f32_t<2, true, 2>(a, grid, block, st);
        case 14: return launch_eval_f32_t<2, true, 4>(a, grid, block, st);
            default: return QMC_ERR_UNSUPPORTED;
        }
    }
    switch (deform * 10 + maxm) {
        case 0: return launch_eval_t<2, false, 0>(a, grid, block, st);
        case 2: return launch_eval_t<2, false, 2>(a, grid, block, st);
        case 4: return launch_eval_t<2, false, 4>(a, grid, block, st);
        case 10: return launch_eval_t<2, true, 0>(a, grid, block, st);
        case 12: return launch_eval_t<2, true, 2>(a, grid, block, st);
        case 14: return launch_eval_t<2, true, 4>(a, grid, block, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_occupancy_d2(int deform, int maxm, int precision, int block, int smem, int *out) {
    if (precision == QMC_PREC_MIXED) {
        switch (deform * 10 + maxm) {
        case 0: return occupancy_f32_t<2, false, 0>(block, smem, out);
        case 2: return occupancy_f32_t<2, false, 2>(block, smem, out);
        case 4: return occupancy_f32_t<2, false, 4>(block, smem, out);
        case 10: return occupancy_f32_t<2, true, 0>(block, smem, out);
        case 12: return occupancy_f32_t<2, true, 2>(block, smem, out);
        case 14: return occupancy_f32_t<2, true, 4>(block, smem, out);
            default: return QMC_ERR_UNSUPPORTED;
        }
    }
    switch (deform * 10 + maxm) {
        case 0: return occupancy_t<2, false, 0>(block, smem, out);
        case 2: return occupancy_t<2, false, 2>(block, smem, out);
        case 4: return occupancy_t<2, false, 4>(block, smem, out);
        case 10: return occupancy_t<2, true, 0>(block, smem, out);
        case 12: return occupancy_t<2, true, 2>(block, smem, out);
        case 14: return occupancy_t<2, true, 4>(block, smem, out);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_points_d2(int deform, int maxm, const PointArgs &a, cudaStream_t st) {
    switch (deform * 10 + maxm) {
        case 0: return launch_points_t<2, false, 0>(a, st);
        case 2: return launch_points_t<2, false, 2>(a, st);
        case 4: return launch_points_t<2, false, 4>(a, st);
        case 10: return launch_points_t<2, true, 0>(a, st);
        case 12: return launch_points_t<2, true, 2>(a, st);
        case 14: return launch_points_t<2, true, 4>(a, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

int qmc_launch_probe_d2(int deform, int maxm, const ProbeArgs &a, cudaStream_t st) {
    switch (deform * 10 + maxm) {
        case 0: return launch_probe_t<2, false, 0>(a, st);
        case 2: return launch_probe_t<2, false, 2>(a, st);
        case 4: return launch_probe_t<2, false, 4>(a, st);
        case 10: return launch_probe_t<2, true, 0>(a, st);
        case 12: return launch_probe_t<2, true, 2>(a, st);
        case 14: return launch_probe_t<2, true, 4>(a, st);
        default: return QMC_ERR_UNSUPPORTED;
    }
}

