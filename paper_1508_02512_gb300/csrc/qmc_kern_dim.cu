/* Instantiations of the ahead-of-time evaluation kernels for QMC_S-dimensional sectors.  The build compiles this
 * file once per sector dimension (-DQMC_S=1..6), so that the library builds in parallel; each copy defines the
 * dispatchers qmc_launch_eval_d<S>, qmc_occupancy_d<S>, qmc_launch_points_d<S> and qmc_launch_probe_d<S>. */
#include "qmc_device.cuh"

#ifndef QMC_S
#error "compile with -DQMC_S=<sector dimension 1..6>"
#endif

#define QMC_CAT2(a, b) a##b
#define QMC_CAT(a, b) QMC_CAT2(a, b)
#define QMC_FN(name) QMC_CAT(name, QMC_S)

/* one case per (sector class, series length): key = class * 10 + maxm, maxm in {0, 2, 4}; class 0 undeformed,
   1 deformed (the template's DEF), 2 undeformed with endpoint exponents alpha <= -2 (FP64 only) */
#define QMC_TAYLOR_CASES(CALL)                                                                                     \
    case 20: return CALL(0);                                                                                       \
    case 22: return CALL(2);                                                                                       \
    case 24: return CALL(4);
#define QMC_CASES(CALL)                                                                                            \
    case 0: return CALL(false, 0);                                                                                 \
    case 2: return CALL(false, 2);                                                                                 \
    case 4: return CALL(false, 4);                                                                                 \
    case 10: return CALL(true, 0);                                                                                 \
    case 12: return CALL(true, 2);                                                                                 \
    case 14: return CALL(true, 4);

int QMC_FN(qmc_launch_eval_d)(int deform, int maxm, int precision, const JobTable &a, int grid, int block,
                              cudaStream_t st) {
#define F32(D, M) launch_eval_f32_t<QMC_S, D, M>(a, grid, block, st)
#define F64(D, M) launch_eval_t<QMC_S, D, M>(a, grid, block, st)
#define TAY(M) launch_eval_taylor_t<QMC_S, M>(a, grid, block, st)
    if (precision == QMC_PREC_MIXED) {
        switch (deform * 10 + maxm) {
            QMC_CASES(F32)
            default: return QMC_ERR_UNSUPPORTED;
        }
    }
    switch (deform * 10 + maxm) {
        QMC_CASES(F64)
        QMC_TAYLOR_CASES(TAY)
        default: return QMC_ERR_UNSUPPORTED;
    }
#undef F32
#undef F64
#undef TAY
}

int QMC_FN(qmc_occupancy_d)(int deform, int maxm, int precision, int block, int smem, int *out) {
#define F32(D, M) occupancy_f32_t<QMC_S, D, M>(block, smem, out)
#define F64(D, M) occupancy_t<QMC_S, D, M>(block, smem, out)
#define TAY(M) occupancy_taylor_t<QMC_S, M>(block, smem, out)
    if (precision == QMC_PREC_MIXED) {
        switch (deform * 10 + maxm) {
            QMC_CASES(F32)
            default: return QMC_ERR_UNSUPPORTED;
        }
    }
    switch (deform * 10 + maxm) {
        QMC_CASES(F64)
        QMC_TAYLOR_CASES(TAY)
        default: return QMC_ERR_UNSUPPORTED;
    }
#undef F32
#undef F64
#undef TAY
}

int QMC_FN(qmc_launch_points_d)(int deform, int maxm, const PointArgs &a, cudaStream_t st) {
#define PTS(D, M) launch_points_t<QMC_S, D, M>(a, st)
#define TAY(M) launch_points_taylor_t<QMC_S, M>(a, st)
    switch (deform * 10 + maxm) {
        QMC_CASES(PTS)
        QMC_TAYLOR_CASES(TAY)
        default: return QMC_ERR_UNSUPPORTED;
    }
#undef PTS
#undef TAY
}

int QMC_FN(qmc_launch_probe_d)(int deform, int maxm, const ProbeArgs &a, cudaStream_t st) {
#define PRB(D, M) launch_probe_t<QMC_S, D, M>(a, st)
    switch (deform * 10 + maxm) {
        QMC_CASES(PRB)
        default: return QMC_ERR_UNSUPPORTED;
    }
#undef PRB
}
