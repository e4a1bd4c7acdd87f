// heat_sweeps_f64.cu -- instantiation of the sweep kernels for the FP64 path (literal form of eqs. "scheme_eq_1", "scheme_eq_2").
#include "heat_kernels.cuh"

namespace heat {

cudaError_t sweep_fp64(heat_ctx *ctx, int dir, const void *a, void *b)
{
    return sweep_mode<double, MODE_LIT>(ctx, dir, (const double *)a, (double *)b, ctx->dR.t64, ctx->dZ.t64);
}

}  // namespace heat
