// heat_sweeps_f32r.cu -- instantiation of the sweep kernels for the refined FP32 path (increment form + FP64 residual correction).
#include "heat_kernels.cuh"

namespace heat {

cudaError_t sweep_fp32_refined(heat_ctx *ctx, int dir, const void *a, void *b)
{
    return sweep_mode<float, MODE_REFINE>(ctx, dir, (const float *)a, (float *)b, ctx->dR.t32, ctx->dZ.t32);
}

}  // namespace heat
