// heat_sweeps_f32.cu -- instantiation of the sweep kernels for the FP32 path (increment form).
#include "heat_kernels.cuh"

namespace heat {

cudaError_t sweep_fp32(heat_ctx *ctx, int dir, const void *a, void *b)
{
    return sweep_mode<float, MODE_DELTA>(ctx, dir, (const float *)a, (float *)b, ctx->dR.t32, ctx->dZ.t32);
}

}  // namespace heat
