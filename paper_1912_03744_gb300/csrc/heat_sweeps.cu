// heat_sweeps.cu -- host launchers of one ADI step (dispatch by precision to
// the per-form translation units), the FP64 energy/flux reduction and the
// field conversions.  The kernels are in heat_kernels.cuh.
#include "heat_kernels.cuh"

namespace heat {

// One half-step from buffer a into buffer b.
cudaError_t launch_sweep_buffers(heat_ctx *ctx, int dir, const void *a, void *b)
{
    switch (ctx->precision) {
    case HEAT_FP64: return sweep_fp64(ctx, dir, a, b);
    case HEAT_FP32: return sweep_fp32(ctx, dir, a, b);
    default: return sweep_fp32_refined(ctx, dir, a, b);
    }
}

cudaError_t launch_sweep(heat_ctx *ctx, int dir)
{
    return launch_sweep_buffers(ctx, dir, ctx->d_field[ctx->cur], ctx->d_field[1 - ctx->cur]);
}

cudaError_t launch_steps(heat_ctx *ctx, int n)
{
    for (int s = 0; s < n; ++s) {
        cudaError_t e = launch_sweep_buffers(ctx, 0, ctx->d_field[ctx->cur], ctx->d_field[1 - ctx->cur]);
        if (e != cudaSuccess) return e;
        e = launch_sweep_buffers(ctx, 1, ctx->d_field[1 - ctx->cur], ctx->d_field[ctx->cur]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// r-sweep: 1 launch; z-sweep: 3 (summaries, carries, solve), 6 on the refined path.
int launches_per_step(const heat_ctx *ctx) { return ctx->precision == HEAT_FP32_REFINED ? 7 : 4; }

int energy_blocks(const heat_ctx *ctx)
{
    const int nb = ctx->g.Nz < 1024 ? ctx->g.Nz : 1024;
    return nb;
}

cudaError_t launch_energy(heat_ctx *ctx)
{
    const int nb = energy_blocks(ctx);
    if (ctx->precision == HEAT_FP64)
        energy_kernel<double><<<nb, 256, 0, ctx->stream>>>(static_cast<const double *>(ctx->d_field[ctx->cur]),
                                                          ctx->g.Nr, ctx->g.Nz, ctx->d_rowcls, ctx->d_colcls,
                                                          ctx->dR.full, ctx->dZ.full, ctx->d_wr, ctx->d_wz,
                                                          ctx->d_part);
    else
        energy_kernel<float><<<nb, 256, 0, ctx->stream>>>(static_cast<const float *>(ctx->d_field[ctx->cur]),
                                                         ctx->g.Nr, ctx->g.Nz, ctx->d_rowcls, ctx->d_colcls,
                                                         ctx->dR.full, ctx->dZ.full, ctx->d_wr, ctx->d_wz,
                                                         ctx->d_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d_part, nb, ctx->d_res);
    return cudaGetLastError();
}

cudaError_t launch_theta_to_T(heat_ctx *ctx, double *T)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        theta_to_T_kernel<double><<<grid, 256, 0, ctx->stream>>>(static_cast<const double *>(ctx->d_field[ctx->cur]), T,
                                                                n, ctx->T_ref);
    else
        theta_to_T_kernel<float><<<grid, 256, 0, ctx->stream>>>(static_cast<const float *>(ctx->d_field[ctx->cur]), T,
                                                               n, ctx->T_ref);
    return cudaGetLastError();
}

cudaError_t launch_T_to_theta(heat_ctx *ctx, const double *T)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        T_to_theta_kernel<double><<<grid, 256, 0, ctx->stream>>>(T, static_cast<double *>(ctx->d_field[ctx->cur]), n,
                                                                ctx->T_ref);
    else
        T_to_theta_kernel<float><<<grid, 256, 0, ctx->stream>>>(T, static_cast<float *>(ctx->d_field[ctx->cur]), n,
                                                               ctx->T_ref);
    return cudaGetLastError();
}

cudaError_t launch_fill(heat_ctx *ctx, int buf, double value)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        fill_kernel<double><<<grid, 256, 0, ctx->stream>>>(static_cast<double *>(ctx->d_field[buf]), n, value);
    else
        fill_kernel<float><<<grid, 256, 0, ctx->stream>>>(static_cast<float *>(ctx->d_field[buf]), n, (float)value);
    return cudaGetLastError();
}

}  // namespace heat
