// heat_noalloc.cu -- heat_energy_noalloc: the energy / boundary-flux reduction
// of heat_energy with its scratch in a fixed file-scope device array instead
// of memory owned by the context.
//
// Who needs it: a caller that must not allocate device memory at the moment it
// asks for the heat balance -- a monitor thread running beside a step loop
// under a hard memory budget, or code that audits a context it did not create
// and so cannot rely on that context's scratch being free.  cudaMalloc can
// synchronise the whole device and can fail once the budget is spent; this
// entry point does neither.  Nothing here calls cudaMalloc, cudaFree or a
// library that allocates.
//
// Decomposition: one block per grid row j (the same energy_kernel as
// heat_energy, launched with Nz blocks), so the partial sums need 2 * Nz
// doubles; a second block folds them into the pair (E - E_ref, Phi).  The
// array holds kNoAllocMaxRows rows' partials, so Nz above that is rejected.
//
// Per-device set-up: the first call on each device (that device current)
// looks up the array's device address with cudaGetSymbolAddress and caches
// it.  That first call may load the module, so it must come before any
// stream capture on that device.
//
// Contents persist between calls: each call's row kernel overwrites the
// partial slots it reads (rows 0..Nz-1) before the fold reads them, and the
// fold writes both result slots, so nothing from a previous call, possibly on
// a larger grid, can leak in.  Two calls whose device work overlapped would
// race on the one array; a process-wide lock, held until the call's stream has
// drained -- on the error paths too, once anything has been queued -- keeps
// calls made through this entry point from overlapping.
//
// The array used is the one on the context's device: the call checks that
// this device is current and otherwise returns HEAT_ERR_ARG (a launch with
// another device current would fail, or with peer access reach the other
// device's array).
#include <cmath>
#include <mutex>

#include "heat_kernels.cuh"

namespace heat {

constexpr int kNoAllocMaxRows = HEAT_NOALLOC_MAX_ROWS;
constexpr int kNoAllocMaxDevices = 64;

// [0, 1]: result (E - E_ref, Phi); [2, 2 + 2 * kNoAllocMaxRows): per-row partials.
static __device__ __align__(256) double g_energy_scratch[2 + 2 * kNoAllocMaxRows];

static std::mutex g_noalloc_lock;
static double *g_scratch_addr[kNoAllocMaxDevices];

}  // namespace heat

using namespace heat;

extern "C" int heat_energy_noalloc(heat_ctx *ctx, double *E, double *Phi, double *Q)
{
    if (!ctx) return HEAT_ERR_ARG;
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    if (Nz > kNoAllocMaxRows) return HEAT_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return HEAT_ERR_CUDA;
    if (dev != ctx->device) return HEAT_ERR_ARG;

    std::lock_guard<std::mutex> hold(g_noalloc_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) return HEAT_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    double *res = g_scratch_addr[dev];
    double *part = res + 2;

    // From the first enqueue on, every exit drains the stream before the lock
    // is released, so no work of this call is left touching the array.
    auto drained = [&](int status) {
        cudaStreamSynchronize(ctx->stream);
        return status;
    };
    if (ctx->precision == HEAT_FP64)
        energy_kernel<double><<<Nz, 256, 0, ctx->stream>>>(static_cast<const double *>(ctx->d_field[ctx->cur]), Nr, Nz,
                                                          ctx->d_rowcls, ctx->d_colcls, ctx->dR.full, ctx->dZ.full,
                                                          ctx->d_wr, ctx->d_wz, part);
    else
        energy_kernel<float><<<Nz, 256, 0, ctx->stream>>>(static_cast<const float *>(ctx->d_field[ctx->cur]), Nr, Nz,
                                                         ctx->d_rowcls, ctx->d_colcls, ctx->dR.full, ctx->dZ.full,
                                                         ctx->d_wr, ctx->d_wz, part);
    if (cudaGetLastError() != cudaSuccess) return drained(HEAT_ERR_CUDA);
    energy_final_kernel<<<1, 256, 0, ctx->stream>>>(part, Nz, res);
    if (cudaGetLastError() != cudaSuccess) return drained(HEAT_ERR_CUDA);

    double out[2];
    if (cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return drained(HEAT_ERR_CUDA);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return HEAT_ERR_CUDA;
    if (E) *E = out[0] + ctx->E_ref;
    if (Phi) *Phi = out[1];
    if (Q) *Q = ctx->Q;
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return HEAT_ERR_NONFINITE;
    return HEAT_OK;
}
