// heat_small.cu -- whole ADI steps (Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2",
// literal FP64 form) of one small instance in a single persistent launch.
//
// A grid of 64 x 128 cells is 8192 cells: one step's two sweeps are too little
// work to fill the GPU, and as four kernel launches per step the step time is
// the launches' latency.  Here one cooperative launch runs n steps: every warp
// solves whole lines (a line of N <= 256 cells held as K = N/32 consecutive
// cells per lane, the factorized recurrences partitioned over the lanes and
// joined by warp scans of their affine maps), the r-lines of a step, a grid
// barrier, the z-lines, a grid barrier.  The barrier is one arrival counter
// in global memory, zeroed before each launch; a cooperative launch guarantees
// that every block is resident, and each wait is bounded (1 s), after which
// the block records the time-out in the context's status word (heat_sync
// reports HEAT_ERR_TIMEOUT) and the kernel ends.
#include "heat_internal.h"

namespace heat {
namespace {

constexpr int kSmMaxWarps = 8;  // warps per block at most
constexpr unsigned long long kSmWaitNs = 1000000000ULL;
constexpr int kSmMaxN = 256;  // longest line either way

__device__ __forceinline__ unsigned long long sm_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned sm_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier over the launch's nblk resident blocks: bar[0] counts every
// arrival of the launch (zeroed before the launch), so the b-th barrier has
// passed when it reaches b nblk; target (thread 0's) is this block's next
// such count.  false when the wait ran out.
__device__ bool sm_grid_sync(unsigned *bar, unsigned nblk, unsigned &target, int *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        target += nblk;
        __threadfence();
        if (atomicAdd(&bar[0], 1u) + 1u != target) {
            const unsigned long long t0 = sm_clock();
            while ((int)(sm_ld_acquire(&bar[0]) - target) < 0) {
                if (sm_clock() - t0 > kSmWaitNs) {
                    atomicOr(status, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Solve the warp's line in place: d holds the right-hand side of each of the
// lane's K cells, on return the solution (d'_i = d_i inv_i + f_i d'_{i-1},
// x_i = d'_i + cp_i x_{i+1}); cells past the line have zero coefficients.
template <int K>
__device__ __forceinline__ void sm_warp_solve(double (&d)[K], const double (&inv)[K], const double (&f)[K],
                                              const double (&cp)[K], int lane)
{
    const unsigned FULL = 0xffffffffu;
    double F = 1.0, B = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        B = fma(d[k], inv[k], f[k] * B);
        F *= f[k];
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double Fp = __shfl_up_sync(FULL, F, off), Bp = __shfl_up_sync(FULL, B, off);
        if (lane >= off) {
            B = fma(F, Bp, B);
            F *= Fp;
        }
    }
    double y = __shfl_up_sync(FULL, B, 1);
    if (lane == 0) y = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        y = fma(d[k], inv[k], f[k] * y);
        d[k] = y;
    }
    double H = 1.0, G = 0.0;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        G = fma(cp[k], G, d[k]);
        H *= cp[k];
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double Hn = __shfl_down_sync(FULL, H, off), Gn = __shfl_down_sync(FULL, G, off);
        if (lane + off < 32) {
            G = fma(H, Gn, G);
            H *= Hn;
        }
    }
    double x = __shfl_down_sync(FULL, G, 1);
    if (lane == 31) x = 0.0;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        x = fma(cp[k], x, d[k]);
        d[k] = x;
    }
}

// n steps; flip: the buffer holding the current field (0: f0), as for the
// sweep plans.  The grid has a warp for every line (each warp owns r-line
// j = its index, if j < Nz, and z-line i = its index, if i < Nr), so a warp's
// coefficients -- the factorization {inv, f, cp} and the explicit direction's
// couplings of its cells -- are loaded once, before the steps, and stay in
// registers.  Field loads bypass L1 (other blocks rewrite the fields between
// the barriers).
template <int KR, int KZ>
__global__ void __launch_bounds__(32 * kSmMaxWarps) small_steps_kernel(const SweepArgs<double> *__restrict__ args,
                                                                      int flip, int nsteps, unsigned *bar, int stall)
{
    const SweepArgs<double> &A = args[0];
    const int Nr = A.Nr, Nz = A.Nz;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    double *__restrict__ fa = flip ? A.f1 : A.f0;  // the field
    double *__restrict__ fb = flip ? A.f0 : A.f1;  // the half layer
    const LineTab<double> &R = A.R, &Z = A.Z;
    const bool rl = gw < Nz, zl = gw < Nr;  // (warp-uniform)
    // r-line j = gw: per cell i = lane KR + k the factorization of its row
    // class and c0 = w_r + ad_z, am_z, ap_z, c1 = s_r + sd_z
    double rinv[KR], rf[KR], rcp[KR], rc0[KR], ram[KR], rap[KR], rc1[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int i = lane * KR + k;
        rinv[k] = rf[k] = rcp[k] = rc0[k] = ram[k] = rap[k] = rc1[k] = 0.0;
        if (rl && i < Nr) {
            const size_t ro = (size_t)A.rowcls[gw] * Nr + i, zo = (size_t)A.colcls[i] * Nz + gw;
            rinv[k] = R.inv[ro], rf[k] = R.f[ro], rcp[k] = R.cp[ro];
            rc0[k] = R.w[ro] + Z.ad[zo], ram[k] = Z.am[zo], rap[k] = Z.ap[zo], rc1[k] = R.s[ro] + Z.sd[zo];
        }
    }
    // z-line i = gw: per cell j = lane KZ + k likewise with the roles swapped
    double zinv[KZ], zf[KZ], zcp[KZ], zc0[KZ], zam[KZ], zap[KZ], zc1[KZ];
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = lane * KZ + k;
        zinv[k] = zf[k] = zcp[k] = zc0[k] = zam[k] = zap[k] = zc1[k] = 0.0;
        if (zl && j < Nz) {
            const size_t zo = (size_t)A.colcls[gw] * Nz + j, ro = (size_t)A.rowcls[j] * Nr + gw;
            zinv[k] = Z.inv[zo], zf[k] = Z.f[zo], zcp[k] = Z.cp[zo];
            zc0[k] = Z.w[zo] + R.ad[ro], zam[k] = R.am[ro], zap[k] = R.ap[ro], zc1[k] = Z.s[zo] + R.sd[ro];
        }
    }
    unsigned target = 0;  // (thread 0) the arrival count that ends the next barrier
    // failure-detection test (heat_test_stall): wait for one block more than
    // the grid has, so the first barrier's wait runs out
    const unsigned nblk = gridDim.x + (stall ? 1u : 0u);
    for (int s = 0; s < nsteps; ++s) {
        // r-line: row j of fa -> row j of fb (implicit in r, explicit in z)
        if (rl) {
            const int j = gw;
            double d[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int i = lane * KR + k;
                d[k] = 0.0;
                if (i < Nr) {
                    const double t0 = __ldcg(fa + (size_t)j * Nr + i);
                    const double tm = j > 0 ? __ldcg(fa + (size_t)(j - 1) * Nr + i) : 0.0;
                    const double tp = j < Nz - 1 ? __ldcg(fa + (size_t)(j + 1) * Nr + i) : 0.0;
                    d[k] = fma(rc0[k], t0, fma(ram[k], tm, fma(rap[k], tp, rc1[k])));
                }
            }
            sm_warp_solve<KR>(d, rinv, rf, rcp, lane);
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int i = lane * KR + k;
                if (i < Nr) fb[(size_t)j * Nr + i] = d[k];
            }
        }
        if (!sm_grid_sync(bar, nblk, target, A.status)) return;
        // z-line: column i of fb -> column i of fa (implicit in z, explicit in r)
        if (zl) {
            const int i = gw;
            double d[KZ];
#pragma unroll
            for (int k = 0; k < KZ; ++k) {
                const int j = lane * KZ + k;
                d[k] = 0.0;
                if (j < Nz) {
                    const double *row = fb + (size_t)j * Nr;
                    const double t0 = __ldcg(row + i);
                    const double tl = i > 0 ? __ldcg(row + i - 1) : 0.0;
                    const double tr = i < Nr - 1 ? __ldcg(row + i + 1) : 0.0;
                    d[k] = fma(zc0[k], t0, fma(zam[k], tl, fma(zap[k], tr, zc1[k])));
                }
            }
            sm_warp_solve<KZ>(d, zinv, zf, zcp, lane);
#pragma unroll
            for (int k = 0; k < KZ; ++k) {
                const int j = lane * KZ + k;
                if (j < Nz) fa[(size_t)j * Nr + i] = d[k];
            }
        }
        if (!sm_grid_sync(bar, nblk, target, A.status)) return;
    }
}

int sm_cells_per_lane(int N)
{
    int K = 1;
    while (32 * K < N) K *= 2;
    return K;
}

template <int KR>
const void *sm_pick_z(int KZ)
{
    switch (KZ) {
    case 1: return (const void *)small_steps_kernel<KR, 1>;
    case 2: return (const void *)small_steps_kernel<KR, 2>;
    case 4: return (const void *)small_steps_kernel<KR, 4>;
    default: return (const void *)small_steps_kernel<KR, 8>;
    }
}
const void *sm_pick(int KR, int KZ)
{
    switch (KR) {
    case 1: return sm_pick_z<1>(KZ);
    case 2: return sm_pick_z<2>(KZ);
    case 4: return sm_pick_z<4>(KZ);
    default: return sm_pick_z<8>(KZ);
    }
}

}  // namespace

// Set up the persistent step kernel for a small FP64 instance (both line
// lengths <= 256 cells, not a batch member, cooperative launch available):
// its kernel, grid and barrier words.  Leaves small_fn null otherwise.
cudaError_t small_setup(heat_ctx *ctx)
{
    ctx->small_fn = nullptr;
    if (ctx->precision != HEAT_FP64 || ctx->batch_member) return cudaSuccess;
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    if (Nr > kSmMaxN || Nz > kSmMaxN) return cudaSuccess;
    int coop = 0;
    cudaError_t e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (e != cudaSuccess) return e;
    if (!coop) return cudaSuccess;
    const void *fn = sm_pick(sm_cells_per_lane(Nr), sm_cells_per_lane(Nz));
    // a warp for every line of the longer direction, one block per SM, as
    // few warps per block as that allows: the FP64 work spreads over the
    // most SMs (FP64 retires 2 FMAs per clock per SM; config 1 at 64 x 128:
    // 13.3 / 10.8 / 10.0 / 10.6 us per step with 8 / 4 / 2 / 1 warps per
    // block -- at one warp per block the barrier's arrivals cost more)
    int nsm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess) return e;
    const int lines = Nr > Nz ? Nr : Nz;
    int wpb = 2;
    while (wpb < kSmMaxWarps && (lines + wpb - 1) / wpb > nsm) wpb *= 2;
    const int blocks = (lines + wpb - 1) / wpb;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * wpb, 0)) != cudaSuccess) return e;
    if (blocks < 1 || blocks > nsm || per_sm < 1) return cudaSuccess;
    if (!ctx->d_small_bar) {
        if ((e = cudaMalloc(&ctx->d_small_bar, 2 * sizeof(unsigned))) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ctx->d_small_bar, 0, 2 * sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
    }
    ctx->small_fn = fn;
    ctx->small_blocks = blocks;
    ctx->small_wpb = wpb;
    return cudaSuccess;
}

// n whole steps in one cooperative launch (small_setup found the instance small).
cudaError_t launch_small_steps(heat_ctx *ctx, int n)
{
    int flip = ctx->cur, steps = n, stall = ctx->rw_stall;
    unsigned *bar = ctx->d_small_bar;
    // a barrier left half-arrived by a wait that ran out must not carry over
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), ctx->stream);
    if (e != cudaSuccess) return e;
    void *kargs[5] = {(void *)&ctx->d_args, (void *)&flip, (void *)&steps, (void *)&bar, (void *)&stall};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctx->small_blocks, 1, 1);
    cfg.blockDim = dim3(32 * ctx->small_wpb, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, ctx->small_fn, kargs);
}

}  // namespace heat
