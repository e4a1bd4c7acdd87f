// heat_kernels.cuh -- sm_103a kernels of one Peaceman-Rachford ADI step
// (templates; instantiated per precision/form in heat_sweeps_*.cu).
//
// One step (Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2") on the field stored
// row-major [Nz][Nr] (FP64: T; FP32: theta = T - T_init):
//   r-sweep: for every row j solve the r-line system
//       (W - L_r) thbar = (W + L_z) th + X        (W = 2C/tau)
//   z-sweep: for every column i solve the z-line system
//       (W - L_z) thhat = (W + L_r) thbar + X
// Each line matrix is fixed per line class (see heat_internal.h), so its
// Thomas factorization is precomputed and a line solve is two first-order
// linear recurrences:  d'_i = d_i inv_i + f_i d'_{i-1},  x_i = d'_i + cp_i x_{i+1}.
//
// Two algebraically identical forms of each half-step:
//   literal (FP64 path): the right-hand side above, solved for the new value;
//   increment (FP32 paths): (W - L_dir) delta = (L_r + L_z) th + X and
//       th_new = th + delta, every coupling applied to a difference
//       (th_nb - th).  In FP32 the factorization error then scales with
//       |delta| instead of |th|, and a steady state is reproduced exactly.
// Refined FP32 path: after the FP32 solve, the residual of the increment
// system is formed in FP64 from FP64 coefficients and one more FP32 solve
// corrects delta (one step of mixed-precision iterative refinement).
//
// r-sweep (rows are contiguous).  One line per block (or per warp segment
// for short rows); thread g owns the K consecutive cells [gK, gK+K).  Each
// thread runs the forward recurrence on its chunk with a zero carry, giving
// the affine map carry_out = B + F carry_in; an exclusive scan of these maps
// (warp shuffles, then shared memory across warps) yields every chunk's true
// carry-in and the thread reruns its chunk; the backward recurrence likewise
// from the other end.  A block walks a band of consecutive rows; the rows it
// needs (j-1, j, j+1 for the explicit z-operator, and rows further ahead) are
// prefetched into a shared-memory ring with cp.async, so many rows are in
// flight per SM while registers hold only the line-class tables and a chunk.
//
// z-sweep (columns are strided).  A block owns 32 columns (one per lane:
// every row access is a coalesced 128-byte segment) and a chunk of Rc rows,
// KZ rows per thread.  Pass 1 (zsum) reduces each column chunk to its two
// carry summaries, written as weighted sums of the right-hand side with
// matrix-only weights (see ZPart in heat_internal.h).  Pass 2 (zsolve)
// derives the exact carries of its chunk from all chunk summaries of the
// column, then solves the chunk (in-block carry scans over warps).  No block
// waits on another block.
#pragma once

#include <cstdio>

#include "heat_internal.h"

namespace heat {

#define HEAT_FULL_MASK 0xffffffffu

enum { MODE_LIT = 0, MODE_DELTA = 1, MODE_REFINE = 2, MODE_CORR = 3 };

// theta_bc of the faces r_lo, r_hi, z_lo, z_hi
struct BcVals {
    double th[4];
};

__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }

// Exclusive left-to-right scan of affine maps y = B + F x over segments of W
// lanes.  On return (F, B) is the inclusive map, (Fe, Be) the exclusive one.
template <typename real>
__device__ __forceinline__ void seg_scan_fwd(real &F, real &B, real &Fe, real &Be, int ls, int W)
{
    for (int off = 1; off < W; off <<= 1) {
        const real F2 = __shfl_up_sync(HEAT_FULL_MASK, F, off, W);
        const real B2 = __shfl_up_sync(HEAT_FULL_MASK, B, off, W);
        if (ls >= off) {
            B = fmad(F, B2, B);
            F = F * F2;
        }
    }
    Fe = __shfl_up_sync(HEAT_FULL_MASK, F, 1, W);
    Be = __shfl_up_sync(HEAT_FULL_MASK, B, 1, W);
    if (ls == 0) {
        Fe = real(1);
        Be = real(0);
    }
}

// Exclusive right-to-left (suffix) scan of maps y = G + H x over segments of W lanes.
template <typename real>
__device__ __forceinline__ void seg_scan_bwd(real &H, real &G, real &He, real &Ge, int ls, int W)
{
    for (int off = 1; off < W; off <<= 1) {
        const real H2 = __shfl_down_sync(HEAT_FULL_MASK, H, off, W);
        const real G2 = __shfl_down_sync(HEAT_FULL_MASK, G, off, W);
        if (ls + off < W) {
            G = fmad(H, G2, G);
            H = H * H2;
        }
    }
    He = __shfl_down_sync(HEAT_FULL_MASK, H, 1, W);
    Ge = __shfl_down_sync(HEAT_FULL_MASK, G, 1, W);
    if (ls == W - 1) {
        He = real(1);
        Ge = real(0);
    }
}

// ---- cp.async helpers (asynchronous global->shared copies; completion is
// awaited with the hardware wait_group, no spin loop)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// K consecutive values from shared memory (16-byte loads; K*sizeof(real) % 16 == 0).
template <typename real, int K>
__device__ __forceinline__ void lds_chunk(const real *p, real (&v)[K])
{
    constexpr int V = 16 / (int)sizeof(real);
#pragma unroll
    for (int k = 0; k < K; k += V) {
        if constexpr (sizeof(real) == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p + k);
            v[k] = t.x;
            v[k + 1] = t.y;
            v[k + 2] = t.z;
            v[k + 3] = t.w;
        } else {
            const double2 t = *reinterpret_cast<const double2 *>(p + k);
            v[k] = t.x;
            v[k + 1] = t.y;
        }
    }
}

template <typename real, int K>
__device__ __forceinline__ void store_chunk(real *__restrict__ row, int i0, int n, bool vec, const real (&v)[K])
{
    constexpr int V = 16 / (int)sizeof(real);
    if (vec && i0 + K <= n) {
#pragma unroll
        for (int k = 0; k < K; k += V) {
            if constexpr (sizeof(real) == 4)
                *reinterpret_cast<float4 *>(row + i0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            else
                *reinterpret_cast<double2 *>(row + i0 + k) = make_double2(v[k], v[k + 1]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i0 + k < n) row[i0 + k] = v[k];
    }
}

// K consecutive values of row x (zero outside the field), 16-byte loads when aligned.
template <typename real, int K>
__device__ __forceinline__ void ldg_row(const real *__restrict__ th, int x, int Nr, int Nz, int i0, bool vec,
                                        real (&v)[K])
{
    constexpr int V = 16 / (int)sizeof(real);
    const bool rin = x >= 0 && x < Nz;
    const real *row = th + (size_t)(rin ? x : 0) * Nr;
    if (rin && vec && i0 + K <= Nr) {
#pragma unroll
        for (int k = 0; k < K; k += V) {
            if constexpr (sizeof(real) == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(row + i0 + k));
                v[k] = t.x, v[k + 1] = t.y, v[k + 2] = t.z, v[k + 3] = t.w;
            } else {
                const double2 t = __ldg(reinterpret_cast<const double2 *>(row + i0 + k));
                v[k] = t.x, v[k + 1] = t.y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (rin && i0 + k < Nr) ? row[i0 + k] : real(0);
    }
}

// Partitioned Thomas solve of one r-line held as K-cell chunks by the G
// threads of a line (segment of W lanes, or whole block when wide).
template <typename real, int K>
__device__ __forceinline__ void solve_row(real (&d)[K], const real (&inv)[K], const real (&f)[K],
                                          const real (&cp)[K], int ls, int W, int lane, int warp, int nwl,
                                          bool wide, real *sA, real *sB, real *sC)
{
    real F = real(1), B = real(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        B = fmad(d[k], inv[k], f[k] * B);
        F *= f[k];
    }
    real Fe, Be;
    seg_scan_fwd(F, B, Fe, Be, ls, W);
    real cin = Be;
    if (wide) {
        if (lane == 31) {
            sA[warp] = F;
            sB[warp] = B;
        }
        __syncthreads();
        if (warp == 0) {
            real f2 = lane < nwl ? sA[lane] : real(1), b2 = lane < nwl ? sB[lane] : real(0), fe, be;
            seg_scan_fwd(f2, b2, fe, be, lane, 32);
            if (lane < nwl) sC[lane] = be;
        }
        __syncthreads();
        cin = fmad(Fe, sC[warp], Be);
    }
    real dp = cin;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dp = fmad(d[k], inv[k], f[k] * dp);
        d[k] = dp;
    }
    real H = real(1), Gm = real(0);
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        Gm = fmad(cp[k], Gm, d[k]);
        H *= cp[k];
    }
    real He, Ge;
    seg_scan_bwd(H, Gm, He, Ge, ls, W);
    real xin = Ge;
    if (wide) {
        __syncthreads();
        if (lane == 0) {
            sA[warp] = H;
            sB[warp] = Gm;
        }
        __syncthreads();
        if (warp == 0) {
            real h2 = lane < nwl ? sA[lane] : real(1), g2 = lane < nwl ? sB[lane] : real(0), he, ge;
            seg_scan_bwd(h2, g2, he, ge, lane, 32);
            if (lane < nwl) sC[lane] = ge;
        }
        __syncthreads();
        xin = fmad(He, sC[warp], Ge);
    }
    real x = xin;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        x = fmad(cp[k], x, d[k]);
        d[k] = x;
    }
}

// ------------------------------------------------------------------ r-sweep
// Block = lpb line slots x G threads; slot s of block b walks rows
// [(b*lpb + s)*band, +band).  Shared memory: a ring of NRING rows per slot
// (row x of the slot's band lives in ring slot (x - jstart + 1) % NRING);
// each thread copies its own K cells of a row with cp.async, one commit group
// per row: group g holds row jstart - 1 + g.  The prologue issues groups
// 0 .. NRING-2; iteration t (row j = jstart + t) needs rows up to j+1 (group
// t+2) while groups up to NRING-2+t are issued, so it waits until at most
// NRING-4 groups are pending.  At its end it issues row j+NRING-2 into the
// slot of row j-2, last read in iteration t-1, i.e. before the barrier that
// opens iteration t; the ring then holds rows j-1 .. j+NRING-2.
// NRING = 0 selects direct global loads of rows j-1, j, j+1 (rows too long
// for a ring in shared memory).
template <typename real, int K, int MODE, int LB, int NRING>
__global__ void __launch_bounds__(LB, LB <= 256 ? 3 : 1) rsweep_kernel(const real *__restrict__ th, real *__restrict__ out, int Nr,
                                                    int Nz, int G, int band, const int *__restrict__ rowcls,
                                                    const int *__restrict__ colcls, LineTab<real> R, LineTab<real> Z,
                                                    LineTab64 R64, LineTab64 Z64, BcVals bc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ real sA[32], sB[32], sC[32];
    __shared__ double sLo[32], sHi[32];
    const int tid = threadIdx.x;
    const int g = tid % G;
    const int slot = tid / G;
    const int lpb = blockDim.x / G;
    const int W = G < 32 ? G : 32;
    const int lane = tid & 31, ls = tid % W, warp = tid >> 5;
    const int nwl = G >> 5;
    const bool wide = G > 32;
    const int i0 = g * K;
    const int Np = G * K;  // padded row length in the ring
    constexpr int V = 16 / (int)sizeof(real);
    const bool vec = (Nr % V) == 0;
    const int jstart = (blockIdx.x * lpb + slot) * band;
    real *ring = reinterpret_cast<real *>(smem_raw) + (size_t)slot * NRING * Np;
    const real bc0 = (real)bc.th[0], bc1 = (real)bc.th[1], bc2 = (real)bc.th[2], bc3 = (real)bc.th[3];

    // copy this thread's K cells of row x (zero outside the field) into its ring slot
    auto fetch = [&](int x) {
        if constexpr (NRING == 0) return;
        real *dst = ring + (size_t)((x - jstart + 1 + NRING) % (NRING > 0 ? NRING : 1)) * Np + i0;
        const bool rin = x >= 0 && x < Nz;
        if (vec) {
#pragma unroll
            for (int k = 0; k < K; k += V) {
                const bool ok = rin && i0 + k < Nr;
                cp_async16(dst + k, ok ? th + (size_t)x * Nr + i0 + k : th, ok ? 16 : 0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) dst[k] = (rin && i0 + k < Nr) ? th[(size_t)x * Nr + i0 + k] : real(0);
        }
        cp_async_commit();
    };

    int zc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) zc[k] = (i0 + k < Nr) ? colcls[i0 + k] : 0;
    bool zuni = true;
#pragma unroll
    for (int k = 1; k < K; ++k) zuni = zuni && (zc[k] == zc[0]);

    // prologue: rows jstart-1 .. jstart+NRING-3
    if constexpr (NRING > 0)
        for (int x = jstart - 1; x <= jstart + NRING - 3; ++x) fetch(x);

    int acls = -1;
    real inv[K], f[K], cp[K], c0[K], c1[K], c2[K];
    real edl = real(0), edh = real(0);  // Dirichlet r-face coefficients of cells 0 / Nr-1
#pragma unroll
    for (int k = 0; k < K; ++k) inv[k] = f[k] = cp[k] = c0[k] = c1[k] = c2[k] = real(0);

    for (int t = 0; t < band; ++t) {
        const int j = jstart + t;
        const bool valid = j < Nz;
        constexpr int NR1 = NRING > 0 ? NRING : 1;
        if constexpr (NRING > 0) {
            cp_async_wait<(NRING >= 4 ? NRING - 4 : 0)>();
            __syncthreads();
        }
        const real *rm = ring + (size_t)((t + 0) % NR1) * Np;  // row j-1
        const real *rc = ring + (size_t)((t + 1) % NR1) * Np;  // row j
        const real *rp = ring + (size_t)((t + 2) % NR1) * Np;  // row j+1
        const int a = valid ? rowcls[j] : (acls < 0 ? 0 : acls);
        if (a != acls) {
            const size_t ro = (size_t)a * Nr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                const bool in = i < Nr;
                inv[k] = in ? R.inv[ro + i] : real(0);
                f[k] = in ? R.f[ro + i] : real(0);
                cp[k] = in ? R.cp[ro + i] : real(0);
                if constexpr (MODE == MODE_LIT) {
                    c0[k] = in ? R.w[ro + i] : real(0);
                    c1[k] = in ? R.s[ro + i] : real(0);
                } else {
                    c0[k] = in ? R.am[ro + i] : real(0);
                    c1[k] = in ? R.ap[ro + i] : real(0);
                    c2[k] = in ? R.q[ro + i] : real(0);
                }
            }
            if constexpr (MODE != MODE_LIT) {
                edl = i0 == 0 ? R.dl[ro] : real(0);
                edh = (i0 <= Nr - 1 && Nr - 1 < i0 + K) ? R.dh[ro + Nr - 1] : real(0);
            }
            acls = a;
        }
        real tc[K], tmv[K], tpv[K];
        real nbl = real(0), nbr = real(0);  // row-j neighbours of the chunk ends
        if constexpr (NRING > 0) {
            lds_chunk<real, K>(rc + i0, tc);
            lds_chunk<real, K>(rm + i0, tmv);
            lds_chunk<real, K>(rp + i0, tpv);
            nbl = i0 > 0 ? rc[i0 - 1] : tc[0];
            nbr = i0 + K < Np ? rc[i0 + K] : tc[K - 1];
        } else {
            ldg_row<real, K>(th, j, Nr, Nz, i0, vec, tc);
            ldg_row<real, K>(th, j - 1, Nr, Nz, i0, vec, tmv);
            ldg_row<real, K>(th, j + 1, Nr, Nz, i0, vec, tpv);
            nbl = (i0 > 0 && valid) ? th[(size_t)j * Nr + i0 - 1] : tc[0];
            nbr = (i0 + K < Nr && valid) ? th[(size_t)j * Nr + i0 + K] : tc[K - 1];
        }
        // z-coefficients of this row for the thread's column classes
        real zam = real(0), zap = real(0), zx = real(0), zy = real(0);
        const bool zdir = valid && (j == 0 || j == Nz - 1);
        if (zuni && valid) {
            const size_t zo = (size_t)zc[0] * Nz + j;
            zam = Z.am[zo];
            zap = Z.ap[zo];
            if constexpr (MODE == MODE_LIT) {
                zx = Z.ad[zo];
                zy = Z.sd[zo];
            } else if (zdir) {
                zx = Z.dl[zo];
                zy = Z.dh[zo];
            }
        }
        real d[K];
        {
            const real left = nbl;
            const real right = nbr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                real am2 = zam, ap2 = zap, x2 = zx, y2 = zy;
                if (!zuni && valid && i0 + k < Nr) {
                    const size_t zo = (size_t)zc[k] * Nz + j;
                    am2 = Z.am[zo];
                    ap2 = Z.ap[zo];
                    if constexpr (MODE == MODE_LIT) {
                        x2 = Z.ad[zo];
                        y2 = Z.sd[zo];
                    } else {
                        x2 = zdir ? Z.dl[zo] : real(0);
                        y2 = zdir ? Z.dh[zo] : real(0);
                    }
                }
                const real t0 = tc[k];
                if constexpr (MODE == MODE_LIT) {
                    d[k] = fmad(c0[k] + x2, t0, fmad(am2, tmv[k], fmad(ap2, tpv[k], c1[k] + y2)));
                } else {
                    const real tl = k > 0 ? tc[k - 1] : left;
                    const real tr = k < K - 1 ? tc[k + 1] : right;
                    real r = c2[k];
                    r = fmad(c0[k], tl - t0, r);
                    r = fmad(c1[k], tr - t0, r);
                    r = fmad(am2, tmv[k] - t0, r);
                    r = fmad(ap2, tpv[k] - t0, r);
                    if (zdir) {
                        r = fmad(x2, bc2 - t0, r);
                        r = fmad(y2, bc3 - t0, r);
                    }
                    if (k == 0) r = fmad(edl, bc0 - t0, r);
                    if (i0 + k == Nr - 1) r = fmad(edh, bc1 - t0, r);
                    d[k] = valid && i0 + k < Nr ? r : real(0);
                }
            }
        }
        if constexpr (MODE == MODE_REFINE) {
            real dl0[K];
#pragma unroll
            for (int k = 0; k < K; ++k) dl0[k] = d[k];
            solve_row<real, K>(dl0, inv, f, cp, ls, W, lane, warp, nwl, wide, sA, sB, sC);
            // FP64 residual of the increment system at delta = dl0
            double xl = __shfl_up_sync(HEAT_FULL_MASK, (double)dl0[K - 1], 1, W);
            double xr = __shfl_down_sync(HEAT_FULL_MASK, (double)dl0[0], 1, W);
            if (wide) {
                __syncthreads();
                if (lane == 0) sLo[warp] = (double)dl0[0];
                if (lane == 31) sHi[warp] = (double)dl0[K - 1];
                __syncthreads();
                if (lane == 0) xl = warp > 0 ? sHi[warp - 1] : 0.0;
                if (lane == 31) xr = warp < nwl - 1 ? sLo[warp + 1] : 0.0;
            } else {
                if (ls == 0) xl = 0.0;
                if (ls == W - 1) xr = 0.0;
            }
            const double tl64 = (double)nbl;
            const double tr64 = (double)nbr;
            const size_t ro = (size_t)acls * Nr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                double rho = 0.0;
                if (valid && i < Nr) {
                    const size_t zo = (size_t)zc[k] * Nz + j;
                    const double t0 = (double)tc[k];
                    const double tl = k > 0 ? (double)tc[k - 1] : tl64;
                    const double tr = k < K - 1 ? (double)tc[k + 1] : tr64;
                    double r = R64.q[ro + i];
                    r = fma(R64.am[ro + i], tl - t0, r);
                    r = fma(R64.ap[ro + i], tr - t0, r);
                    r = fma(R64.dl[ro + i], bc.th[0] - t0, r);
                    r = fma(R64.dh[ro + i], bc.th[1] - t0, r);
                    r = fma(Z64.am[zo], (double)tmv[k] - t0, r);
                    r = fma(Z64.ap[zo], (double)tpv[k] - t0, r);
                    r = fma(Z64.dl[zo], bc.th[2] - t0, r);
                    r = fma(Z64.dh[zo], bc.th[3] - t0, r);
                    const double xm = k > 0 ? (double)dl0[k - 1] : xl;
                    const double xp = k < K - 1 ? (double)dl0[k + 1] : xr;
                    const double Ax = R64.b[ro + i] * (double)dl0[k] - R64.m[ro + i] * xm - R64.p[ro + i] * xp;
                    rho = r - Ax;
                }
                d[k] = (real)rho;
            }
            solve_row<real, K>(d, inv, f, cp, ls, W, lane, warp, nwl, wide, sA, sB, sC);
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = (real)((double)dl0[k] + (double)d[k]);
        } else {
            solve_row<real, K>(d, inv, f, cp, ls, W, lane, warp, nwl, wide, sA, sB, sC);
        }
        if constexpr (MODE != MODE_LIT) {
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = tc[k] + d[k];
        }
        if (valid) store_chunk<real, K>(out + (size_t)j * Nr, i0, Nr, vec, d);
        if constexpr (NRING > 0) fetch(j + NRING - 2);
    }
    cp_async_wait<0>();
}

// ------------------------------------------------------------------ z-sweep
// Right-hand side of the z-line system at (i, j) for a lane, given the column
// values tm, t, tp (rows j-1, j, j+1) and the row neighbours tl, tr.
template <typename real, int MODE>
__device__ __forceinline__ real z_rhs(real tm, real t, real tp, real tl, real tr, real e0, real e1, real e2, real ra,
                                      real rb, real rc, real rd, real zdl, real zdh, const real (&bcv)[4])
{
    if constexpr (MODE == MODE_LIT) {
        // e0 = w, e1 = s; ra, rb, rc, rd = R.am, R.ap, R.ad, R.sd
        return fmad(e0 + rc, t, fmad(ra, tl, fmad(rb, tr, e1 + rd)));
    } else {
        // e0 = Z.am, e1 = Z.ap, e2 = q; ra, rb, rc, rd = R.am, R.ap, R.dl, R.dh
        real r = e2;
        r = fmad(e0, tm - t, r);
        r = fmad(e1, tp - t, r);
        r = fmad(ra, tl - t, r);
        r = fmad(rb, tr - t, r);
        r = fmad(rc, bcv[0] - t, r);
        r = fmad(rd, bcv[1] - t, r);
        r = fmad(zdl, bcv[2] - t, r);
        r = fmad(zdh, bcv[3] - t, r);
        return r;
    }
}

template <typename real>
__device__ __forceinline__ void ld_pack(const real *p, real (&e)[8])
{
    if constexpr (sizeof(real) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(p + 4));
        e[0] = a.x, e[1] = a.y, e[2] = a.z, e[3] = a.w, e[4] = b.x, e[5] = b.y, e[6] = b.z, e[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(p + q));
            e[q] = a.x, e[q + 1] = a.y;
        }
    }
}

// Per-thread context of the z kernels: the thread's column, rows and the
// right-hand side of its rows (computed from the field, or read from rho).
template <typename real, int KZ>
struct ZThread {
    int i, j0, j1, b;
    bool col;
    real d[KZ];
    real t[KZ];
};

template <typename real, int KZ, int MODE>
__device__ __forceinline__ void z_load_rhs(ZThread<real, KZ> &T, const real *__restrict__ th,
                                           const real *__restrict__ rho, int Nr, int Nz,
                                           const int *__restrict__ rowcls, const real *__restrict__ pkb,
                                           LineTab<real> R, LineTab<real> Z, const real (&bcv)[4], int lane)
{
    const int i = T.i;
    const bool col = T.col;
    if constexpr (MODE == MODE_CORR) {
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int j = T.j0 + k;
            T.d[k] = (col && j < T.j1) ? rho[(size_t)j * Nr + i] : real(0);
            T.t[k] = real(0);
        }
        return;
    }
    int acur = -1;
    real ra = real(0), rb = real(0), rc = real(0), rd = real(0);
    real tprev = (col && T.j0 - 1 >= 0 && T.j0 - 1 < Nz) ? th[(size_t)(T.j0 - 1) * Nr + i] : real(0);
    real tcur = (col && T.j0 < Nz) ? th[(size_t)T.j0 * Nr + i] : real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = T.j0 + k;
        const bool vr = j < T.j1;
        const real tnext = (col && j + 1 < Nz) ? th[(size_t)(j + 1) * Nr + i] : real(0);
        const int a = vr ? rowcls[j] : acur;
        if (a != acur && vr) {
            if (col) {
                const size_t ro = (size_t)a * Nr + i;
                ra = R.am[ro];
                rb = R.ap[ro];
                if constexpr (MODE == MODE_LIT) {
                    rc = R.ad[ro];
                    rd = R.sd[ro];
                } else {
                    rc = R.dl[ro];
                    rd = R.dh[ro];
                }
            }
            acur = a;
        }
        real tl = __shfl_up_sync(HEAT_FULL_MASK, tcur, 1);
        real tr = __shfl_down_sync(HEAT_FULL_MASK, tcur, 1);
        if (lane == 0) tl = (col && i > 0 && vr) ? th[(size_t)j * Nr + i - 1] : tcur;
        if (lane == 31) tr = (i + 1 < Nr && vr) ? th[(size_t)j * Nr + i + 1] : tcur;
        real dd = real(0);
        if (col && vr) {
            real e[8];
            ld_pack(pkb + (size_t)j * 8, e);
            real zdl = real(0), zdh = real(0);
            if (MODE != MODE_LIT && (j == 0 || j == Nz - 1)) {
                zdl = Z.dl[(size_t)T.b * Nz + j];
                zdh = Z.dh[(size_t)T.b * Nz + j];
            }
            dd = z_rhs<real, MODE>(tprev, tcur, tnext, tl, tr, e[5], e[6], e[7], ra, rb, rc, rd, zdl, zdh, bcv);
        }
        T.d[k] = dd;
        T.t[k] = tcur;
        tprev = tcur;
        tcur = tnext;
    }
}

// Pass 1: chunk summaries B = sum r wB, G0 = sum r wG per column.
// Grid (strips, chunks); block 32 x NW; summaries written to zsum[c][0|1][i].
template <typename real, int KZ, int MODE>
__global__ void __launch_bounds__(512, 2) zsum_kernel(const real *__restrict__ th, const real *__restrict__ rho, int Nr,
                                                   int Nz, int Rc, const int *__restrict__ rowcls,
                                                   const int *__restrict__ colcls, const real *__restrict__ pk,
                                                   LineTab<real> R, LineTab<real> Z, BcVals bc,
                                                   real *__restrict__ zsum)
{
    __shared__ real sBs[16][33], sGs[16][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int c = blockIdx.y;
    ZThread<real, KZ> T;
    T.i = blockIdx.x * 32 + lane;
    T.col = T.i < Nr;
    T.b = T.col ? colcls[T.i] : 0;
    const int r0 = c * Rc, r1 = min(Nz, r0 + Rc);
    T.j0 = min(r0 + w * KZ, r1);
    T.j1 = min(T.j0 + KZ, r1);
    const real bcv[4] = {(real)bc.th[0], (real)bc.th[1], (real)bc.th[2], (real)bc.th[3]};
    const real *pkb = pk + (size_t)T.b * Nz * 8;
    z_load_rhs<real, KZ, MODE>(T, th, rho, Nr, Nz, rowcls, pkb, R, Z, bcv, lane);
    real sb = real(0), sg = real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = T.j0 + k;
        if (T.col && j < T.j1) {
            sb = fmad(T.d[k], pkb[(size_t)j * 8 + 3], sb);
            sg = fmad(T.d[k], pkb[(size_t)j * 8 + 4], sg);
        }
    }
    sBs[w][lane] = sb;
    sGs[w][lane] = sg;
    __syncthreads();
    if (w == 0 && T.col) {
        real B = real(0), Gs = real(0);
        for (int v = 0; v < NW; ++v) {
            B += sBs[v][lane];
            Gs += sGs[v][lane];
        }
        zsum[((size_t)c * 2) * Nr + T.i] = B;
        zsum[((size_t)c * 2 + 1) * Nr + T.i] = Gs;
    }
}

// Pass 2: carries of this chunk from all chunk summaries of the column, then
// the chunk solve (in-block carry scans over warps).
template <typename real, int KZ, int MODE>
__global__ void __launch_bounds__(512, 2) zsolve_kernel(const real *__restrict__ th, real *__restrict__ out,
                                                     real *__restrict__ rho_out, const real *__restrict__ rho_in,
                                                     int Nr, int Nz, int Rc, int nch, const int *__restrict__ rowcls,
                                                     const int *__restrict__ colcls, const real *__restrict__ pk,
                                                     const real *__restrict__ chk, LineTab<real> R, LineTab<real> Z,
                                                     LineTab64 R64, LineTab64 Z64, BcVals bc,
                                                     const real *__restrict__ zsum)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *Dsm = reinterpret_cast<real *>(smem_raw);  // [nch][32]: D_{c'-1} per column
    __shared__ real sF[16][33], sB[16][33], sEF[16][33], sEB[16][33];
    __shared__ real cinS[32], xinS[32];
    __shared__ double dLo[16][33], dHi[16][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int c = blockIdx.y;
    ZThread<real, KZ> T;
    T.i = blockIdx.x * 32 + lane;
    T.col = T.i < Nr;
    T.b = T.col ? colcls[T.i] : 0;
    const int r0 = c * Rc, r1 = min(Nz, r0 + Rc);
    T.j0 = min(r0 + w * KZ, r1);
    T.j1 = min(T.j0 + KZ, r1);
    const real bcv[4] = {(real)bc.th[0], (real)bc.th[1], (real)bc.th[2], (real)bc.th[3]};
    const real *pkb = pk + (size_t)T.b * Nz * 8;
    const real *chb = chk + (size_t)T.b * nch * 4;

    // carries into / out of this chunk, per column (warp 0)
    if (w == 0) {
        real D = real(0), X = real(0);
        if (T.col) {
            for (int cc = 0; cc < nch; ++cc) {
                Dsm[cc * 32 + lane] = D;
                if (cc < nch - 1) D = fmad(chb[cc * 4 + 0], D, zsum[((size_t)cc * 2) * Nr + T.i]);
            }
            for (int cc = nch - 1; cc > c; --cc)
                X = fmad(chb[cc * 4 + 1], X,
                         fmad(chb[cc * 4 + 2], Dsm[cc * 32 + lane], zsum[((size_t)cc * 2 + 1) * Nr + T.i]));
        }
        cinS[lane] = T.col ? Dsm[c * 32 + lane] : real(0);
        xinS[lane] = X;
    }
    z_load_rhs<real, KZ, MODE>(T, th, rho_in, Nr, Nz, rowcls, pkb, R, Z, bcv, lane);

    // forward local
    real F = real(1), B = real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = T.j0 + k;
        real iv = real(0), ff = real(0);
        if (T.col && j < T.j1) {
            iv = pkb[(size_t)j * 8 + 0];
            ff = pkb[(size_t)j * 8 + 1];
        }
        B = fmad(T.d[k], iv, ff * B);
        F *= ff;
    }
    sF[w][lane] = F;
    sB[w][lane] = B;
    __syncthreads();
    // exclusive scan over warps, one column per (warp, pass): lane p holds warp p's map
    for (int cc = w; cc < 32; cc += NW) {
        real f2 = lane < NW ? sF[lane][cc] : real(1), b2 = lane < NW ? sB[lane][cc] : real(0), fe, be;
        seg_scan_fwd(f2, b2, fe, be, lane, 32);
        if (lane < NW) {
            sEF[lane][cc] = fe;
            sEB[lane][cc] = be;
        }
    }
    __syncthreads();
    real dp = fmad(sEF[w][lane], cinS[lane], sEB[w][lane]);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = T.j0 + k;
        real iv = real(0), ff = real(0);
        if (T.col && j < T.j1) {
            iv = pkb[(size_t)j * 8 + 0];
            ff = pkb[(size_t)j * 8 + 1];
        }
        dp = fmad(T.d[k], iv, ff * dp);
        T.d[k] = dp;
    }
    real H = real(1), Gm = real(0);
#pragma unroll
    for (int k = KZ - 1; k >= 0; --k) {
        const int j = T.j0 + k;
        const real cc = (T.col && j < T.j1) ? pkb[(size_t)j * 8 + 2] : real(0);
        Gm = fmad(cc, Gm, T.d[k]);
        H *= cc;
    }
    __syncthreads();
    sF[w][lane] = H;
    sB[w][lane] = Gm;
    __syncthreads();
    for (int cc = w; cc < 32; cc += NW) {
        real h2 = lane < NW ? sF[lane][cc] : real(1), g2 = lane < NW ? sB[lane][cc] : real(0), he, ge;
        seg_scan_bwd(h2, g2, he, ge, lane, 32);
        if (lane < NW) {
            sEF[lane][cc] = he;
            sEB[lane][cc] = ge;
        }
    }
    __syncthreads();
    real x = fmad(sEF[w][lane], xinS[lane], sEB[w][lane]);
#pragma unroll
    for (int k = KZ - 1; k >= 0; --k) {
        const int j = T.j0 + k;
        const real cc = (T.col && j < T.j1) ? pkb[(size_t)j * 8 + 2] : real(0);
        x = fmad(cc, x, T.d[k]);
        T.d[k] = x;
    }

    if constexpr (MODE == MODE_REFINE) {
        // FP64 residual of the increment system at the FP32 solution; the
        // neighbours of the chunk ends come from the adjacent warps, or from
        // the carries at the block's chunk ends:
        //   x_{r0-1} = D_{c-1} + cp_{r0-1} x_{r0},   x_{r1} = X_{c+1}.
        dLo[w][lane] = (double)T.d[0];
        dHi[w][lane] = (double)T.d[KZ - 1];
        __syncthreads();
        double xm_end = 0.0, xp_end = 0.0;
        const int i = T.i;
        if (T.col) {
            if (w > 0) {
                xm_end = dHi[w - 1][lane];
            } else if (r0 > 0) {
                xm_end = (double)cinS[lane] + (double)pkb[(size_t)(r0 - 1) * 8 + 2] * (double)T.d[0];
            }
            if (T.j1 < r1) {
                xp_end = dLo[w + 1][lane];
            } else if (r1 < Nz) {
                xp_end = (double)xinS[lane];
            }
        }
        int a64 = -1;
        double A0 = 0, A1 = 0, A2 = 0, A3 = 0;
        double tprev = (T.col && T.j0 - 1 >= 0 && T.j0 - 1 < Nz) ? (double)th[(size_t)(T.j0 - 1) * Nr + i] : 0.0;
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int j = T.j0 + k;
            const bool vr = j < T.j1;
            const double tcur = (double)T.t[k];
            const double tnext = (T.col && j + 1 < Nz) ? (double)th[(size_t)(j + 1) * Nr + i] : 0.0;
            const int a = vr ? rowcls[j] : a64;
            if (a != a64 && vr) {
                if (T.col) {
                    const size_t ro = (size_t)a * Nr + i;
                    A0 = R64.am[ro];
                    A1 = R64.ap[ro];
                    A2 = R64.dl[ro];
                    A3 = R64.dh[ro];
                }
                a64 = a;
            }
            double tl = __shfl_up_sync(HEAT_FULL_MASK, tcur, 1);
            double tr = __shfl_down_sync(HEAT_FULL_MASK, tcur, 1);
            if (lane == 0) tl = (T.col && i > 0 && vr) ? (double)th[(size_t)j * Nr + i - 1] : tcur;
            if (lane == 31) tr = (i + 1 < Nr && vr) ? (double)th[(size_t)j * Nr + i + 1] : tcur;
            if (T.col && vr) {
                const size_t zj = (size_t)T.b * Nz + j;
                double r = Z64.q[zj];
                r = fma(Z64.am[zj], tprev - tcur, r);
                r = fma(Z64.ap[zj], tnext - tcur, r);
                r = fma(Z64.dl[zj], bc.th[2] - tcur, r);
                r = fma(Z64.dh[zj], bc.th[3] - tcur, r);
                r = fma(A0, tl - tcur, r);
                r = fma(A1, tr - tcur, r);
                r = fma(A2, bc.th[0] - tcur, r);
                r = fma(A3, bc.th[1] - tcur, r);
                const double xm = k > 0 ? (double)T.d[k - 1] : xm_end;
                const double xp = k < KZ - 1 ? (double)T.d[k + 1] : xp_end;
                const double rr = r - (Z64.b[zj] * (double)T.d[k] - Z64.m[zj] * xm - Z64.p[zj] * xp);
                rho_out[(size_t)j * Nr + i] = (real)rr;
            }
            tprev = tcur;
        }
    }
    if (T.col) {
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int j = T.j0 + k;
            if (j < T.j1) {
                const size_t c2 = (size_t)j * Nr + T.i;
                if constexpr (MODE == MODE_LIT)
                    out[c2] = T.d[k];
                else if constexpr (MODE == MODE_CORR)
                    out[c2] = out[c2] + T.d[k];
                else
                    out[c2] = T.t[k] + T.d[k];
            }
        }
    }
}

// ------------------------------------------------------------- reductions
// FP64 energy and boundary flux of theta, one partial pair per block, rows
// block-strided; fixed reduction order (bitwise reproducible).
template <typename real>
__global__ void __launch_bounds__(256) energy_kernel(const real *__restrict__ th, int Nr, int Nz,
                                                     const int *__restrict__ rowcls, const int *__restrict__ colcls,
                                                     LineTab64 R, LineTab64 Z, const double *__restrict__ wr,
                                                     const double *__restrict__ wz, double *__restrict__ part)
{
    __shared__ double se[256], sf[256];
    double e = 0.0, f = 0.0;
    for (int j = blockIdx.x; j < Nz; j += gridDim.x) {
        const size_t ro = (size_t)rowcls[j] * Nr;
        for (int i = threadIdx.x; i < Nr; i += blockDim.x) {
            const size_t zo = (size_t)colcls[i] * Nz + j;
            const double t = (double)th[(size_t)j * Nr + i];
            const double wgt = wr[i] * wz[j];
            e = fma(wgt * Z.cap[zo], t, e);
            f = fma(wgt, (R.dbc[ro + i] - R.dsum[ro + i] * t) + (Z.dbc[zo] - Z.dsum[zo] * t), f);
        }
    }
    se[threadIdx.x] = e;
    sf[threadIdx.x] = f;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sf[threadIdx.x] += sf[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = se[0];
        part[2 * blockIdx.x + 1] = sf[0];
    }
}

static __global__ void __launch_bounds__(256) energy_final_kernel(const double *__restrict__ part, int n,
                                                           double *__restrict__ res)
{
    __shared__ double se[256], sf[256];
    double e = 0.0, f = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        e += part[2 * b];
        f += part[2 * b + 1];
    }
    se[threadIdx.x] = e;
    sf[threadIdx.x] = f;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sf[threadIdx.x] += sf[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        res[0] = se[0];
        res[1] = sf[0];
    }
}

// ------------------------------------------------------------- conversions
template <typename real>
__global__ void theta_to_T_kernel(const real *__restrict__ th, double *__restrict__ T, size_t n, double Tref)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        T[c] = (double)th[c] + Tref;
}

template <typename real>
__global__ void T_to_theta_kernel(const double *__restrict__ T, real *__restrict__ th, size_t n, double Tref)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        th[c] = (real)(T[c] - Tref);
}

template <typename real>
__global__ void fill_kernel(real *__restrict__ th, size_t n, real v)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        th[c] = v;
}

// ------------------------------------------------------------- launchers
constexpr int kSMs = 152;

static int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

static BcVals bc_vals(const heat_ctx *ctx)
{
    BcVals b;
    for (int f = 0; f < 4; ++f) b.th[f] = ctx->theta_bc[f];
    return b;
}

template <typename real>
struct ZBufs;
template <>
struct ZBufs<float> {
    static const float *pk(const heat_ctx *c) { return c->zp.pk32; }
    static const float *ch(const heat_ctx *c) { return c->zp.ch32; }
    static float *sum(const heat_ctx *c) { return c->d_zsum; }
};
template <>
struct ZBufs<double> {
    static const double *pk(const heat_ctx *c) { return c->zp.pk64; }
    static const double *ch(const heat_ctx *c) { return c->zp.ch64; }
    static double *sum(const heat_ctx *c) { return c->d_zsum64; }
};

template <typename real, int K, int MODE>
static cudaError_t rsweep_k(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                            const LineTab<real> &Z)
{
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    const int G = next_pow2((Nr + K - 1) / K);
    const int block = G <= 32 ? 128 : G;
    const int lpb = block / G;
    // deepest ring that fits: 8 rows, else 4, else direct loads
    const size_t row_bytes = (size_t)lpb * G * K * sizeof(real);
    const size_t budget = 200 * 1024;
    const int nring = 8 * row_bytes <= budget ? 8 : (4 * row_bytes <= budget ? 4 : 0);
    const size_t smem = nring * row_bytes;
    int per_sm = smem ? (int)(budget / (smem + 4096)) : 4;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    const int slots_wanted = kSMs * per_sm * lpb;
    const int slots = Nz < slots_wanted ? Nz : slots_wanted;
    const int band = (Nz + slots - 1) / slots;
    const int grid = ((Nz + band - 1) / band + lpb - 1) / lpb;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, block, smem, ctx->stream>>>(in, out, Nr, Nz, G, band, ctx->d_rowcls, ctx->d_colcls, R, Z,
                                                 ctx->dR.full, ctx->dZ.full, bc_vals(ctx));
        return cudaGetLastError();
    };
    if (block <= 256) {
        if (nring == 8) return go(rsweep_kernel<real, K, MODE, 256, 8>);
        if (nring == 4) return go(rsweep_kernel<real, K, MODE, 256, 4>);
        return go(rsweep_kernel<real, K, MODE, 256, 0>);
    }
    if (nring == 8) return go(rsweep_kernel<real, K, MODE, 1024, 8>);
    if (nring == 4) return go(rsweep_kernel<real, K, MODE, 1024, 4>);
    return go(rsweep_kernel<real, K, MODE, 1024, 0>);
}

template <typename real, int MODE>
static cudaError_t launch_rsweep(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                                 const LineTab<real> &Z)
{
    const int Nr = ctx->g.Nr;
    if (sizeof(real) == 8 && Nr <= 1024) return rsweep_k<real, 4, MODE>(ctx, in, out, R, Z);
    if (Nr <= 8192) return rsweep_k<real, 8, MODE>(ctx, in, out, R, Z);
    if (Nr <= 16384) return rsweep_k<real, 16, MODE>(ctx, in, out, R, Z);
    return rsweep_k<real, 32, MODE>(ctx, in, out, R, Z);
}

template <typename real, int KZ, int MODE>
static cudaError_t zsweep_pass(const heat_ctx *ctx, const real *in, real *out, real *rho_out, const real *rho_in,
                               const LineTab<real> &R, const LineTab<real> &Z)
{
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    const int Rc = ctx->zp.Rc, nch = ctx->zp.n_chunks;
    const int NW = Rc / KZ;
    const dim3 grid((Nr + 31) / 32, nch, 1);
    const dim3 block(32 * NW, 1, 1);
    real *zs = ZBufs<real>::sum(ctx);
    zsum_kernel<real, KZ, MODE><<<grid, block, 0, ctx->stream>>>(in, rho_in, Nr, Nz, Rc, ctx->d_rowcls,
                                                                 ctx->d_colcls, ZBufs<real>::pk(ctx), R, Z,
                                                                 bc_vals(ctx), zs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)nch * 32 * sizeof(real);
    auto kern = zsolve_kernel<real, KZ, MODE>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    kern<<<grid, block, smem, ctx->stream>>>(in, out, rho_out, rho_in, Nr, Nz, Rc, nch, ctx->d_rowcls, ctx->d_colcls,
                                             ZBufs<real>::pk(ctx), ZBufs<real>::ch(ctx), R, Z, ctx->dR.full,
                                             ctx->dZ.full, bc_vals(ctx), zs);
    return cudaGetLastError();
}

template <typename real, int MODE>
static cudaError_t launch_zsweep(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                                 const LineTab<real> &Z)
{
    if constexpr (sizeof(real) == 8) {
        return zsweep_pass<real, 8, MODE>(ctx, in, out, nullptr, nullptr, R, Z);
    } else if constexpr (MODE == MODE_REFINE) {
        cudaError_t e = zsweep_pass<real, 16, MODE_REFINE>(ctx, in, out, ctx->d_rho, nullptr, R, Z);
        if (e != cudaSuccess) return e;
        return zsweep_pass<real, 16, MODE_CORR>(ctx, in, out, nullptr, ctx->d_rho, R, Z);
    } else {
        return zsweep_pass<real, 16, MODE>(ctx, in, out, nullptr, nullptr, R, Z);
    }
}
template <typename real, int MODE>
static cudaError_t sweep_mode(heat_ctx *ctx, int dir, const real *a, real *b, const LineTab<real> &R,
                              const LineTab<real> &Z)
{
    return dir == 0 ? launch_rsweep<real, MODE>(ctx, a, b, R, Z) : launch_zsweep<real, MODE>(ctx, a, b, R, Z);
}

// Per-form entry points, each compiled in its own translation unit.
cudaError_t sweep_fp64(heat_ctx *ctx, int dir, const void *a, void *b);
cudaError_t sweep_fp32(heat_ctx *ctx, int dir, const void *a, void *b);
cudaError_t sweep_fp32_refined(heat_ctx *ctx, int dir, const void *a, void *b);

}  // namespace heat
