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
// system is formed in extended precision (FP32 pairs, about 44 bits) from the
// FP64 coefficients and one more FP32 solve corrects delta (one step of
// mixed-precision iterative refinement).
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

__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---- extended precision from FP32 pairs (the refined path's residual).
// A value is carried as hi + lo, two FP32 numbers.  Sums and products use the
// error-free transformations TwoSum (Knuth: s + e = a + b exactly) and
// TwoProduct (one FMA: p + e = a b exactly), so the residual of a line
// system -- a sum of about ten terms that cancel to a small remainder -- keeps
// about 44 significant bits, far more than the one FP32 correction needs.
// GB300's FP64 units retire two FMAs per clock per SM against 128 FP32 ones;
// the ~17 FP32 operations a term costs here are a tenth of the FP64 time.
// The _rn intrinsics keep the compiler from fusing or reordering them.
struct Pair {
    float hi, lo;
};
__device__ __forceinline__ Pair two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// acc += c x, c = (c.x, c.y) a pair, x an FP32 value
__device__ __forceinline__ void pair_add_cx(Pair &acc, float2 c, float x)
{
    const float p = __fmul_rn(c.x, x);
    const float small = __fmaf_rn(c.y, x, __fmaf_rn(c.x, x, -p));
    const Pair t = two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, small));
}
// acc += c (u - v), the difference of two FP32 values taken exactly
__device__ __forceinline__ void pair_add_cdiff(Pair &acc, float2 c, float u, float v)
{
    const Pair d = two_sum(u, -v);
    const float p = __fmul_rn(c.x, d.hi);
    const float small = __fmaf_rn(c.x, d.lo, __fmaf_rn(c.y, d.hi, __fmaf_rn(c.x, d.hi, -p)));
    const Pair t = two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, small));
}

}  // namespace heat

#include "heat_rline.cuh"
#include "heat_rblock.cuh"
#include "heat_rwalk.cuh"
#include "heat_rclus.cuh"
#include "heat_zline.cuh"

namespace heat {

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
__global__ void __launch_bounds__(LB, LB <= 256 ? 3 : 1) rsweep_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    pdl_launch_dependents();
    pdl_wait();
    const SweepArgs<real> &A = args[blockIdx.y];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    const int Nr = A.Nr, Nz = A.Nz, G = A.G, band = A.band;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;
    const LineTab<real> &R = A.R, &Z = A.Z;
    const BcVals bc = A.bc;
    if ((int)blockIdx.x * (int)(blockDim.x / G) * band >= Nz) return;  // past this instance (block-uniform)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ real sA[32], sB[32], sC[32];
    __shared__ real sLo[32], sHi[32];
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
            static_assert(sizeof(real) == 4, "the refined path is FP32");
            real dl0[K];
#pragma unroll
            for (int k = 0; k < K; ++k) dl0[k] = d[k];
            solve_row<real, K>(dl0, inv, f, cp, ls, W, lane, warp, nwl, wide, sA, sB, sC);
            // residual of the increment system at delta = dl0, from the FP64
            // coefficients (as FP32 pairs) with exact differences and products
            real xl = __shfl_up_sync(HEAT_FULL_MASK, dl0[K - 1], 1, W);
            real xr = __shfl_down_sync(HEAT_FULL_MASK, dl0[0], 1, W);
            if (wide) {
                __syncthreads();
                if (lane == 0) sLo[warp] = dl0[0];
                if (lane == 31) sHi[warp] = dl0[K - 1];
                __syncthreads();
                if (lane == 0) xl = warp > 0 ? sHi[warp - 1] : real(0);
                if (lane == 31) xr = warp < nwl - 1 ? sLo[warp + 1] : real(0);
            } else {
                if (ls == 0) xl = real(0);
                if (ls == W - 1) xr = real(0);
            }
            const LineTab2 &R2 = A.R2, &Z2 = A.Z2;
            const size_t ro = (size_t)acls * Nr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                real rho = real(0);
                if (valid && i < Nr) {
                    const size_t zo = (size_t)zc[k] * Nz + j;
                    const real t0 = tc[k];
                    const real tl = k > 0 ? tc[k - 1] : nbl;
                    const real tr = k < K - 1 ? tc[k + 1] : nbr;
                    const float2 q2 = R2.q[ro + i];
                    Pair acc{q2.x, q2.y};
                    pair_add_cdiff(acc, R2.am[ro + i], tl, t0);
                    pair_add_cdiff(acc, R2.ap[ro + i], tr, t0);
                    if (i == 0) pair_add_cdiff(acc, R2.dl[ro + i], bc0, t0);
                    if (i == Nr - 1) pair_add_cdiff(acc, R2.dh[ro + i], bc1, t0);
                    pair_add_cdiff(acc, Z2.am[zo], tmv[k], t0);
                    pair_add_cdiff(acc, Z2.ap[zo], tpv[k], t0);
                    if (j == 0) pair_add_cdiff(acc, Z2.dl[zo], bc2, t0);
                    if (j == Nz - 1) pair_add_cdiff(acc, Z2.dh[zo], bc3, t0);
                    const real xm = k > 0 ? dl0[k - 1] : xl;
                    const real xp = k < K - 1 ? dl0[k + 1] : xr;
                    pair_add_cx(acc, R2.b[ro + i], -dl0[k]);
                    pair_add_cx(acc, R2.m[ro + i], xm);
                    pair_add_cx(acc, R2.p[ro + i], xp);
                    rho = __fadd_rn(acc.hi, acc.lo);
                }
                d[k] = rho;
            }
            solve_row<real, K>(d, inv, f, cp, ls, W, lane, warp, nwl, wide, sA, sB, sC);
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = dl0[k] + d[k];
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
// Interleaved Thomas inside column chunks.  A warp owns 32*V adjacent columns
// (V per lane: one 16-byte segment of a row, so every row access of the warp
// is one contiguous run) and one chunk of Rc rows; each lane walks its chunk
// row by row.  Pass 1 (zsum) reduces every (column, chunk) to its two carry
// summaries; pass 2 (zcarry) runs the carry recurrences of each column over
// its chunks; pass 3 (zsolve) walks each chunk forward from its carry
// (forward results in shared memory) and back from its other carry, writing
// the new field.  In the increment form every outer Dirichlet face is folded
// into the coupling of the boundary cell (xm, xp tables) and the ghost
// neighbour holds theta_bc, so the right-hand side needs no boundary branch.

template <typename real, int V>
struct VecIO;
template <>
struct VecIO<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float (&v)[4])
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct VecIO<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, double (&v)[2])
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x, v[1] = t.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&v)[2])
    {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};

// Four consecutive reals (aligned) from a read-only table.
template <typename real>
__device__ __forceinline__ void ld4(const real *p, real (&e)[4])
{
    if constexpr (sizeof(real) == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        e[0] = t.x, e[1] = t.y, e[2] = t.z, e[3] = t.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
        e[0] = a.x, e[1] = a.y, e[2] = b.x, e[3] = b.y;
    }
}

// Per-lane state of the z kernels, everything loop-invariant hoisted.
template <typename real, int V, int MODE>
struct ZLane {
    static constexpr bool LIT = MODE == MODE_LIT;
    const real *th;          // field base
    int Nr, Nz, ib, lane;
    bool any, vec, uni, lo_edge, hi_edge;
    int b[V];
    const real *pa[V], *pb[V];  // packed table rows of each column's class at row 0
    const real *stg;             // this warp's staged rows [Rc][8] of class bw (shared memory)
    int bw, jst;                 // staged class and first staged row
    bool allstg;                 // every column of the lane has class bw
    int acur;
    real ra[V], rb[V], rc[V], rd[V];  // increment: xm, xp; literal: am, ap, ad, sd
    real bz_lo, bz_hi, br_lo, br_hi;   // ghost values beyond the outer faces

    const real *pkA_base, *pkB_base;
    __device__ __forceinline__ void init(const real *th_, const int *__restrict__ colcls, const real *__restrict__ pkA,
                                         const real *__restrict__ pkB, int Nr_, int Nz_, int ib_, int lane_,
                                         const BcVals &bc)
    {
        th = th_, Nr = Nr_, Nz = Nz_, ib = ib_, lane = lane_;
        pkA_base = pkA, pkB_base = pkB;
        any = ib < Nr;
        vec = (Nr % V) == 0;
        lo_edge = ib == 0;
        hi_edge = ib < Nr && ib + V >= Nr;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            b[q] = ib + q < Nr ? colcls[ib + q] : (any ? colcls[ib] : 0);
            pa[q] = pkA + (size_t)b[q] * Nz * 4;
            pb[q] = pkB + (size_t)b[q] * Nz * 4;
        }
        uni = true;
#pragma unroll
        for (int q = 1; q < V; ++q) uni = uni && b[q] == b[0];
        acur = -1;
#pragma unroll
        for (int q = 0; q < V; ++q) ra[q] = rb[q] = rc[q] = rd[q] = real(0);
        // the literal form has zero couplings on the outer faces; the ghost
        // value then only has to be finite
        bz_lo = LIT ? real(0) : (real)bc.th[2];
        bz_hi = LIT ? real(0) : (real)bc.th[3];
        br_lo = LIT ? real(0) : (real)bc.th[0];
        br_hi = LIT ? real(0) : (real)bc.th[1];
    }
    __device__ __forceinline__ void row_class(int a, const LineTab<real> &R)
    {
        if (a == acur) return;
        acur = a;
        const size_t ro = (size_t)a * Nr;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int i = ib + q;
            const bool in = i < Nr;
            if constexpr (LIT) {
                ra[q] = in ? R.am[ro + i] : real(0);
                rb[q] = in ? R.ap[ro + i] : real(0);
                rc[q] = in ? R.ad[ro + i] : real(0);
                rd[q] = in ? R.sd[ro + i] : real(0);
            } else {
                ra[q] = in ? R.xm[ro + i] : real(0);
                rb[q] = in ? R.xp[ro + i] : real(0);
            }
        }
    }
    // row j of the lane's columns; ghost rows hold theta_bc
    __device__ __forceinline__ void row(const real *__restrict__ src, int j, real (&v)[V]) const
    {
        if (j < 0 || j >= Nz) {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = j < 0 ? bz_lo : bz_hi;
            return;
        }
        const real *p = src + (size_t)j * Nr + ib;
        if (vec) {
            if (any) VecIO<real, V>::ld(p, v);
            else
#pragma unroll
                for (int q = 0; q < V; ++q) v[q] = real(0);
        } else {
            // columns past the field sit right of the last column: they hold
            // its ghost value, which its folded coupling xp multiplies
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? p[q] : br_hi;
        }
    }
    // left / right neighbours of the lane's first / last column in row j
    __device__ __forceinline__ void halo(int j, const real (&t)[V], real &tl, real &tr) const
    {
        tl = __shfl_up_sync(HEAT_FULL_MASK, t[V - 1], 1);
        tr = __shfl_down_sync(HEAT_FULL_MASK, t[0], 1);
        if (lane == 0 && ib > 0 && ib - 1 < Nr) tl = th[(size_t)j * Nr + ib - 1];
        if (lane == 31 && ib + V < Nr) tr = th[(size_t)j * Nr + ib + V];
        if (lo_edge) tl = br_lo;
        if (hi_edge) tr = br_hi;
    }
    // Stage the warp's table rows [j0, j1) of class bw (lane 0's first column)
    // into shared memory: 8 reals per row (pkA then pkB).
    __device__ __forceinline__ void stage(real *buf, int j0, int j1)
    {
        bw = __shfl_sync(HEAT_FULL_MASK, b[0], 0);
        jst = j0;
        stg = buf;
        allstg = true;
#pragma unroll
        for (int q = 0; q < V; ++q) allstg = allstg && b[q] == bw;
        const real *A = pkA_base + (size_t)bw * Nz * 4, *B = pkB_base + (size_t)bw * Nz * 4;
        for (int e = lane; e < (j1 - j0) * 8; e += 32) {
            const int r = e >> 3, u = e & 7;
            buf[e] = u < 4 ? A[4 * (j0 + r) + u] : B[4 * (j0 + r) + u - 4];
        }
        __syncwarp();
    }
    // the staged 8 table values of row j (lanes with allstg)
    __device__ __forceinline__ void srow(int j, real (&e)[8]) const
    {
        const real *p = stg + (j - jst) * 8;
        if constexpr (sizeof(real) == 4) {
            const float4 a = *reinterpret_cast<const float4 *>(p), c = *reinterpret_cast<const float4 *>(p + 4);
            e[0] = a.x, e[1] = a.y, e[2] = a.z, e[3] = a.w, e[4] = c.x, e[5] = c.y, e[6] = c.z, e[7] = c.w;
        } else {
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const double2 a = *reinterpret_cast<const double2 *>(p + u);
                e[u] = a.x, e[u + 1] = a.y;
            }
        }
    }
    // entry u of table A / B of row j for column q
    __device__ __forceinline__ real tA(int q, int j, int u) const
    {
        return b[q] == bw ? stg[(j - jst) * 8 + u] : pa[q][4 * j + u];
    }
    __device__ __forceinline__ real tB(int q, int j, int u) const
    {
        return b[q] == bw ? stg[(j - jst) * 8 + 4 + u] : pb[q][4 * j + u];
    }
    // right-hand side of row j from rows j-1, j, j+1 and the row neighbours;
    // e[q][0..7] are the table values of column q (pkA then pkB)
    __device__ __forceinline__ void rhs(const real (&tm)[V], const real (&t)[V], const real (&tp)[V], real tl,
                                        real tr, const real (&e)[V][8], real (&d)[V]) const
    {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const real x = t[q];
            const real l = q > 0 ? t[q - 1] : tl;
            const real r = q < V - 1 ? t[q + 1] : tr;
            if constexpr (LIT) {
                // A[3] = s, B[0] = w
                d[q] = fmad(e[q][4] + rc[q], x, fmad(ra[q], l, fmad(rb[q], r, e[q][3] + rd[q])));
            } else {
                // A[3] = q, B[0] = xm (z), B[1] = xp (z)
                real v = fmad(e[q][4], tm[q] - x, e[q][3]);
                v = fmad(e[q][5], tp[q] - x, v);
                v = fmad(ra[q], l - x, v);
                d[q] = fmad(rb[q], r - x, v);
            }
        }
    }
    // table values of row j for every column: one staged row when the lane's
    // columns share the staged class, else per column
    __device__ __forceinline__ void trow(int j, real (&e)[V][8]) const
    {
        if (allstg) {
            real s8[8];
            srow(j, s8);
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int u = 0; u < 8; ++u) e[q][u] = s8[u];
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int u = 0; u < 4; ++u) e[q][u] = tA(q, j, u), e[q][4 + u] = tB(q, j, u);
        }
    }
};

// Walks rows [j0, j1), computing each row's right-hand side (or reading rho)
// and calling emit(j, d, eA, eB).  Rows are loaded ZP at a time (field rows,
// halo values and table rows of the whole group issued together) so that a
// lane has ZP rows of loads in flight.
constexpr int ZP = 4;

// Row pointer walk: rows are read through an incrementing pointer; the ghost
// row beyond the top face is substituted once at the end of the column.
template <typename real, int V, int MODE, typename Emit>
__device__ __forceinline__ void z_walk(ZLane<real, V, MODE> &L, const real *__restrict__ rho, int j0, int j1,
                                       int ucls, const int *__restrict__ rowcls, const LineTab<real> &R, Emit emit)
{
    const int Nr = L.Nr;
    const bool fast = L.vec && L.any;
    real tm[V], t[V];
    if constexpr (MODE != MODE_CORR) {
        L.row(L.th, j0 - 1, tm);
        L.row(L.th, j0, t);
        if (ucls >= 0) L.row_class(ucls, R);
    }
    // halo pointers: the neighbours left / right of the warp's columns
    const bool hasl = L.lane == 0 && L.ib > 0 && L.ib - 1 < Nr;
    const bool hasr = L.lane == 31 && L.ib + V < Nr;
    const real *src = MODE == MODE_CORR ? rho : L.th;
    const int lead = MODE == MODE_CORR ? 0 : 1;  // rows ahead of j that the walk needs
    const real *np = src + (size_t)(j0 + lead) * Nr + L.ib;
    const real *hlp = L.th + (size_t)j0 * Nr + L.ib - 1;
    const real *hrp = L.th + (size_t)j0 * Nr + L.ib + V;
    for (int jb = j0; jb < j1; jb += ZP) {
        real nx[ZP][V], hl[ZP], hr[ZP];
#pragma unroll
        for (int p = 0; p < ZP; ++p) {
            const int jn = jb + p + lead;  // row loaded into nx[p]
            const bool ok = jn < L.Nz && jb + p < j1;
            if (fast && ok) {
                VecIO<real, V>::ld(np, nx[p]);
            } else if (ok) {
#pragma unroll
                for (int q = 0; q < V; ++q) nx[p][q] = L.ib + q < Nr ? np[q] : L.br_hi;
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) nx[p][q] = L.bz_hi;
            }
            np += Nr;
            if constexpr (MODE != MODE_CORR) {
                hl[p] = (hasl && jb + p < j1) ? *hlp : real(0);
                hr[p] = (hasr && jb + p < j1) ? *hrp : real(0);
                hlp += Nr;
                hrp += Nr;
            }
        }
#pragma unroll
        for (int p = 0; p < ZP; ++p) {
            const int j = jb + p;
            if (j >= j1) break;
            real d[V], e[V][8];
            L.trow(j, e);
            if constexpr (MODE == MODE_CORR) {
#pragma unroll
                for (int q = 0; q < V; ++q) d[q] = nx[p][q];
            } else {
                real tl = __shfl_up_sync(HEAT_FULL_MASK, t[V - 1], 1);
                real tr = __shfl_down_sync(HEAT_FULL_MASK, t[0], 1);
                if (hasl) tl = hl[p];
                if (hasr) tr = hr[p];
                if (L.lo_edge) tl = L.br_lo;
                if (L.hi_edge) tr = L.br_hi;
                if (ucls < 0) L.row_class(rowcls[j], R);
                L.rhs(tm, t, nx[p], tl, tr, e, d);
#pragma unroll
                for (int q = 0; q < V; ++q) tm[q] = t[q], t[q] = nx[p][q];
            }
            emit(j, d, e);
        }
    }
}

// Pass 1: summaries B = sum r wB and G0 = sum r wG of every (column, chunk):
// zs[(c*2 + s)*Nr + i].  Grid (column groups / warps per block, chunks).
template <typename real, int V, int MODE>
__global__ void __launch_bounds__(128, 4) zsum_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    pdl_launch_dependents();
    pdl_wait();
    const SweepArgs<real> &A = args[blockIdx.z];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    const real *__restrict__ rho = MODE == MODE_CORR ? A.rho : nullptr;
    const int Nr = A.Nr, Nz = A.Nz, Rc = A.Rc;
    if ((int)blockIdx.y >= A.nch) return;
    const int *__restrict__ ucls = A.ucls;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;
    const real *__restrict__ pkA = A.pkA;
    const real *__restrict__ pkB = A.pkB;
    const LineTab<real> &R = A.R;
    const BcVals bc = A.bc;
    real *__restrict__ zs = A.zs;
    const int lane = threadIdx.x & 31;
    const int grp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (grp * 32 * V >= Nr) return;  // whole warp past the field (warp-uniform)
    const int c = blockIdx.y;
    const int j0 = c * Rc, j1 = min(Nz, j0 + Rc);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ZLane<real, V, MODE> L;
    L.init(th, colcls, pkA, pkB, Nr, Nz, grp * 32 * V + lane * V, lane, bc);
    L.stage(reinterpret_cast<real *>(smem_raw) + (size_t)(threadIdx.x >> 5) * Rc * 8, j0, j1);
    real sb[V], sg[V];
#pragma unroll
    for (int q = 0; q < V; ++q) sb[q] = sg[q] = real(0);
    z_walk<real, V, MODE>(L, rho, j0, j1, ucls[c], rowcls, R, [&](int, const real(&d)[V], const real(&e)[V][8]) {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            sb[q] = fmad(d[q], e[q][6], sb[q]);
            sg[q] = fmad(d[q], e[q][7], sg[q]);
        }
    });
    if (L.vec) {
        if (L.any) {
            VecIO<real, V>::st(zs + ((size_t)c * 2) * Nr + L.ib, sb);
            VecIO<real, V>::st(zs + ((size_t)c * 2 + 1) * Nr + L.ib, sg);
        }
    } else {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            if (L.ib + q < Nr) {
                zs[((size_t)c * 2) * Nr + L.ib + q] = sb[q];
                zs[((size_t)c * 2 + 1) * Nr + L.ib + q] = sg[q];
            }
        }
    }
}

// Pass 2: chunk carries.  A block of ZSEG warps serves 32 columns (lane =
// column: every access is coalesced); warp s runs the carry recurrences over
// chunks [s*m, (s+1)*m) and the segments are joined through shared memory
// (composition of the segments' affine maps).  Writes cin_c = D_{c-1} and
// xin_c = X_{c+1} to zc[(c*2 + 0|1)*Nr + i].
constexpr int ZSEG = 8;

template <typename real>
__global__ void __launch_bounds__(32 * ZSEG) zcarry_kernel(const SweepArgs<real> *__restrict__ args)
{
    pdl_launch_dependents();
    pdl_wait();
    const SweepArgs<real> &A = args[blockIdx.y];
    const int Nr = A.Nr, nch = A.nch;
    if ((int)blockIdx.x * 32 >= Nr) return;  // past this instance (block-uniform)
    const int *__restrict__ colcls = A.colcls;
    const real *__restrict__ chk = A.chk;
    const real *__restrict__ zs = A.zs;
    real *__restrict__ zc = A.zc;
    __shared__ real sF[ZSEG][32], sB[ZSEG][32];
    const int lane = threadIdx.x & 31, sgm = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const bool col = i < Nr;
    const real *chb = chk + (size_t)(col ? colcls[i] : 0) * nch * 4;
    const int m = (nch + ZSEG - 1) / ZSEG;
    const int c0 = min(sgm * m, nch), c1 = min(c0 + m, nch);
    const size_t st = (size_t)2 * Nr;
    // forward segment map
    real F = real(1), B = real(0);
    if (col)
        for (int c = c0; c < c1; ++c) {
            const real Fc = chb[c * 4];
            B = fmad(Fc, B, zs[c * st + i]);
            F *= Fc;
        }
    sF[sgm][lane] = F;
    sB[sgm][lane] = B;
    __syncthreads();
    real D = real(0);
    for (int v = 0; v < sgm; ++v) D = fmad(sF[v][lane], D, sB[v][lane]);
    if (col)
        for (int c = c0; c < c1; ++c) {
            zc[c * st + i] = D;
            D = fmad(chb[c * 4], D, zs[c * st + i]);
        }
    // backward segment map X_c = (G0_c + GP_c D_{c-1}) + H_c X_{c+1}
    real H = real(1), Gm = real(0);
    if (col)
        for (int c = c1 - 1; c >= c0; --c) {
            Gm = fmad(chb[c * 4 + 1], Gm, fmad(chb[c * 4 + 2], zc[c * st + i], zs[c * st + Nr + i]));
            H *= chb[c * 4 + 1];
        }
    __syncthreads();
    sF[sgm][lane] = H;
    sB[sgm][lane] = Gm;
    __syncthreads();
    real X = real(0);
    for (int v = ZSEG - 1; v > sgm; --v) X = fmad(sF[v][lane], X, sB[v][lane]);
    if (col)
        for (int c = c1 - 1; c >= c0; --c) {
            zc[c * st + Nr + i] = X;
            X = fmad(chb[c * 4 + 1], X, fmad(chb[c * 4 + 2], zc[c * st + i], zs[c * st + Nr + i]));
        }
}

// Pass 3: solve every (column, chunk) from its carries.  Shared memory holds
// the forward results of each warp: [warps][Rc][32*V] reals.
template <typename real, int V, int MODE>
__global__ void __launch_bounds__(64, 8) zsolve_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    pdl_launch_dependents();
    pdl_wait();
    const SweepArgs<real> &A = args[blockIdx.z];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    real *__restrict__ rho_out = MODE == MODE_REFINE ? A.rho : nullptr;
    const real *__restrict__ rho_in = MODE == MODE_CORR ? A.rho : nullptr;
    const int Nr = A.Nr, Nz = A.Nz, Rc = A.Rc;
    if ((int)blockIdx.y >= A.nch) return;
    const int *__restrict__ ucls = A.ucls;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;
    const real *__restrict__ pkA = A.pkA;
    const real *__restrict__ pkB = A.pkB;
    const LineTab<real> &R = A.R;
    const BcVals bc = A.bc;
    const real *__restrict__ zc = A.zc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int COLS = 32 * V;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = blockIdx.x * (blockDim.x >> 5) + w;
    if (grp * COLS >= Nr) return;  // whole warp past the field (warp-uniform)
    const int c = blockIdx.y;
    const int j0 = c * Rc, j1 = min(Nz, j0 + Rc);
    real *dsm = reinterpret_cast<real *>(smem_raw) + (size_t)w * Rc * (COLS + 8) + lane * V;
    ZLane<real, V, MODE> L;
    L.init(th, colcls, pkA, pkB, Nr, Nz, grp * COLS + lane * V, lane, bc);
    L.stage(reinterpret_cast<real *>(smem_raw) + (size_t)w * Rc * (COLS + 8) + (size_t)Rc * COLS, j0, j1);
    real dp[V], x[V], cin[V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const bool in = L.ib + q < Nr;
        cin[q] = in ? zc[((size_t)c * 2) * Nr + L.ib + q] : real(0);
        x[q] = in ? zc[((size_t)c * 2 + 1) * Nr + L.ib + q] : real(0);
        dp[q] = cin[q];
    }
    z_walk<real, V, MODE>(L, rho_in, j0, j1, ucls[c], rowcls, R, [&](int j, const real(&d)[V], const real(&e)[V][8]) {
#pragma unroll
        for (int q = 0; q < V; ++q) dp[q] = fmad(d[q], e[q][0], e[q][1] * dp[q]);
        VecIO<real, V>::st(dsm + (size_t)(j - j0) * COLS, dp);
    });
    // backward from the carry-out, writing the solution rows; the rows added
    // to the increments are loaded ZP at a time
    for (int jt = j1 - 1; jt >= j0; jt -= ZP) {
        real base[ZP][V];
        if constexpr (MODE != MODE_LIT) {
#pragma unroll
            for (int p = 0; p < ZP; ++p) {
                const int j = jt - p;
                L.row(MODE == MODE_CORR ? out : th, j >= j0 ? j : j0, base[p]);
            }
        }
#pragma unroll
        for (int p = 0; p < ZP; ++p) {
            const int j = jt - p;
            if (j < j0) break;
            real dd[V], cpv[V];
            {
                const real *ps = dsm + (size_t)(j - j0) * COLS;
#pragma unroll
                for (int q = 0; q < V; ++q) dd[q] = ps[q];
            }
            if (L.allstg) {
                const real c2 = L.stg[(j - L.jst) * 8 + 2];
#pragma unroll
                for (int q = 0; q < V; ++q) cpv[q] = c2;
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) cpv[q] = L.tA(q, j, 2);
            }
#pragma unroll
            for (int q = 0; q < V; ++q) x[q] = fmad(cpv[q], x[q], dd[q]);
            if constexpr (MODE == MODE_REFINE) VecIO<real, V>::st(dsm + (size_t)(j - j0) * COLS, x);
            if (!L.any) continue;
            real o[V];
#pragma unroll
            for (int q = 0; q < V; ++q) o[q] = MODE == MODE_LIT ? x[q] : base[p][q] + x[q];
            real *orow = out + (size_t)j * Nr + L.ib;
            if (L.vec) {
                VecIO<real, V>::st(orow, o);
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q)
                    if (L.ib + q < Nr) orow[q] = o[q];
            }
        }
    }

    if constexpr (MODE == MODE_REFINE) {
        static_assert(sizeof(real) == 4, "the refined path is FP32");
        // residual of the increment system at the FP32 solution x (now in
        // shared memory), from the FP64 coefficients as FP32 pairs with exact
        // differences and products; outside the chunk:
        // x_{j0-1} = D_{c-1} + cp_{j0-1} x_{j0} and x_{j1} = X_{c+1}.
        const LineTab2 &R2 = A.R2, &Z2 = A.Z2;
        const int ib = L.ib;
        real xlo[V], xhi[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const bool in = ib + q < Nr;
            const real x0 = dsm[q];
            xlo[q] = (j0 > 0 && in) ? fmad(L.pa[q][4 * (j0 - 1) + 2], x0, cin[q]) : real(0);
            xhi[q] = (j1 < Nz && in) ? zc[((size_t)c * 2 + 1) * Nr + ib + q] : real(0);
        }
        real tm[V], t[V], tp[V];
        L.row(th, j0 - 1, tm);
        L.row(th, j0, t);
        int a2 = -1;
        float2 A0[V], A1[V];
#pragma unroll
        for (int q = 0; q < V; ++q) A0[q] = A1[q] = make_float2(0.f, 0.f);
        for (int j = j0; j < j1; ++j) {
            L.row(th, j + 1, tp);
            real tl, tr;
            L.halo(j, t, tl, tr);
            const int a = rowcls[j];
            if (a != a2) {
                a2 = a;
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    const int i = ib + q;
                    const size_t ro = (size_t)a * Nr + i;
                    A0[q] = i < Nr ? (i == 0 ? R2.dl[ro] : R2.am[ro]) : make_float2(0.f, 0.f);
                    A1[q] = i < Nr ? (i == Nr - 1 ? R2.dh[ro] : R2.ap[ro]) : make_float2(0.f, 0.f);
                }
            }
            real rr[V];
            const real *xs = dsm + (size_t)(j - j0) * COLS;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const size_t zj = (size_t)L.b[q] * Nz + j;
                const real l = q > 0 ? t[q - 1] : tl;
                const real r = q < V - 1 ? t[q + 1] : tr;
                const float2 q2 = Z2.q[zj];
                Pair acc{q2.x, q2.y};
                pair_add_cdiff(acc, j == 0 ? Z2.dl[zj] : Z2.am[zj], tm[q], t[q]);
                pair_add_cdiff(acc, j == Nz - 1 ? Z2.dh[zj] : Z2.ap[zj], tp[q], t[q]);
                pair_add_cdiff(acc, A0[q], l, t[q]);
                pair_add_cdiff(acc, A1[q], r, t[q]);
                const real xm = j > j0 ? xs[q - COLS] : xlo[q];
                const real xp = j + 1 < j1 ? xs[q + COLS] : xhi[q];
                pair_add_cx(acc, Z2.b[zj], -xs[q]);
                pair_add_cx(acc, Z2.m[zj], xm);
                pair_add_cx(acc, Z2.p[zj], xp);
                rr[q] = __fadd_rn(acc.hi, acc.lo);
            }
            if (L.any) {
                real *row = rho_out + (size_t)j * Nr + ib;
                if (L.vec) {
                    VecIO<real, V>::st(row, rr);
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q)
                        if (ib + q < Nr) row[q] = rr[q];
                }
            }
#pragma unroll
            for (int q = 0; q < V; ++q) tm[q] = t[q], t[q] = tp[q];
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

// Cells per thread of the r-sweep for lines of up to Nr cells.
static int default_rK(int word, int Nr)
{
    if (word == 8 && Nr <= 1024) return 4;
    if (Nr <= 8192) return 8;
    if (Nr <= 16384) return 16;
    return 32;
}

static cudaError_t allow_smem(const void *fn, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    const int maxdyn = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in maximum
    if (smem > (size_t)maxdyn) return cudaErrorInvalidValue;
    // The attribute only raises a per-kernel ceiling; setting it to the device
    // maximum keeps every plan's launches valid whichever plan was made last.
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
}

// r-sweep launch for n instances, all sharing K: instance m runs in grid row
// blockIdx.y = m with G_m threads per line and lpb_m = block / G_m lines per
// block, each line slot walking band_m consecutive rows.  A batch (n > 1)
// keeps every line inside one warp (G <= 32), so the block size is uniform.
template <typename real, int K, int MODE>
static cudaError_t plan_rsweep_k(SweepArgs<real> *h, int n, int band_req, Launch &L)
{
    int Gmax = 1;
    for (int m = 0; m < n; ++m) {
        h[m].G = next_pow2((h[m].Nr + K - 1) / K);
        Gmax = h[m].G > Gmax ? h[m].G : Gmax;
    }
    if (n > 1 && Gmax > 32) return cudaErrorInvalidValue;
    if (Gmax > 1024) return cudaErrorInvalidValue;  // a line longer than one block of K-cell threads
    const int block = Gmax <= 32 ? 128 : Gmax;
    // deepest ring that fits: 8 rows, else 4, else direct loads
    const size_t row_bytes = (size_t)block * K * sizeof(real);
    const size_t budget = 200 * 1024;
    const int nring = 8 * row_bytes <= budget ? 8 : (4 * row_bytes <= budget ? 4 : 0);
    const size_t smem = nring * row_bytes;
    int per_sm = smem ? (int)(budget / (smem + 4096)) : 4;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    // rows per slot: the largest band (<= 64) that still gives two waves of
    // resident blocks over all instances, or one row per slot if none does
    auto blocks_for = [&](int band) {
        long long tot = 0;
        for (int m = 0; m < n; ++m) {
            const int lpb = block / h[m].G;
            tot += ((h[m].Nz + band - 1) / band + lpb - 1) / lpb;
        }
        return tot;
    };
    int band = band_req;
    if (band <= 0) {
        if (n == 1) {
            const int lpb = block / h[0].G;
            const int slots_wanted = kSMs * per_sm * lpb;
            const int slots = h[0].Nz < slots_wanted ? h[0].Nz : slots_wanted;
            band = (h[0].Nz + slots - 1) / slots;
        } else {
            band = 1;
            for (int b = 64; b > 1; b >>= 1)
                if (blocks_for(b) >= 2LL * kSMs * per_sm) { band = b; break; }
        }
    }
    int gx = 1;
    for (int m = 0; m < n; ++m) {
        h[m].band = band;
        const int lpb = block / h[m].G;
        const int bx = ((h[m].Nz + band - 1) / band + lpb - 1) / lpb;
        gx = bx > gx ? bx : gx;
    }
    const void *fn;
    if (block <= 256)
        fn = nring == 8 ? (const void *)rsweep_kernel<real, K, MODE, 256, 8>
                        : nring == 4 ? (const void *)rsweep_kernel<real, K, MODE, 256, 4>
                                     : (const void *)rsweep_kernel<real, K, MODE, 256, 0>;
    else
        fn = nring == 8 ? (const void *)rsweep_kernel<real, K, MODE, 1024, 8>
                        : nring == 4 ? (const void *)rsweep_kernel<real, K, MODE, 1024, 4>
                                     : (const void *)rsweep_kernel<real, K, MODE, 1024, 0>;
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    L.fn = fn;
    L.grid = dim3(gx, n, 1);
    L.block = dim3(block, 1, 1);
    L.smem = smem;
    L.flip = true;
    return cudaSuccess;
}

// Line-team r-sweep for n instances that all have their tables (rl.tA set).
// One instance: a persistent grid (every resident block slot, lines dealt in
// contiguous runs).  A batch: blockIdx.y = member, and enough blocks along x
// that the member with the most line teams' worth of rows gets `band` rows per
// team (default: the largest band that still fills two waves).
template <typename real, int MODE>
static cudaError_t plan_rline(SweepArgs<real> *h, int n, Tuning &tu, Launch &L)
{
    constexpr int K = rline_K<real>();
    constexpr int R = rline_rows(sizeof(real) == 8);
    const void *fn = (const void *)rline_kernel<real, K, R, MODE>;
    int maxseg = 1;
    for (int m = 0; m < n; ++m) {
        if (!h[m].rl.tA) return cudaErrorInvalidValue;
        maxseg = h[m].rl.nseg > maxseg ? h[m].rl.nseg : maxseg;
    }
    const size_t warp_buf = (size_t)32 * maxseg * K * R * sizeof(real);  // (32/LW) teams x R x Npad
    int NW = (int)((64 * 1024) / warp_buf);
    NW = NW < 1 ? 1 : (NW > 4 ? 4 : NW);
    const size_t smem = (size_t)NW * warp_buf;
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * NW, smem)) != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    auto teams_per_block = [&](int m) { return NW * (32 / h[m].rl.LW); };
    int gx = 1;
    if (n == 1) {
        const int U = h[0].rl.n_units;
        const int need = (U + teams_per_block(0) - 1) / teams_per_block(0);
        gx = kSMs * per_sm < need ? kSMs * per_sm : need;
        tu.band = (U + gx * teams_per_block(0) - 1) / (gx * teams_per_block(0));
    } else {
        auto blocks_for = [&](int band, long long *tot) {
            int mx = 1;
            *tot = 0;
            for (int m = 0; m < n; ++m) {
                const int U = h[m].rl.n_units;
                const int bx = (U + teams_per_block(m) * band - 1) / (teams_per_block(m) * band);
                *tot += bx;
                mx = bx > mx ? bx : mx;
            }
            return mx;
        };
        int band = tu.band;
        if (band <= 0) {
            band = 1;
            for (int b = 16; b > 1; b >>= 1) {
                long long tot;
                blocks_for(b, &tot);
                if (tot >= 2LL * kSMs * per_sm) { band = b; break; }
            }
        }
        long long tot;
        gx = blocks_for(band, &tot);
        tu.band = band;
    }
    for (int m = 0; m < n; ++m) h[m].band = tu.band, h[m].G = 32;
    tu.rK = 1;
    L.fn = fn;
    L.grid = dim3(gx, n, 1);
    L.block = dim3(32 * NW, 1, 1);
    L.smem = smem;
    L.flip = true;
    return cudaSuccess;
}

// Register-resident r-sweep (heat_rblock.cuh; FP32 increment form, K = 8
// cells per thread, lines of up to 2048 cells): G = the power of two >= Nr/8
// threads per line (at least 4), 256/G line slots per block, each slot walking
// `band` rows.  One instance: the band that fills every resident block slot
// once; a batch: the largest band that still gives two waves.
constexpr int kRBlockK = 8, kRBlockRing = 8;

static cudaError_t plan_rblock(SweepArgs<float> *h, int n, Tuning &tu, Launch &L)
{
    constexpr int K = kRBlockK;
    bool exact = true;  // every line fills its threads exactly, rows 16-byte aligned
    for (int m = 0; m < n; ++m) {
        if (h[m].Nr > 256 * K) return cudaErrorInvalidValue;
        int G = 4;
        while (G * K < h[m].Nr) G <<= 1;
        h[m].G = G;
        exact = exact && G * K == h[m].Nr && h[m].Nr % 4 == 0;
    }
    // a single instance reads its arguments from the by-value copy
    const void *fn = n == 1 ? (exact ? (const void *)rblock_kernel<K, kRBlockRing, true, true>
                                     : (const void *)rblock_kernel<K, kRBlockRing, false, true>)
                            : (exact ? (const void *)rblock_kernel<K, kRBlockRing, true, false>
                                     : (const void *)rblock_kernel<K, kRBlockRing, false, false>);
    const int block = 256;
    const size_t smem = (size_t)kRBlockRing * block * K * sizeof(float);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem)) != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    auto blocks_for = [&](int band, long long *tot) {
        int mx = 1;
        *tot = 0;
        for (int m = 0; m < n; ++m) {
            const int lpb = block / h[m].G;
            const int bx = ((h[m].Nz + band - 1) / band + lpb - 1) / lpb;
            *tot += bx;
            mx = bx > mx ? bx : mx;
        }
        return mx;
    };
    for (int m = 0; m < n; ++m) h[m].rb_runs = 0;
    // A single instance whose lines take whole warps splits every row-class
    // run into its own bands, so that no band changes class (a change costs
    // the slot a class load and up to two one-row passes, and the slowest
    // slot sets the launch's time): the smallest even band whose bands fit
    // in one wave of slots.
    if (n == 1 && h[0].G >= 32 && h[0].n_run > 0) {
        SweepArgs<float> &a = h[0];
        const int lpb = block / a.G;
        const long long avail = (long long)kSMs * per_sm * lpb;
        auto slots_for = [&](int b) {
            long long t = 0;
            for (int r = 0; r < a.n_run; ++r) t += (a.run_lo[r + 1] - a.run_lo[r] + b - 1) / b;
            return t;
        };
        int b = tu.band > 0 ? tu.band : 2;
        if (tu.band <= 0)
            while (slots_for(b) > avail) b += 2;
        a.band = b;
        a.run_slot[0] = 0;
        for (int r = 0; r < a.n_run; ++r)
            a.run_slot[r + 1] = a.run_slot[r] + (a.run_lo[r + 1] - a.run_lo[r] + b - 1) / b;
        a.rb_runs = 1;
        tu.band = b;
        tu.rK = 2;
        L.pargs.assign(1, 0);  // (the three-parameter kernel; filled at the end of the plan)
        L.fn = fn;
        L.grid = dim3((a.run_slot[a.n_run] + lpb - 1) / lpb, 1, 1);
        L.block = dim3(block, 1, 1);
        L.smem = smem;
        L.flip = true;
        return cudaSuccess;
    }
    int band = tu.band;
    if (band <= 0) {
        if (n == 1) {
            const int lpb = block / h[0].G;
            const long long slots = (long long)kSMs * per_sm * lpb;
            band = (int)((h[0].Nz + slots - 1) / slots);
            band = band < 2 ? 2 : band;
        } else {
            band = 2;
            for (int b = 64; b > 2; b >>= 1) {
                long long tot;
                blocks_for(b, &tot);
                if (tot >= 2LL * kSMs * per_sm) { band = b; break; }
            }
        }
    }
    long long tot;
    const int gx = blocks_for(band, &tot);
    for (int m = 0; m < n; ++m) h[m].band = band;
    tu.band = band;
    tu.rK = 2;
    L.fn = fn;
    L.grid = dim3(gx, n, 1);
    L.block = dim3(block, 1, 1);
    L.smem = smem;
    L.flip = true;
    L.pargs.assign(1, 0);
    return cudaSuccess;
}

// Walk r-sweep (heat_rwalk.cuh) for one FP32 instance with its tables
// built (rw_K > 0): a band of rows per block, a multiple of the block's 4
// rows, one block per SM.
template <int K>
static cudaError_t plan_rwalk_k(SweepArgs<float> *h, Tuning &tu, Launch &L)
{
    const void *fn = (const void *)rwalk_kernel<K>;
    const size_t smem = RwLayout<K>::bytes;
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * kRwWarps, smem)) != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int groups = (h[0].Nz + kRwWarps - 1) / kRwWarps;
    const int per_block = (groups + kSMs * per_sm - 1) / (kSMs * per_sm);
    h[0].band = per_block * kRwWarps;
    h[0].G = 32;
    tu.band = h[0].band;
    tu.rK = 3;
    L.fn = fn;
    L.grid = dim3((h[0].Nz + h[0].band - 1) / h[0].band, 1, 1);
    L.block = dim3(32 * kRwWarps, 1, 1);
    L.smem = smem;
    L.flip = true;
    return cudaSuccess;
}

static cudaError_t plan_rwalk(SweepArgs<float> *h, int n, Tuning &tu, Launch &L)
{
    if (n != 1 || h[0].rw_K == 0 || h[0].rw_tab == nullptr) return cudaErrorInvalidValue;
    switch (h[0].rw_K) {
    case 17: return plan_rwalk_k<17>(h, tu, L);
    case 33: return plan_rwalk_k<33>(h, tu, L);
    case 65: return plan_rwalk_k<65>(h, tu, L);
    default: return cudaErrorInvalidValue;
    }
}

// Cluster r-sweep (heat_rclus.cuh) for one FP32 instance in an increment
// form: CL = ceil(Nr / 2048) blocks per line (at most 8), bands of rows
// sized so that the clusters that fit on the device at once take one band
// each.
template <int MODE>
static cudaError_t plan_rclus(SweepArgs<float> *h, int n, Tuning &tu, Launch &L)
{
    if (n != 1) return cudaErrorInvalidValue;
    const int Nr = h[0].Nr, Nz = h[0].Nz;
    const int CL = (Nr + kRcSeg - 1) / kRcSeg;
    if (CL > kRcMaxCl) return cudaErrorInvalidValue;
    if (MODE == MODE_REFINE && h[0].R2.q == nullptr) return cudaErrorInvalidValue;
    const bool exact = Nr == CL * kRcSeg;
    const void *fn = exact ? (const void *)rclus_kernel<MODE, true> : (const void *)rclus_kernel<MODE, false>;
    const size_t smem = rc_smem_bytes<MODE>();
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int active = 0;
    if (CL > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CL, 1, 1);
        cfg.blockDim = dim3(kRcThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = (unsigned)CL;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        if ((e = cudaOccupancyMaxActiveClusters(&active, fn, &cfg)) != cudaSuccess) return e;
    } else {
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRcThreads, smem)) != cudaSuccess) return e;
        active = kSMs * per_sm;
    }
    if (active < 1) return cudaErrorInvalidValue;
    int band = tu.band > 0 ? tu.band : (Nz + active - 1) / active;
    band = band < 1 ? 1 : band;
    h[0].G = CL * kRcThreads;
    h[0].band = band;
    tu.band = band;
    tu.rK = 5;
    L.fn = fn;
    L.grid = dim3(CL * ((Nz + band - 1) / band), 1, 1);
    L.block = dim3(kRcThreads, 1, 1);
    L.smem = smem;
    L.flip = true;
    L.cluster = CL;
    // no early launch: blocks of a cluster are placed together, and placed
    // while the previous kernel's blocks still hold the SMs they land
    // unevenly, so that part of the band-sized grid waited for a second wave
    // (refined steps back to back: 773 us against 602 us one at a time)
    L.pdl = false;
    return cudaSuccess;
}

template <typename real, int MODE>
static cudaError_t plan_rsweep(SweepArgs<real> *h, int n, Tuning &tu, Launch &L)
{
    int maxNr = 0;
    for (int m = 0; m < n; ++m) maxNr = h[m].Nr > maxNr ? h[m].Nr : maxNr;
    int K = tu.rK;
    if (K <= 0) {
        K = default_rK((int)sizeof(real), maxNr);
        if (n > 1)
            while (K < 32 && (maxNr + K - 1) / K > 32) K *= 2;
    }
    tu.rK = K;
    cudaError_t e;
    switch (K) {
    case 4: e = plan_rsweep_k<real, 4, MODE>(h, n, tu.band, L); break;
    case 8: e = plan_rsweep_k<real, 8, MODE>(h, n, tu.band, L); break;
    case 16: e = plan_rsweep_k<real, 16, MODE>(h, n, tu.band, L); break;
    case 32: e = plan_rsweep_k<real, 32, MODE>(h, n, tu.band, L); break;
    default: return cudaErrorInvalidValue;
    }
    tu.band = h[0].band;
    return e;
}

// One z pass: chunk summaries, carries, chunk solves, for n instances
// (instance m in the last grid dimension; blocks past an instance's columns
// or chunks return at once).
// OUT selects the solve pass's output (zsolve2_kernel) and CSUM the summary
// pass that reads its right-hand side from the output buffer (zsumc_kernel):
// the two z solves of the refined path.
template <typename real, int MODE, int OUT = ZOUT_FIELD, bool CSUM = false>
static cudaError_t plan_zpass(const SweepArgs<real> *h, int n, Tuning &tu, std::vector<Launch> &out)
{
    constexpr int V = 16 / (int)sizeof(real);
    constexpr int COLS = 32 * V;
    int maxNr = 0, maxRc = 0, maxNch = 0;
    for (int m = 0; m < n; ++m) {
        maxNr = h[m].Nr > maxNr ? h[m].Nr : maxNr;
        maxRc = h[m].Rc > maxRc ? h[m].Rc : maxRc;
        maxNch = h[m].nch > maxNch ? h[m].nch : maxNch;
    }
    constexpr bool lean = MODE == MODE_LIT || MODE == MODE_DELTA;  // heat_zline.cuh passes
    // warps per instance: one per 32 V columns, or (lean passes) one per
    // column tile where the instance has a tile table
    int groups = (maxNr + COLS - 1) / COLS;
    bool tiled = false;
    for (int m = 0; m < n && lean; ++m)
        if (h[m].n_ztile > 0) tiled = true, groups = h[m].n_ztile > groups ? h[m].n_ztile : groups;
    Launch a, b, c;
    // warps per block: the most of 4, 2, 1 whose grid still runs as one wave
    // of 16 resident warps per SM (the passes' register use), as every chunk
    // walk then runs at once (config 2 tiled: 17 tiles x 128 chunks in blocks
    // of 2; 4 would leave part of a second wave)
    int SWPB = 4;
    if (tiled)
        while (SWPB > 1 && (long long)((groups + SWPB - 1) / SWPB) * maxNch * n > (long long)kSMs * 16 / SWPB)
            SWPB /= 2;
    // a batch with a work list: one warp per (instance, chunk, column tile)
    const int nitem = lean ? h[0].n_zitem : 0;
    auto lean_grid = [&](int wpb) {
        return nitem > 0 ? dim3((nitem + wpb - 1) / wpb, 1, 1) : dim3((groups + wpb - 1) / wpb, maxNch, n);
    };
    constexpr int LM = lean ? MODE : MODE_DELTA;
    a.fn = !lean      ? (const void *)zsum_kernel<real, V, MODE>
           : nitem > 0 ? (const void *)zsum2_kernel<real, V, LM, true>
                       : (const void *)zsum2_kernel<real, V, LM, false>;
    if constexpr (CSUM) {
        static_assert(sizeof(real) == 4 && lean, "the correction summary is FP32, lean");
        a.fn = nitem > 0 ? (const void *)zsumc_kernel<V, true> : (const void *)zsumc_kernel<V, false>;
    }
    a.grid = lean ? lean_grid(SWPB) : dim3((groups + SWPB - 1) / SWPB, maxNch, n);
    a.block = dim3(32 * SWPB, 1, 1);
    a.smem = (size_t)SWPB * maxRc * 8 * sizeof(real);
    a.flip = true;
    cudaError_t e = allow_smem(a.fn, a.smem);
    if (e != cudaSuccess) return e;
    if (maxNch > ZSEG2 * ZMAXM) return cudaErrorInvalidValue;
    // carry pass: the fewest segments (warps per block) that cover the chunks
    // -- a 1024-thread block of 32 segments holds a whole SM's registers, so a
    // batch of short columns would run its column groups one block per SM,
    // and in FP64 it spills
    const int seg = maxNch <= 4 * ZMAXM ? 4 : maxNch <= 16 * ZMAXM ? 16 : ZSEG2;
    b.fn = seg == 4    ? (const void *)zcarry2_kernel<real, 4>
           : seg == 16 ? (const void *)zcarry2_kernel<real, 16>
                       : (const void *)zcarry2_kernel<real, ZSEG2>;
    b.grid = dim3((maxNr + 31) / 32, n, 1);
    b.block = dim3(32 * seg, 1, 1);
    b.smem = 0;
    b.flip = false;
    int wpb = tu.zwpb;
    if (wpb != 1 && wpb != 2) wpb = (size_t)maxRc * COLS * sizeof(real) <= 32 * 1024 ? 2 : 1;
    tu.zwpb = wpb;
    // the lean solve keeps no forward results: 4 warps per block (as the
    // summary pass: 1 for a single tiled instance), staged (P, cp) rows only
    const int cw = lean ? SWPB : wpb;
    c.fn = !lean      ? (const void *)zsolve_kernel<real, V, MODE>
           : nitem > 0 ? (const void *)zsolve2_kernel<real, V, LM, true, OUT>
                       : (const void *)zsolve2_kernel<real, V, LM, false, OUT>;
    c.grid = lean ? lean_grid(cw) : dim3((groups + cw - 1) / cw, maxNch, n);
    c.block = dim3(32 * cw, 1, 1);
    c.smem = lean ? (size_t)cw * ZNC * maxRc * 2 * sizeof(real) : (size_t)wpb * maxRc * (COLS + 8) * sizeof(real);
    c.flip = true;
    if ((e = allow_smem(c.fn, c.smem)) != cudaSuccess) return e;
    out.push_back(a);
    out.push_back(b);
    out.push_back(c);
    return cudaSuccess;
}

// The whole plan of one form.  Fills G and band of every h[m].
template <typename real, int MODE>
static cudaError_t plan_mode(SweepArgs<real> *h, int n, const Tuning &req, SweepPlan &plan)
{
    plan = SweepPlan();
    Tuning tu = req;
    // column tiles only for a single instance: in a batch the widest
    // member's tile count would set every member's grid width
    if (n > 1)
        for (int m = 0; m < n; ++m) h[m].n_ztile = 0, h[m].ztile = nullptr;
    Launch r;
    cudaError_t e = cudaErrorInvalidValue;
    bool line_tables = MODE == MODE_LIT || MODE == MODE_DELTA;
    for (int m = 0; m < n && line_tables; ++m) line_tables = h[m].rl.tA != nullptr;
    // rK: 0 = default, 1 = line teams, 2 = register-resident lines (FP32
    // increment form), 3 = walked lines (FP32 increment form, one instance),
    // 5 = cluster lines (FP32 increment forms, one instance), 4, 8, 16, 32 =
    // block lines with rK cells per thread
    if constexpr (MODE == MODE_DELTA && sizeof(real) == 4) {
        // walked lines on request only: measured slower than the register-
        // resident lines on lines of 512 to 2048 cells
        if (tu.rK == 3) {
            e = plan_rwalk(h, n, tu, r);
            if (e != cudaSuccess) return e;
        }
        if (e != cudaSuccess && (tu.rK == 0 || tu.rK == 2)) {
            e = plan_rblock(h, n, tu, r);
            if (e != cudaSuccess && tu.rK == 2) return e;
        }
        // lines longer than one block holds: a cluster per line
        if (e != cudaSuccess && (tu.rK == 0 || tu.rK == 5)) {
            e = plan_rclus<MODE>(h, n, tu, r);
            if (e != cudaSuccess && tu.rK == 5) return e;
            if (e != cudaSuccess) {  // not available: the next kernel in line
                (void)cudaGetLastError();
                e = cudaErrorInvalidValue;
            }
        }
    } else if constexpr (MODE == MODE_REFINE) {
        if (tu.rK == 2 || tu.rK == 3) return cudaErrorInvalidValue;
        if (tu.rK == 0 || tu.rK == 5) {
            e = plan_rclus<MODE>(h, n, tu, r);
            if (e != cudaSuccess && tu.rK == 5) return e;
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                e = cudaErrorInvalidValue;
            }
        }
    } else {
        if (tu.rK == 2 || tu.rK == 3 || tu.rK == 5) return cudaErrorInvalidValue;
    }
    if constexpr (MODE == MODE_LIT || MODE == MODE_DELTA) {
        if (e == cudaErrorInvalidValue) {
            if (tu.rK == 1 && !line_tables) return cudaErrorInvalidValue;
            if (tu.rK <= 1 && line_tables) e = plan_rline<real, MODE>(h, n, tu, r);
        }
    }
    if (e == cudaErrorInvalidValue) {
        if (tu.rK <= 2) tu.rK = 0;
        e = plan_rsweep<real, MODE>(h, n, tu, r);
    }
    if (e != cudaSuccess) return e;
    plan.dir[0].push_back(r);
    if constexpr (MODE == MODE_REFINE) {
        if (n == 1) {
            // lean passes: delta0 into the rho buffer; the residual at delta0
            // (zres_kernel) into the output buffer; the correction's summary
            // from it and the solve that stores theta + (delta0 + e)
            if ((e = plan_zpass<real, MODE_DELTA, ZOUT_DELTA0>(h, n, tu, plan.dir[1])) != cudaSuccess) return e;
            Launch rz;
            constexpr int V = 4;
            const int warps = (h[0].Nr + 32 * V - 1) / (32 * V);
            rz.fn = (const void *)zres_kernel<V>;
            rz.grid = dim3((warps + 3) / 4, (h[0].Nz + kZResRows - 1) / kZResRows, 1);
            rz.block = dim3(128, 1, 1);
            rz.smem = 0;
            rz.flip = true;
            plan.dir[1].push_back(rz);
            if ((e = plan_zpass<real, MODE_DELTA, ZOUT_CORR, true>(h, n, tu, plan.dir[1])) != cudaSuccess) return e;
        } else {
            if ((e = plan_zpass<real, MODE_REFINE>(h, n, tu, plan.dir[1])) != cudaSuccess) return e;
            if ((e = plan_zpass<real, MODE_CORR>(h, n, tu, plan.dir[1])) != cudaSuccess) return e;
        }
    } else {
        if ((e = plan_zpass<real, MODE>(h, n, tu, plan.dir[1])) != cudaSuccess) return e;
    }
    // by-value arguments: the first instance's final arguments
    for (auto &dir : plan.dir)
        for (Launch &L : dir)
            if (!L.pargs.empty())
                L.pargs.assign(reinterpret_cast<const unsigned char *>(&h[0]),
                               reinterpret_cast<const unsigned char *>(&h[0]) + sizeof(SweepArgs<real>));
    plan.used = tu;
    return cudaSuccess;
}

// Per-form plan builders, each compiled in its own translation unit.
cudaError_t plan_fp64(SweepArgs<double> *h, int n, const Tuning &req, SweepPlan &plan);
cudaError_t plan_fp32(SweepArgs<float> *h, int n, const Tuning &req, SweepPlan &plan);
cudaError_t plan_fp32_refined(SweepArgs<float> *h, int n, const Tuning &req, SweepPlan &plan);

}  // namespace heat
