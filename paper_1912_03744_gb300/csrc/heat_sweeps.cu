// heat_sweeps.cu -- sm_103a kernels of one Peaceman-Rachford ADI step.
//
// One step (Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2") on the field stored as
// theta = T - T_ref, row-major [Nz][Nr]:
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
// Partitioned Thomas.  A line is cut into chunks owned by different threads.
// Each thread runs the forward recurrence on its chunk with a zero carry,
// giving the affine map  carry_out = B + F carry_in  (F = prod f); an
// exclusive scan of these maps yields every chunk's true carry-in and the
// thread reruns its chunk with it.  The backward recurrence is handled the
// same way from the other end (x_start = G + H x_next, H = prod cp).
//   r-sweep: lines are contiguous rows; one line per block (or per warp
//     segment for short rows), K consecutive cells per thread loaded with
//     128-bit loads; scans by warp shuffles, then shared memory across warps.
//     A block walks a band of consecutive rows keeping rows j-1, j, j+1 in
//     registers, so each row is read once from memory.
//   z-sweep: lines are columns; a block owns a strip of 32 columns (one per
//     lane, loads coalesced into 128-byte rows) and a run of rows, KZ rows per
//     thread.  Long columns are split over a thread-block cluster; the carries
//     between its blocks go through distributed shared memory.
#include <cooperative_groups.h>

#include <cstdio>

#include "heat_internal.h"

namespace cg = cooperative_groups;

namespace heat {

#define HEAT_FULL_MASK 0xffffffffu

enum { MODE_LIT = 0, MODE_DELTA = 1, MODE_REFINE = 2 };

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

// K consecutive values row[i0 .. i0+K), zero past n; 16-byte loads when aligned.
template <typename real, int K>
__device__ __forceinline__ void load_chunk(const real *__restrict__ row, int i0, int n, bool vec, real (&v)[K])
{
    constexpr int V = 16 / (int)sizeof(real);
    if (vec && i0 + K <= n) {
#pragma unroll
        for (int k = 0; k < K; k += V) {
            if constexpr (sizeof(real) == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(row + i0 + k));
                v[k] = t.x;
                v[k + 1] = t.y;
                v[k + 2] = t.z;
                v[k + 3] = t.w;
            } else {
                const double2 t = __ldg(reinterpret_cast<const double2 *>(row + i0 + k));
                v[k] = t.x;
                v[k + 1] = t.y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (i0 + k < n) ? row[i0 + k] : real(0);
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
// [(b*lpb + s)*band, +band).  G <= 32: slots are lane segments; G > 32: one
// slot per block (wide), cross-warp carries through shared memory.
template <typename real, int K, int MODE, int LB>
__global__ void __launch_bounds__(LB) rsweep_kernel(const real *__restrict__ th, real *__restrict__ out, int Nr,
                                                      int Nz, int G, int band, const int *__restrict__ rowcls,
                                                      const int *__restrict__ colcls, LineTab<real> R,
                                                      LineTab<real> Z, LineTab64 R64, LineTab64 Z64, BcVals bc)
{
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
    constexpr int V = 16 / (int)sizeof(real);
    const bool vec = (Nr % V) == 0;
    const int jstart = (blockIdx.x * lpb + slot) * band;
    const real bc0 = (real)bc.th[0], bc1 = (real)bc.th[1], bc2 = (real)bc.th[2], bc3 = (real)bc.th[3];

    // column classes of this thread's cells; uniform flag for the fast path
    int zc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) zc[k] = (i0 + k < Nr) ? colcls[i0 + k] : 0;
    bool zuni = true;
#pragma unroll
    for (int k = 1; k < K; ++k) zuni = zuni && (zc[k] == zc[0]);

    real tp[K], tc[K], tn[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tp[k] = tc[k] = tn[k] = real(0);
    if (jstart - 1 >= 0 && jstart - 1 < Nz) load_chunk<real, K>(th + (size_t)(jstart - 1) * Nr, i0, Nr, vec, tp);
    if (jstart < Nz) load_chunk<real, K>(th + (size_t)jstart * Nr, i0, Nr, vec, tc);
    if (jstart + 1 < Nz) load_chunk<real, K>(th + (size_t)(jstart + 1) * Nr, i0, Nr, vec, tn);

    int acls = -1;
    real inv[K], f[K], cp[K], c0[K], c1[K], c2[K], c3[K], c4[K];
#pragma unroll
    for (int k = 0; k < K; ++k) inv[k] = f[k] = cp[k] = c0[k] = c1[k] = c2[k] = c3[k] = c4[k] = real(0);

    for (int t = 0; t < band; ++t) {
        const int j = jstart + t;
        const bool valid = j < Nz;
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
                    c2[k] = in ? R.dl[ro + i] : real(0);
                    c3[k] = in ? R.dh[ro + i] : real(0);
                    c4[k] = in ? R.q[ro + i] : real(0);
                }
            }
            acls = a;
        }
        // right-hand side
        real d[K];
        real left = real(0), right = real(0);
        if constexpr (MODE != MODE_LIT) {
            left = __shfl_up_sync(HEAT_FULL_MASK, tc[K - 1], 1, W);
            right = __shfl_down_sync(HEAT_FULL_MASK, tc[0], 1, W);
            if (ls == 0) left = (valid && i0 > 0) ? th[(size_t)j * Nr + i0 - 1] : tc[0];
            if (ls == W - 1) right = (valid && i0 + K < Nr) ? th[(size_t)j * Nr + i0 + K] : tc[K - 1];
        }
        {
            real zam = real(0), zap = real(0), zx = real(0), zy = real(0);
            if (zuni && valid) {
                const size_t zo = (size_t)zc[0] * Nz + j;
                if constexpr (MODE == MODE_LIT) {
                    zam = Z.am[zo];
                    zap = Z.ap[zo];
                    zx = Z.ad[zo];
                    zy = Z.sd[zo];
                } else {
                    zam = Z.am[zo];
                    zap = Z.ap[zo];
                    zx = Z.dl[zo];
                    zy = Z.dh[zo];
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                real am2 = zam, ap2 = zap, x2 = zx, y2 = zy;
                if (!zuni && valid && i0 + k < Nr) {
                    const size_t zo = (size_t)zc[k] * Nz + j;
                    am2 = Z.am[zo];
                    ap2 = Z.ap[zo];
                    x2 = MODE == MODE_LIT ? Z.ad[zo] : Z.dl[zo];
                    y2 = MODE == MODE_LIT ? Z.sd[zo] : Z.dh[zo];
                }
                const real t0 = tc[k];
                if constexpr (MODE == MODE_LIT) {
                    d[k] = fmad(c0[k] + x2, t0, fmad(am2, tp[k], fmad(ap2, tn[k], c1[k] + y2)));
                } else {
                    const real tl = k > 0 ? tc[k - 1] : left;
                    const real tr = k < K - 1 ? tc[k + 1] : right;
                    real r = c4[k];
                    r = fmad(c0[k], tl - t0, r);
                    r = fmad(c1[k], tr - t0, r);
                    r = fmad(c2[k], bc0 - t0, r);
                    r = fmad(c3[k], bc1 - t0, r);
                    r = fmad(am2, tp[k] - t0, r);
                    r = fmad(ap2, tn[k] - t0, r);
                    r = fmad(x2, bc2 - t0, r);
                    r = fmad(y2, bc3 - t0, r);
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
            double tl64 = __shfl_up_sync(HEAT_FULL_MASK, (double)tc[K - 1], 1, W);
            double tr64 = __shfl_down_sync(HEAT_FULL_MASK, (double)tc[0], 1, W);
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
            if (ls == 0) tl64 = (valid && i0 > 0) ? (double)th[(size_t)j * Nr + i0 - 1] : (double)tc[0];
            if (ls == W - 1) tr64 = (valid && i0 + K < Nr) ? (double)th[(size_t)j * Nr + i0 + K] : (double)tc[K - 1];
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
                    r = fma(Z64.am[zo], (double)tp[k] - t0, r);
                    r = fma(Z64.ap[zo], (double)tn[k] - t0, r);
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
        // advance the window
#pragma unroll
        for (int k = 0; k < K; ++k) {
            tp[k] = tc[k];
            tc[k] = tn[k];
            tn[k] = real(0);
        }
        if (j + 2 < Nz) load_chunk<real, K>(th + (size_t)(j + 2) * Nr, i0, Nr, vec, tn);
    }
}

// ------------------------------------------------------------------ z-sweep
// Cluster of Q blocks per strip of 32 columns; block rank q owns rows
// [q*NW*KZ, (q+1)*NW*KZ), warp w of it rows [(q*NW+w)*KZ, +KZ); lane = column.
// Per-lane carries: warps compose through shared memory, blocks of the
// cluster through distributed shared memory (one hardware cluster barrier
// per direction, no spin-waits).
template <typename real>
struct ZScan {
    real F[32][33], B[32][33];  // per warp, per lane
    real tF[32], tB[32];        // forward block total per lane (read by other blocks)
    real tH[32], tG[32];        // backward block total per lane (read by other blocks)
    real cin[32], xin[32];      // carries into this block per lane
    double eLo[32][33], eHi[32][33];  // refined path: first/last increment of each chunk
};

// Solve this thread's chunk d[KZ] of a column with the cluster-wide carries.
template <typename real, int KZ>
__device__ __forceinline__ void solve_col(real (&d)[KZ], const real *__restrict__ inv, const real *__restrict__ f,
                                          const real *__restrict__ cp, int j0, int Nz, bool col, int lane, int w,
                                          int NW, int q, int Q, ZScan<real> &S, cg::cluster_group &cl)
{
    real F = real(1), B = real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = j0 + k;
        const real iv = (col && j < Nz) ? inv[j] : real(0), ff = (col && j < Nz) ? f[j] : real(0);
        B = fmad(d[k], iv, ff * B);
        F *= ff;
    }
    S.F[w][lane] = F;
    S.B[w][lane] = B;
    __syncthreads();
    real Fx = real(1), Bx = real(0);
    for (int v = 0; v < w; ++v) {
        Bx = fmad(S.F[v][lane], Bx, S.B[v][lane]);
        Fx *= S.F[v][lane];
    }
    if (w == 0) {
        real Ft = real(1), Bt = real(0);
        for (int v = 0; v < NW; ++v) {
            Bt = fmad(S.F[v][lane], Bt, S.B[v][lane]);
            Ft *= S.F[v][lane];
        }
        S.tF[lane] = Ft;
        S.tB[lane] = Bt;
    }
    cl.sync();
    if (w == 0) {
        real c = real(0);
        for (int r = 0; r < q; ++r) {
            const ZScan<real> *rs = cl.map_shared_rank(&S, r);
            c = fmad(rs->tF[lane], c, rs->tB[lane]);
        }
        S.cin[lane] = c;
    }
    __syncthreads();
    real dp = fmad(Fx, S.cin[lane], Bx);
    real H = real(1), Gm = real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = j0 + k;
        const real iv = (col && j < Nz) ? inv[j] : real(0), ff = (col && j < Nz) ? f[j] : real(0);
        dp = fmad(d[k], iv, ff * dp);
        d[k] = dp;
    }
#pragma unroll
    for (int k = KZ - 1; k >= 0; --k) {
        const int j = j0 + k;
        const real cc = (col && j < Nz) ? cp[j] : real(0);
        Gm = fmad(cc, Gm, d[k]);
        H *= cc;
    }
    S.F[w][lane] = H;
    S.B[w][lane] = Gm;
    __syncthreads();
    real Hx = real(1), Gx = real(0);
    for (int v = NW - 1; v > w; --v) {
        Gx = fmad(S.F[v][lane], Gx, S.B[v][lane]);
        Hx *= S.F[v][lane];
    }
    if (w == 0) {
        real Ht = real(1), Gt = real(0);
        for (int v = NW - 1; v >= 0; --v) {
            Gt = fmad(S.F[v][lane], Gt, S.B[v][lane]);
            Ht *= S.F[v][lane];
        }
        S.tH[lane] = Ht;
        S.tG[lane] = Gt;
    }
    cl.sync();
    if (w == 0) {
        real c = real(0);
        for (int r = Q - 1; r > q; --r) {
            const ZScan<real> *rs = cl.map_shared_rank(&S, r);
            c = fmad(rs->tH[lane], c, rs->tG[lane]);
        }
        S.xin[lane] = c;
    }
    __syncthreads();
    real x = fmad(Hx, S.xin[lane], Gx);
#pragma unroll
    for (int k = KZ - 1; k >= 0; --k) {
        const int j = j0 + k;
        const real cc = (col && j < Nz) ? cp[j] : real(0);
        x = fmad(cc, x, d[k]);
        d[k] = x;
    }
    // the shared scan buffers are reused by the caller: everyone must be past
    // the remote reads of this solve first
    cl.sync();
}

template <typename real, int KZ, int MODE>
__global__ void __launch_bounds__(1024) zsweep_kernel(const real *__restrict__ th, real *__restrict__ out, int Nr,
                                                      int Nz, const int *__restrict__ rowcls,
                                                      const int *__restrict__ colcls, LineTab<real> R,
                                                      LineTab<real> Z, LineTab64 R64, LineTab64 Z64, BcVals bc)
{
    __shared__ ZScan<real> S;
    cg::cluster_group cl = cg::this_cluster();
    const int Q = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int strip = blockIdx.x / Q;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int i = strip * 32 + lane;
    const bool col = i < Nr;
    const int j0 = (q * NW + w) * KZ;
    const size_t zo = (size_t)(col ? colcls[i] : 0) * Nz;
    const real bc0 = (real)bc.th[0], bc1 = (real)bc.th[1], bc2 = (real)bc.th[2], bc3 = (real)bc.th[3];

    // right-hand side, streaming down the thread's rows
    real d[KZ];
    int acur = -1;
    real ra = real(0), rb = real(0), rc = real(0), rd = real(0);
    real tprev = (col && j0 - 1 >= 0 && j0 - 1 < Nz) ? th[(size_t)(j0 - 1) * Nr + i] : real(0);
    real tcur = (col && j0 < Nz) ? th[(size_t)j0 * Nr + i] : real(0);
#pragma unroll
    for (int k = 0; k < KZ; ++k) {
        const int j = j0 + k;
        const bool vr = j < Nz;
        const real tnext = (col && j + 1 < Nz) ? th[(size_t)(j + 1) * Nr + i] : real(0);
        const int a = vr ? rowcls[j] : acur;
        if (a != acur && vr) {
            if (col) {
                const size_t ro = (size_t)a * Nr + i;
                if constexpr (MODE == MODE_LIT) {
                    ra = R.am[ro];
                    rb = R.ap[ro];
                    rc = R.ad[ro];
                    rd = R.sd[ro];
                } else {
                    ra = R.am[ro];
                    rb = R.ap[ro];
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
            if constexpr (MODE == MODE_LIT) {
                dd = fmad(Z.w[zo + j] + rc, tcur, fmad(ra, tl, fmad(rb, tr, Z.s[zo + j] + rd)));
            } else {
                real r = Z.q[zo + j];
                r = fmad(Z.am[zo + j], tprev - tcur, r);
                r = fmad(Z.ap[zo + j], tnext - tcur, r);
                r = fmad(Z.dl[zo + j], bc2 - tcur, r);
                r = fmad(Z.dh[zo + j], bc3 - tcur, r);
                r = fmad(ra, tl - tcur, r);
                r = fmad(rb, tr - tcur, r);
                r = fmad(rc, bc0 - tcur, r);
                r = fmad(rd, bc1 - tcur, r);
                dd = r;
            }
        }
        d[k] = dd;
        tprev = tcur;
        tcur = tnext;
    }

    const real *inv = Z.inv + zo, *f = Z.f + zo, *cp = Z.cp + zo;
    if constexpr (MODE == MODE_REFINE) {
        real x0[KZ];
#pragma unroll
        for (int k = 0; k < KZ; ++k) x0[k] = d[k];
        solve_col<real, KZ>(x0, inv, f, cp, j0, Nz, col, lane, w, NW, q, Q, S, cl);
        // neighbours of the chunk ends along the column (other warps / blocks)
        S.eLo[w][lane] = (double)x0[0];
        S.eHi[w][lane] = (double)x0[KZ - 1];
        cl.sync();
        double xm_end = 0.0, xp_end = 0.0;
        if (w > 0) xm_end = S.eHi[w - 1][lane];
        else if (q > 0) xm_end = cl.map_shared_rank(&S, q - 1)->eHi[NW - 1][lane];
        if (w < NW - 1) xp_end = S.eLo[w + 1][lane];
        else if (q < Q - 1) xp_end = cl.map_shared_rank(&S, q + 1)->eLo[0][lane];
        double tprev64 = (col && j0 - 1 >= 0 && j0 - 1 < Nz) ? (double)th[(size_t)(j0 - 1) * Nr + i] : 0.0;
        double tcur64 = (col && j0 < Nz) ? (double)th[(size_t)j0 * Nr + i] : 0.0;
        int a64 = -1;
        double A0 = 0, A1 = 0, A2 = 0, A3 = 0;
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int j = j0 + k;
            const bool vr = j < Nz;
            const double tnext64 = (col && j + 1 < Nz) ? (double)th[(size_t)(j + 1) * Nr + i] : 0.0;
            const int a = vr ? rowcls[j] : a64;
            if (a != a64 && vr) {
                if (col) {
                    const size_t ro = (size_t)a * Nr + i;
                    A0 = R64.am[ro];
                    A1 = R64.ap[ro];
                    A2 = R64.dl[ro];
                    A3 = R64.dh[ro];
                }
                a64 = a;
            }
            double tl = __shfl_up_sync(HEAT_FULL_MASK, tcur64, 1);
            double tr = __shfl_down_sync(HEAT_FULL_MASK, tcur64, 1);
            if (lane == 0) tl = (col && i > 0 && vr) ? (double)th[(size_t)j * Nr + i - 1] : tcur64;
            if (lane == 31) tr = (i + 1 < Nr && vr) ? (double)th[(size_t)j * Nr + i + 1] : tcur64;
            double rho = 0.0;
            if (col && vr) {
                const size_t zj = zo + j;
                double r = Z64.q[zj];
                r = fma(Z64.am[zj], tprev64 - tcur64, r);
                r = fma(Z64.ap[zj], tnext64 - tcur64, r);
                r = fma(Z64.dl[zj], bc.th[2] - tcur64, r);
                r = fma(Z64.dh[zj], bc.th[3] - tcur64, r);
                r = fma(A0, tl - tcur64, r);
                r = fma(A1, tr - tcur64, r);
                r = fma(A2, bc.th[0] - tcur64, r);
                r = fma(A3, bc.th[1] - tcur64, r);
                const double xm = k > 0 ? (double)x0[k - 1] : xm_end;
                const double xp = k < KZ - 1 ? (double)x0[k + 1] : xp_end;
                rho = r - (Z64.b[zj] * (double)x0[k] - Z64.m[zj] * xm - Z64.p[zj] * xp);
            }
            d[k] = (real)rho;
            tprev64 = tcur64;
            tcur64 = tnext64;
        }
        solve_col<real, KZ>(d, inv, f, cp, j0, Nz, col, lane, w, NW, q, Q, S, cl);
#pragma unroll
        for (int k = 0; k < KZ; ++k) d[k] = (real)((double)x0[k] + (double)d[k]);
    } else {
        solve_col<real, KZ>(d, inv, f, cp, j0, Nz, col, lane, w, NW, q, Q, S, cl);
    }
    if (col) {
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int j = j0 + k;
            if (j < Nz) {
                const size_t c = (size_t)j * Nr + i;
                if constexpr (MODE == MODE_LIT)
                    out[c] = d[k];
                else
                    out[c] = th[c] + d[k];
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

__global__ void __launch_bounds__(256) energy_final_kernel(const double *__restrict__ part, int n,
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

template <typename real, int K, int MODE>
static cudaError_t rsweep_k(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                            const LineTab<real> &Z)
{
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    const int G = next_pow2((Nr + K - 1) / K);
    const int block = G <= 32 ? 128 : G;
    const int lpb = block / G;
    const int per_sm = G <= 256 ? 4 : (G <= 512 ? 2 : 1);
    int slots_wanted = kSMs * per_sm * lpb;
    int slots = Nz < slots_wanted ? Nz : slots_wanted;
    const int band = (Nz + slots - 1) / slots;
    const int grid = ((Nz + band - 1) / band + lpb - 1) / lpb;
    if (block <= 256)
        rsweep_kernel<real, K, MODE, 256><<<grid, block, 0, ctx->stream>>>(
            in, out, Nr, Nz, G, band, ctx->d_rowcls, ctx->d_colcls, R, Z, ctx->dR.full, ctx->dZ.full, bc_vals(ctx));
    else
        rsweep_kernel<real, K, MODE, 1024><<<grid, block, 0, ctx->stream>>>(
            in, out, Nr, Nz, G, band, ctx->d_rowcls, ctx->d_colcls, R, Z, ctx->dR.full, ctx->dZ.full, bc_vals(ctx));
    return cudaGetLastError();
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
static cudaError_t zsweep_k(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                            const LineTab<real> &Z)
{
    const int Nr = ctx->g.Nr, Nz = ctx->g.Nz;
    const int rows_max = 32 * KZ;  // rows per block at 32 warps
    const int Q = (Nz + rows_max - 1) / rows_max;
    int NW = (Nz + Q * KZ - 1) / (Q * KZ);
    NW = NW < 1 ? 1 : NW;
    auto kern = zsweep_kernel<real, KZ, MODE>;
    if (Q > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    const int strips = (Nr + 31) / 32;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(strips * Q, 1, 1);
    cfg.blockDim = dim3(32 * NW, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, in, out, Nr, Nz, (const int *)ctx->d_rowcls, (const int *)ctx->d_colcls, R,
                              Z, ctx->dR.full, ctx->dZ.full, bc_vals(ctx));
}

// Longest column a cluster of 16 blocks covers: 16 x 32 warps x 32 rows.
constexpr int kMaxNz = 16 * 32 * 32;

template <typename real, int MODE>
static cudaError_t launch_zsweep(const heat_ctx *ctx, const real *in, real *out, const LineTab<real> &R,
                                 const LineTab<real> &Z)
{
    const int Nz = ctx->g.Nz;
    if (Nz <= 8 * 32 * 8) return zsweep_k<real, 8, MODE>(ctx, in, out, R, Z);
    if (Nz <= 8 * 32 * 16) return zsweep_k<real, 16, MODE>(ctx, in, out, R, Z);
    return zsweep_k<real, 32, MODE>(ctx, in, out, R, Z);
}

template <typename real, int MODE>
static cudaError_t sweep_mode(heat_ctx *ctx, int dir, const real *a, real *b, const LineTab<real> &R,
                              const LineTab<real> &Z)
{
    return dir == 0 ? launch_rsweep<real, MODE>(ctx, a, b, R, Z) : launch_zsweep<real, MODE>(ctx, a, b, R, Z);
}

// One half-step from buffer cur into the other buffer (the caller flips cur).
cudaError_t launch_sweep_buffers(heat_ctx *ctx, int dir, const void *a, void *b)
{
    switch (ctx->precision) {
    case HEAT_FP64:
        return sweep_mode<double, MODE_LIT>(ctx, dir, (const double *)a, (double *)b, ctx->dR.t64, ctx->dZ.t64);
    case HEAT_FP32:
        return sweep_mode<float, MODE_DELTA>(ctx, dir, (const float *)a, (float *)b, ctx->dR.t32, ctx->dZ.t32);
    default:
        return sweep_mode<float, MODE_REFINE>(ctx, dir, (const float *)a, (float *)b, ctx->dR.t32, ctx->dZ.t32);
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

int launches_per_step(const heat_ctx *) { return 2; }

int max_nz() { return kMaxNz; }

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

}  // namespace heat
