// heat_rline.cuh -- the r-sweep as one short team of lanes per r-line
// (half-step 1 of the Peaceman-Rachford step, Sec. 3, eq. "scheme_eq_1";
// the line matrix is the radial operator of eq. "Lambda_r" plus the mass term).
//
// A line team of LW lanes (LW = 4..32, a power of two, 32/LW teams per warp)
// owns one r-line at a time and walks it in segments of S = LW*K cells, lane t
// holding the K consecutive cells [c K, c K + K) of chunk c = s LW + t.  The
// line matrix is fixed per row class, so everything that depends on it alone
// is tabulated once per dt (see RLine in heat_internal.h):
//   forward  (d'_i = d_i inv_i + f_i d'_{i-1}):  the chunk's carry-out with a
//            zero carry-in is B = sum_k d_k wB_k and the carry-out for carry-in
//            D is B + F D, F = prod f over the chunk;
//   backward (x_i = d'_i + cp_i x_{i+1}):        the chunk's first value with a
//            zero carry-in is G = sum_k d'_k wC_k and G + H X for carry-in X,
//            H = prod cp over the chunk.
// The carries across the team are a Kogge-Stone scan of these affine maps in
// which the multiplier of every level (a product of F, or of H, over the lanes
// it spans, 0 where the level reaches past the segment) is a table entry, so
// a level costs one shuffle and one FMA.  Segment s hands its last d' (and,
// walking back, its first x) to the next segment in registers.
//
// Walk 1 (segments in order): right-hand side from rows j-1, j, j+1 (the
// explicit z-operator of eq. "scheme_eq_1"), forward summaries, scan, forward
// recurrence; d' goes to a per-team shared-memory buffer.  Walk 2 (segments in
// reverse): backward summaries, scan, backward recurrence, and the new value
// (theta + delta in the increment form, x in the literal form) is stored.
// Lanes never synchronise beyond their warp: no block barrier, no waits.
//
// A team solves R rows of one row class together (a "unit", listed by the
// host): the table values each lane loads serve all R rows, and the R
// recurrences and scans are independent instruction streams.
//
// Work split: the units of an instance are dealt to the teams of the grid in
// contiguous runs (team g gets units [g U / T, (g+1) U / T)), so every team
// has the same number of units up to one.  Teams of a warp with fewer units
// repeat their last unit without storing it, to keep the warp's shuffles full.
#pragma once

#include "heat_internal.h"

namespace heat {

template <typename real, int K>
struct RLineIO {
    static constexpr int V = 16 / (int)sizeof(real);  // reals per 16-byte access
    // K values of row `row` from cell i0 on; cells past Nr read `pad`.
    static __device__ __forceinline__ void load(const real *__restrict__ row, int i0, int Nr, bool vec, real pad,
                                                real (&v)[K])
    {
        if (vec && i0 + K <= Nr) {
#pragma unroll
            for (int k = 0; k < K; k += V) {
                if constexpr (sizeof(real) == 4) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(row + i0 + k));
                    v[k] = a.x, v[k + 1] = a.y, v[k + 2] = a.z, v[k + 3] = a.w;
                } else {
                    const double2 a = __ldg(reinterpret_cast<const double2 *>(row + i0 + k));
                    v[k] = a.x, v[k + 1] = a.y;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = i0 + k < Nr ? row[i0 + k] : pad;
        }
    }
    static __device__ __forceinline__ void fill(real x, real (&v)[K])
    {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = x;
    }
    static __device__ __forceinline__ void store(real *__restrict__ row, int i0, int Nr, bool vec, const real (&v)[K])
    {
        if (vec && i0 + K <= Nr) {
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
                if (i0 + k < Nr) row[i0 + k] = v[k];
        }
    }
    // team-private buffer: vector q of lane t in segment s at ((s K/V + q) LW + t) V
    static __device__ __forceinline__ void sput(real *buf, int s, int t, int LW, const real (&v)[K])
    {
#pragma unroll
        for (int q = 0; q < K / V; ++q) {
            real *p = buf + ((size_t)(s * (K / V) + q) * LW + t) * V;
            if constexpr (sizeof(real) == 4)
                *reinterpret_cast<float4 *>(p) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            else
                *reinterpret_cast<double2 *>(p) = make_double2(v[2 * q], v[2 * q + 1]);
        }
    }
    static __device__ __forceinline__ void sget(const real *buf, int s, int t, int LW, real (&v)[K])
    {
#pragma unroll
        for (int q = 0; q < K / V; ++q) {
            const real *p = buf + ((size_t)(s * (K / V) + q) * LW + t) * V;
            if constexpr (sizeof(real) == 4) {
                const float4 a = *reinterpret_cast<const float4 *>(p);
                v[4 * q] = a.x, v[4 * q + 1] = a.y, v[4 * q + 2] = a.z, v[4 * q + 3] = a.w;
            } else {
                const double2 a = *reinterpret_cast<const double2 *>(p);
                v[2 * q] = a.x, v[2 * q + 1] = a.y;
            }
        }
    }
};

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// Four reals of a table (16-byte aligned for float, two 16-byte loads for double).
template <typename real>
__device__ __forceinline__ void rl_ld4(const real *__restrict__ p, real &a, real &b, real &c, real &d)
{
    if constexpr (sizeof(real) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        a = v.x, b = v.y, c = v.z, d = v.w;
    } else {
        const double2 u = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p + 2));
        a = u.x, b = u.y, c = v.x, d = v.y;
    }
}

template <typename real, int K, int R, int MODE>
__global__ void __launch_bounds__(128) rline_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    static_assert(MODE == MODE_LIT || MODE == MODE_DELTA, "the line kernel runs the literal and increment forms");
    using IO = RLineIO<real, K>;
    constexpr bool LIT = MODE == MODE_LIT;
    pdl_launch_dependents();
    pdl_wait();
    const SweepArgs<real> &A = args[blockIdx.y];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    const int Nr = A.Nr, Nz = A.Nz;
    const RLine<real> &RL = A.rl;
    const int LW = RL.LW, nseg = RL.nseg;
    const int nchunk = nseg * LW;
    const int Npad = nchunk * K;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tpw = 32 / LW, team = lane / LW, t = lane % LW;
    const int NW = blockDim.x >> 5;
    const long long T = (long long)gridDim.x * NW * tpw;
    const long long g = ((long long)blockIdx.x * NW + w) * tpw + team;
    const int nu = RL.n_units;
    const int u0 = (int)(g * nu / T), u1 = (int)((g + 1) * nu / T);
    const int nl = u1 - u0;
    const int nlmax = __reduce_max_sync(0xffffffffu, nl);
    if (nlmax == 0) return;  // warp-uniform
    extern __shared__ __align__(16) unsigned char rl_smem[];
    real *buf = reinterpret_cast<real *>(rl_smem) + ((size_t)w * tpw + team) * R * Npad;
    const bool vec = (Nr % IO::V) == 0;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;
    const LineTab<real> &Z = A.Z;
    const real bc0 = LIT ? real(0) : (real)A.bc.th[0], bc1 = LIT ? real(0) : (real)A.bc.th[1];
    const real bc2 = LIT ? real(0) : (real)A.bc.th[2], bc3 = LIT ? real(0) : (real)A.bc.th[3];
    const unsigned FULL = 0xffffffffu;

    for (int it = 0; it < nlmax; ++it) {
        const bool act = it < nl;
        const int unit = RL.unit[act ? u0 + it : (nl > 0 ? u1 - 1 : 0)];  // idle teams redo a valid unit
        const int j0 = unit & 0xffff, nrow = act ? unit >> 16 : 0;     // rows j0 .. j0+nrow-1 stored
        const int a = rowcls[j0];
        const real *__restrict__ tA = RL.tA + (size_t)a * Npad * 4;
        const real *__restrict__ tB = RL.tB + (size_t)a * Npad * 2;
        const real *__restrict__ tD = RL.tD + (size_t)a * Npad * 2;
        const real *__restrict__ tC = RL.tC + (size_t)a * nchunk * 12;
        // rows j0-1 .. j0+R: x[q] = row j0-1+q (ghost rows beyond the z faces)
        const real *rowp[R + 2];
        bool rin[R + 2];
#pragma unroll
        for (int q = 0; q < R + 2; ++q) {
            const int r = j0 - 1 + q;
            rin[q] = r >= 0 && r < Nz;
            rowp[q] = th + (size_t)(rin[q] ? r : j0) * Nr;
        }
        real Dseg[R], left[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Dseg[r] = real(0), left[r] = bc0;
#pragma unroll 1
        for (int s = 0; s < nseg; ++s) {
            const int i0 = (s * LW + t) * K;
            if (i0 < Nr)
#pragma unroll
                for (int q = 0; q < R + 2; ++q)
                    if (rin[q]) prefetch_l2(rowp[q] + i0);
        }

        // ---- walk 1: right-hand sides, forward summaries, scans, forward recurrences
#pragma unroll 1
        for (int s = 0; s < nseg; ++s) {
            const int c = s * LW + t;
            const int i0 = c * K;
            real x[R + 2][K];
#pragma unroll
            for (int q = 0; q < R + 2; ++q) {
                if (rin[q]) IO::load(rowp[q], i0, Nr, vec, (q >= 1 && q <= R) ? bc1 : real(0), x[q]);
                else IO::fill(q == 0 ? bc2 : bc3, x[q]);
            }
            // z coefficients of each row: one value per row for a chunk inside one
            // column class (the chunk's first cell's class otherwise; the cells of
            // another class are redone below)
            const int zc = RL.zcl[c];
            const int zc0 = zc >= 0 ? zc : (i0 < Nr ? colcls[i0] : 0);
            real zm[R], zp[R], zd[R], zs[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const size_t zo = (size_t)zc0 * Nz + min(j0 + r, Nz - 1);
                zd[r] = zs[r] = real(0);
                if constexpr (LIT) zm[r] = Z.am[zo], zp[r] = Z.ap[zo], zd[r] = Z.ad[zo], zs[r] = Z.sd[zo];
                else zm[r] = Z.xm[zo], zp[r] = Z.xp[zo];
            }
            // right neighbour of the last cell of the lane: next lane's first cell,
            // for the team's last lane the next segment's first cell (or the ghost)
            real nl_[R], nr_[R];
            if constexpr (!LIT) {
                const bool more = i0 + K < Nr;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    nl_[r] = __shfl_up_sync(FULL, x[r + 1][K - 1], 1, LW);
                    nr_[r] = __shfl_down_sync(FULL, x[r + 1][0], 1, LW);
                    if (t == 0) nl_[r] = left[r];
                    if (t == LW - 1) nr_[r] = more ? rowp[r + 1][i0 + K] : bc1;
                    left[r] = __shfl_sync(FULL, x[r + 1][K - 1], LW - 1, LW);
                }
            }
            // right-hand side of cell k of row r with z coefficients (y0..y3)
            auto rhs = [&](int r, int k, real a0, real a1, real a2, real y0, real y1, real y2, real y3) {
                const real xc = x[r + 1][k];
                if constexpr (LIT) {
                    // {w, s, -, inv}: (w + ad_z) x + am_z x_{j-1} + ap_z x_{j+1} + s + sd_z
                    return fmad(a0 + y2, xc, fmad(y0, x[r][k], fmad(y1, x[r + 2][k], a1 + y3)));
                } else {
                    // {xm, xp, q, inv}: every coupling applied to a difference
                    const real l = k > 0 ? x[r + 1][k - 1] : nl_[r];
                    const real rr = k < K - 1 ? x[r + 1][k + 1] : nr_[r];
                    real v = fmad(a0, l - xc, a2);
                    v = fmad(a1, rr - xc, v);
                    v = fmad(y0, x[r][k] - xc, v);
                    return fmad(y1, x[r + 2][k] - xc, v);
                }
            };
            real d[R][K], iv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                real a0, a1, a2, a3;
                rl_ld4(tA + (size_t)(i0 + k) * 4, a0, a1, a2, a3);
                iv[k] = a3;
#pragma unroll
                for (int r = 0; r < R; ++r) d[r][k] = rhs(r, k, a0, a1, a2, zm[r], zp[r], zd[r], zs[r]);
            }
            if (zc < 0) {
                // a chunk across a column-class boundary (layer interface): the
                // cells of another class again, with their own z coefficients
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = i0 + k;
                    const int cc = i < Nr ? colcls[i] : zc0;
                    if (cc != zc0) {
                        real a0, a1, a2, a3;
                        rl_ld4(tA + (size_t)i * 4, a0, a1, a2, a3);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const size_t zo = (size_t)cc * Nz + min(j0 + r, Nz - 1);
                            real y0, y1, y2 = real(0), y3 = real(0);
                            if constexpr (LIT) y0 = Z.am[zo], y1 = Z.ap[zo], y2 = Z.ad[zo], y3 = Z.sd[zo];
                            else y0 = Z.xm[zo], y1 = Z.xp[zo];
                            d[r][k] = rhs(r, k, a0, a1, a2, y0, y1, y2, y3);
                        }
                    }
                }
            }
            // forward summaries of the chunk and the team scans
            real fk[K], B[R];
#pragma unroll
            for (int r = 0; r < R; ++r) B[r] = real(0);
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                real f0, w0, f1, w1;
                rl_ld4(tB + (size_t)(i0 + k) * 2, f0, w0, f1, w1);
                fk[k] = f0, fk[k + 1] = f1;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    B[r] = fmad(d[r][k], w0, B[r]);
                    B[r] = fmad(d[r][k + 1], w1, B[r]);
                }
            }
            // scan constants {m0..m4, Fe, n0..n4, He} of the chunk
            real ms[5], Fe, u0_, u1_;
            rl_ld4(tC + (size_t)c * 12, ms[0], ms[1], ms[2], ms[3]);
            rl_ld4(tC + (size_t)c * 12 + 4, ms[4], Fe, u0_, u1_);
#pragma unroll
            for (int l = 0; l < 5; ++l)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const real b2 = __shfl_up_sync(FULL, B[r], 1 << l, LW);
                    B[r] = fmad(ms[l], b2, B[r]);
                }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                real Be = __shfl_up_sync(FULL, B[r], 1, LW);
                if (t == 0) Be = real(0);
                real y = fmad(Fe, Dseg[r], Be);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    y = fmad(d[r][k], iv[k], fk[k] * y);
                    d[r][k] = y;
                }
                IO::sput(buf + (size_t)r * Npad, s, t, LW, d[r]);
                Dseg[r] = __shfl_sync(FULL, y, LW - 1, LW);
            }
        }

        // ---- walk 2: backward summaries, scans, backward recurrences, store
        real Xseg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Xseg[r] = real(0);
#pragma unroll 1
        for (int s = nseg - 1; s >= 0; --s) {
            const int c = s * LW + t;
            const int i0 = c * K;
            real base[R][K];
            if constexpr (!LIT)
#pragma unroll
                for (int r = 0; r < R; ++r) IO::load(rowp[r + 1], i0, Nr, vec, real(0), base[r]);
            real y[R][K], cp[K], G[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                IO::sget(buf + (size_t)r * Npad, s, t, LW, y[r]);
                G[r] = real(0);
            }
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                real c0, w0, c1, w1;
                rl_ld4(tD + (size_t)(i0 + k) * 2, c0, w0, c1, w1);
                cp[k] = c0, cp[k + 1] = c1;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    G[r] = fmad(y[r][k], w0, G[r]);
                    G[r] = fmad(y[r][k + 1], w1, G[r]);
                }
            }
            real ns[5], He, u0_, u1_;
            rl_ld4(tC + (size_t)c * 12 + 4, u0_, u1_, ns[0], ns[1]);
            rl_ld4(tC + (size_t)c * 12 + 8, ns[2], ns[3], ns[4], He);
#pragma unroll
            for (int l = 0; l < 5; ++l)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const real g2 = __shfl_down_sync(FULL, G[r], 1 << l, LW);
                    G[r] = fmad(ns[l], g2, G[r]);
                }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                real Ge = __shfl_down_sync(FULL, G[r], 1, LW);
                if (t == LW - 1) Ge = real(0);
                real xv = fmad(He, Xseg[r], Ge);
#pragma unroll
                for (int k = K - 1; k >= 0; --k) {
                    xv = fmad(cp[k], xv, y[r][k]);
                    y[r][k] = xv;
                }
                Xseg[r] = __shfl_sync(FULL, xv, 0, LW);
                if (r < nrow) {
                    if constexpr (!LIT) {
#pragma unroll
                        for (int k = 0; k < K; ++k) y[r][k] = base[r][k] + y[r][k];
                    }
                    IO::store(out + (size_t)(j0 + r) * Nr, i0, Nr, vec, y[r]);
                }
            }
        }
    }
}

}  // namespace heat
