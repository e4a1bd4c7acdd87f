// heat_rblock.cuh -- the r-sweep of the increment form (half-step 1 of the
// Peaceman-Rachford step, Sec. 3, eq. "scheme_eq_1") with every r-line held
// on chip by a group of G threads, K consecutive cells each (G K >= Nr).
//
// A block holds 256 / G line slots (or one line of G <= 256 threads); slot s
// walks a band of consecutive rows.  The line matrix is fixed per row class,
// so each thread keeps its K cells' coefficients {xm, xp, q, inv} in
// registers for as long as the rows it walks keep their class, pre-scaled by
// the pivot: xm inv (= the Thomas multiplier f), xp inv (= cp), q inv, inv
// (at the line ends f and cp multiply a zero carry, so the folded Dirichlet
// couplings there do no harm); the right-hand side is formed times inv, so
// each recurrence step is one FMA.
// A pass solves n = 2 rows of one class (1 at a class change):
//   right-hand side of every cell (rows j-1, j, j+1, j+2 from the ring);
//   forward: chunk summary B (recurrence from a zero carry), team scan of
//     the maps y -> B + F y (F = prod f of the chunk) with multipliers
//     precomputed per class, warps of a wide line joined through shared
//     memory, then the chunk recurrence from its carry;
//   backward: the same with G (recurrence from a zero carry) and H = prod cp;
//   new value theta + x stored.
// Rows reach shared memory through a ring of NRING rows per slot filled with
// cp.async, each thread copying and later reading only its own cells, so the
// ring needs no block barrier; row j+1..j+NRING-2 are in flight while row j is
// solved.  The neighbours of a thread's first / last cell come from the next
// lanes by shuffles, across a warp boundary from global memory.
// EXACT: the lines fill their threads exactly (Nr = G K, rows 16-byte
// aligned), so no cell needs a range check; passes away from the z faces
// read their rows without checks either.  Wide lines
// join their warps with one named barrier per direction and pass.
#pragma once

#include "heat_internal.h"

namespace heat {

__device__ __forceinline__ void rb_cp16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void rb_cp4(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void rb_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p)); }
template <int N>
__device__ __forceinline__ void rb_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
__device__ __forceinline__ void rb_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// rows per pass as a type (the pass is a generic lambda)
template <int N>
struct RbRows {
    static constexpr int value = N;
};

// BYVAL: one instance, whose arguments are read from the by-value parameter a1
// (the constant bank) rather than from args in global memory.
template <int K, int NRING, bool EXACT, bool BYVAL>
__global__ void __launch_bounds__(256, 2)
    rblock_kernel(const SweepArgs<float> *__restrict__ args, int flip, const __grid_constant__ SweepArgs<float> a1)
{
    using real = float;
    const SweepArgs<real> &A = BYVAL ? a1 : args[blockIdx.y];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    const int Nr = A.Nr, Nz = A.Nz, G = A.G;
    const int tid = threadIdx.x;
    const int lpb = blockDim.x / G;
    const int slot = tid / G, g = tid % G;
    const int W = G < 32 ? G : 32;
    const int lane = tid & 31, ls = tid % W;
    const int wil = g >> 5;  // warp index within a wide line
    const int nwl = G >> 5;  // warps per wide line
    const bool wide = G > 32;
    // the slot's band: rows [jstart, jstart + band) (stored below Nz); with
    // row-class runs (lines of whole warps, so a warp holds one slot) the
    // bands of run r start at run_lo[r]
    const int sid = blockIdx.x * lpb + slot;
    int jstart, band = A.band, a0;  // a0: row class of the band's first row
    pdl_launch_dependents();
    if (A.rb_runs) {
        if (sid >= A.run_slot[A.n_run]) return;  // a slot past the last band (warp-uniform)
        int r = 0;
        while (r + 1 < A.n_run && sid >= A.run_slot[r + 1]) ++r;
        jstart = A.run_lo[r] + (sid - A.run_slot[r]) * band;
        band = min(band, A.run_lo[r + 1] - jstart);
        a0 = A.run_cls[r];
    } else {
        jstart = sid * band;
        if ((int)blockIdx.x * lpb * band >= Nz) return;  // past this instance (block-uniform)
        a0 = A.rowcls[min(jstart, Nz - 1)];
    }
    const int jend = min(Nz, jstart + band);  // rows this slot stores: [jstart, jend)
    const int i0 = g * K;
    const bool vec = EXACT || (Nr & 3) == 0;
    static_assert((NRING & (NRING - 1)) == 0, "the ring length is a power of two");
    const unsigned FULL = 0xffffffffu;
    const real bc0 = (real)A.bc.th[0], bc1 = (real)A.bc.th[1];
    const real bc2 = (real)A.bc.th[2], bc3 = (real)A.bc.th[3];
    const LineTab<real> &R = A.R, &Z = A.Z;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;

    extern __shared__ __align__(16) unsigned char rb_smem[];
    const int Np = G * K;
    real *ring = reinterpret_cast<real *>(rb_smem) + (size_t)slot * NRING * Np + i0;  // this thread's cells
    __shared__ real sxF[8][8], sxB[2][8][8], sxH[8][8], sxG[2][8][8];  // [slot][warp] (wide lines: <= 4 slots)
    const int bar_id = 1 + slot;

    // this thread's K cells of row x into its ring slot (zero past the field)
    // (rows past jstart + band, which no pass of the slot reads, commit an
    // empty group)
    auto fetch = [&](int x) {
        real *dst = ring + (size_t)((x - jstart + 1) & (NRING - 1)) * Np;  // x >= jstart - 1
        if (x > jstart + band) {
            rb_commit();
            return;
        }
        const bool rin = x >= 0 && x < Nz;
        const real *src = th + (size_t)(rin ? x : 0) * Nr;
        if (vec) {
#pragma unroll
            for (int k = 0; k < K; k += 4) {
                const bool ok = rin && (EXACT || i0 + k < Nr);
                rb_cp16(dst + k, ok ? src + i0 + k : th, ok ? 16 : 0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool ok = rin && i0 + k < Nr;
                rb_cp4(dst + k, ok ? src + i0 + k : th, ok ? 4 : 0);
            }
        }
        rb_commit();
    };
    // column class of the thread's cells: one for all K, or per cell (a chunk
    // across a layer interface)
    // zc0: class of the first cell, zc1: of the last cell inside the field;
    // bit k of zsel set for cells of class zc1 (!= zc0); zmany when a cell has
    // a third class (a layer thinner than K cells), whose cells are redone
    const int zc0 = i0 < Nr ? colcls[i0] : 0;
    int zc1 = zc0;
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (i0 + k < Nr) zc1 = colcls[i0 + k];
    unsigned zsel = 0;
    bool zmany = false;  // (then zany: for some lane of the warp)
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (i0 + k < Nr) {
            const int c = colcls[i0 + k];
            if (c == zc1 && c != zc0) zsel |= 1u << k;
            zmany = zmany || (c != zc0 && c != zc1);
        }
    bool zany, zone;  // (set below) some cell of the warp has a third class; one column class in every chunk of the warp

    // class state: the coefficients scaled by the pivot, fx = xm inv (also
    // the Thomas multiplier f), cx = xp inv (also cp), qi = q inv, and inv
    int acls = -1;
    real fx[K], cx[K], qi[K], iv[K];
    real Fc = real(1), Hc = real(1);  // products of f and cp over the chunk
    real m[5], Fe = real(1), n[5], He = real(1);
    // wide lines: lane v's multiplier of warp v's forward map into this
    // warp's carry, prod of F over the warps between (0 for v >= wil), and
    // of warp v's backward map, prod of H over the warps between (0 for v <= wil)
    real jf = real(0), jh = real(0);

    // the coefficients of class a as stored (issued together; used by class_finish)
    auto class_loads = [&](int a) {
        const size_t ro = (size_t)a * Nr;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = i0 + k;
            const bool in = i < Nr;
            iv[k] = in ? R.inv[ro + i] : real(0);
            fx[k] = in ? R.xm[ro + i] : real(0);
            cx[k] = in ? R.xp[ro + i] : real(0);
            qi[k] = in ? R.q[ro + i] : real(0);
        }
        acls = a;
    };
    // scale them by the pivot and form the scan multipliers (all threads of the slot)
    auto class_finish = [&]() {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            fx[k] *= iv[k];
            cx[k] *= iv[k];
            qi[k] *= iv[k];
        }
        Fc = Hc = real(1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            Fc *= fx[k];
            Hc *= cx[k];
        }
        // level multipliers of the team scans: m_l = prod F over lanes ls-2^l+1..ls
        // (0 below 2^l), n_l = prod H over lanes ls..ls+2^l-1 (0 past the team)
        real pf = Fc, ph = Hc;
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int off = 1 << l;
            m[l] = ls >= off ? pf : real(0);
            n[l] = ls + off < W ? ph : real(0);
            const real pf2 = __shfl_up_sync(FULL, pf, off, W);
            const real ph2 = __shfl_down_sync(FULL, ph, off, W);
            if (off < W) {
                pf = ls >= off ? pf * pf2 : pf;
                ph = ls + off < W ? ph * ph2 : ph;
            }
        }
        // pf = prod F over lanes 0..ls, ph = prod H over lanes ls..W-1
        Fe = __shfl_up_sync(FULL, pf, 1, W);
        He = __shfl_down_sync(FULL, ph, 1, W);
        if (ls == 0) Fe = real(1);
        if (ls == W - 1) He = real(1);
        if (wide) {
            if (lane == 31) sxF[slot][wil] = pf;
            if (lane == 0) sxH[slot][wil] = ph;
        }
    };
    // (wide lines, after the barrier that publishes sxF / sxH)
    auto join_multipliers = [&]() {
        jf = jh = real(0);
        if (lane < wil) {
            jf = real(1);
            for (int u = lane + 1; u < wil; ++u) jf *= sxF[slot][u];
        }
        if (lane > wil && lane < nwl) {
            jh = real(1);
            for (int u = wil + 1; u < lane; ++u) jh *= sxH[slot][u];
        }
    };
    // sum over the first 8 lanes (the warps of a wide line are at most 8),
    // returned to every lane of the warp
    auto sum8 = [&](real v) {
        v += __shfl_xor_sync(FULL, v, 1);
        v += __shfl_xor_sync(FULL, v, 2);
        v += __shfl_xor_sync(FULL, v, 4);
        return __shfl_sync(FULL, v, 0);
    };

    // one pass over rows j .. j+NR-1 (same class); wait first for their rows
    auto pass = [&](auto nr_tag, int j) {
        constexpr int NR = decltype(nr_tag)::value;
        rb_wait<NRING - 2 - NR>();
        // rows j-1 .. j+NR from the ring (ghost rows at the z faces)
        real x[NR + 2][K];
        auto ld_row = [&](int q, int r) {
            const real *p = ring + (size_t)((r - jstart + 1) & (NRING - 1)) * Np;
#pragma unroll
            for (int k = 0; k < K; k += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(p + k);
                x[q][k] = v.x, x[q][k + 1] = v.y, x[q][k + 2] = v.z, x[q][k + 3] = v.w;
            }
        };
        if (__all_sync(FULL, j >= 1 && j + NR < Nz)) {
#pragma unroll
            for (int q = 0; q < NR + 2; ++q) ld_row(q, j - 1 + q);
        } else {
#pragma unroll
            for (int q = 0; q < NR + 2; ++q) {
                const int r = j - 1 + q;
                if (r < 0 || r >= Nz) {
#pragma unroll
                    for (int k = 0; k < K; ++k) x[q][k] = r < 0 ? bc2 : bc3;
                } else {
                    ld_row(q, r);
                }
            }
        }
        if (!EXACT && i0 + K > Nr)
#pragma unroll
            for (int q = 0; q < NR + 2; ++q)
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (i0 + k >= Nr && j - 1 + q >= 0 && j - 1 + q < Nz) x[q][k] = bc1;  // ghost past the outer r face
        // right-hand sides
        real d[NR][K];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int jr = min(j + r, Nz - 1);
            const real *xr = x[r + 1];
            real nl = __shfl_up_sync(FULL, xr[K - 1], 1, W);
            real nrt = __shfl_down_sync(FULL, xr[0], 1, W);
            if (ls == 0) nl = (i0 > 0 && (EXACT || i0 - 1 < Nr)) ? th[(size_t)jr * Nr + i0 - 1] : bc0;
            if (ls == W - 1) nrt = (i0 + K < Nr) ? th[(size_t)jr * Nr + i0 + K] : bc1;
            const size_t zo = (size_t)zc0 * Nz + jr;
            const real zmA = Z.xm[zo], zpA = Z.xp[zo];
            if (zone) {
                // every chunk of the warp has one column class
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const real xc = xr[k];
                    const real l = k > 0 ? xr[k - 1] : nl;
                    const real rr = k < K - 1 ? xr[k + 1] : nrt;
                    real v = fmad(fx[k], l - xc, qi[k]);
                    v = fmad(cx[k], rr - xc, v);
                    const real zz = fmad(zpA, x[r + 2][k] - xc, zmA * (x[r][k] - xc));
                    d[r][k] = fmad(iv[k], zz, v);
                }
            } else {
                const size_t zo1 = (size_t)zc1 * Nz + jr;
                const real zmB = Z.xm[zo1], zpB = Z.xp[zo1];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    // the right-hand side times the pivot inv
                    const real xc = xr[k];
                    const real l = k > 0 ? xr[k - 1] : nl;
                    const real rr = k < K - 1 ? xr[k + 1] : nrt;
                    real v = fmad(fx[k], l - xc, qi[k]);
                    v = fmad(cx[k], rr - xc, v);
                    const bool bsel = (zsel >> k) & 1u;
                    const real zm = bsel ? zmB : zmA, zp = bsel ? zpB : zpA;
                    const real zz = fmad(zp, x[r + 2][k] - xc, zm * (x[r][k] - xc));
                    d[r][k] = fmad(iv[k], zz, v);
                }
            }
            if (zany) {
                // the chunk crosses a column-class boundary: per-cell z coefficients
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = i0 + k;
                    if (i < Nr && colcls[i] != zc0 && colcls[i] != zc1) {
                        const size_t zk = (size_t)colcls[i] * Nz + jr;
                        const real xc = xr[k];
                        const real l = k > 0 ? xr[k - 1] : nl;
                        const real rr = k < K - 1 ? xr[k + 1] : nrt;
                        real v = fmad(fx[k], l - xc, qi[k]);
                        v = fmad(cx[k], rr - xc, v);
                        const real zz = fmad(Z.xp[zk], x[r + 2][k] - xc, Z.xm[zk] * (x[r][k] - xc));
                        d[r][k] = fmad(iv[k], zz, v);
                    }
                }
            }
        }
        // forward: chunk summaries, team scans, joins, recurrences
        real B[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real b = real(0);
#pragma unroll
            for (int k = 0; k < K; ++k) b = fmad(fx[k], b, d[r][k]);
            B[r] = b;
        }
#pragma unroll
        for (int l = 0; l < 5; ++l)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const real b2 = __shfl_up_sync(FULL, B[r], 1 << l, W);
                B[r] = fmad(m[l], b2, B[r]);
            }
        real Din[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real be = __shfl_up_sync(FULL, B[r], 1, W);
            if (ls == 0) be = real(0);
            Din[r] = be;
        }
        if (wide) {
            if (lane == 31)
#pragma unroll
                for (int r = 0; r < NR; ++r) sxB[r][slot][wil] = B[r];
            rb_bar(bar_id, G);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                // only lanes v < wil read a published slot (the others may hold garbage)
                const real D = sum8(lane < wil ? jf * sxB[r][slot][lane] : real(0));
                Din[r] = fmad(Fe, D, Din[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real y = Din[r];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                y = fmad(fx[k], y, d[r][k]);
                d[r][k] = y;
            }
        }
        // backward
        real Gs[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real gg = real(0);
#pragma unroll
            for (int k = K - 1; k >= 0; --k) gg = fmad(cx[k], gg, d[r][k]);
            Gs[r] = gg;
        }
#pragma unroll
        for (int l = 0; l < 5; ++l)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const real g2 = __shfl_down_sync(FULL, Gs[r], 1 << l, W);
                Gs[r] = fmad(n[l], g2, Gs[r]);
            }
        real Xin[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real ge = __shfl_down_sync(FULL, Gs[r], 1, W);
            if (ls == W - 1) ge = real(0);
            Xin[r] = ge;
        }
        if (wide) {
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < NR; ++r) sxG[r][slot][wil] = Gs[r];
            rb_bar(bar_id, G);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                // only lanes wil < v < nwl read a published slot
                const real X = sum8(lane > wil && lane < nwl ? jh * sxG[r][slot][lane] : real(0));
                Xin[r] = fmad(He, X, Xin[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real xv = Xin[r];
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                xv = fmad(cx[k], xv, d[r][k]);
                d[r][k] = x[r + 1][k] + xv;
            }
            if (j + r >= jend) continue;  // a row of no slot of this block (or past the field)
            real *orow = out + (size_t)(j + r) * Nr;
            if (EXACT || (vec && i0 + K <= Nr)) {
#pragma unroll
                for (int k = 0; k < K; k += 4)
                    *reinterpret_cast<float4 *>(orow + i0 + k) = make_float4(d[r][k], d[r][k + 1], d[r][k + 2], d[r][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (i0 + k < Nr) orow[i0 + k] = d[r][k];
            }
        }
        // refill the slots of rows j-1 .. j+NR-2 with rows j+NRING-1 .. j+NRING+NR-2
#pragma unroll
        for (int r = 0; r < NR; ++r) fetch(j + NRING - 1 + r);
    };

    // Start of the band.  The tables do not change between launches, so the
    // first class's coefficients, and the z coefficients of the band's rows
    // (into L1), are requested before the wait for the previous kernel and
    // ahead of the ring's rows, which would otherwise queue them behind
    // several megabytes of row traffic.
    class_loads(a0);
    {
        const int jl = min(jstart + band, Nz - 1);
        for (int x = min(jstart, Nz - 1); x <= jl; x += 16) {
            prefetch_l1(Z.xm + (size_t)zc0 * Nz + x);
            prefetch_l1(Z.xp + (size_t)zc0 * Nz + x);
            if (zc1 != zc0) {
                prefetch_l1(Z.xm + (size_t)zc1 * Nz + x);
                prefetch_l1(Z.xp + (size_t)zc1 * Nz + x);
            }
        }
    }
    zany = __any_sync(FULL, zmany);
    zone = __all_sync(FULL, zsel == 0u && !zmany);
    pdl_wait();
    // prologue: rows jstart-1 .. jstart+NRING-2
    for (int x = jstart - 1; x <= jstart + NRING - 2; ++x) fetch(x);
    class_finish();
    if (wide) {
        rb_bar(bar_id, G);
        join_multipliers();
    }

    // The slots of a warp (sub-warp lines) walk their bands in lockstep, and
    // every decision below is taken for the whole warp, so the warp's
    // shuffles always see all 32 lanes; the warps of a wide line see the same
    // rows and take the same decisions.
    for (int t = 0; t < band;) {
        const int j = jstart + t;
        const int a = rowcls[min(j, Nz - 1)];
        if (__any_sync(FULL, a != acls)) {
            if (wide) rb_bar(bar_id, G);  // nobody still reads the previous class's sxF / sxH
            class_loads(a);
            class_finish();
            if (wide) {
                rb_bar(bar_id, G);
                join_multipliers();
            }
        }
        const bool two = __all_sync(FULL, t + 1 < band && rowcls[min(j + 1, Nz - 1)] == a);
        if (two) {
            pass(RbRows<2>(), j);
            t += 2;
        } else {
            pass(RbRows<1>(), j);
            t += 1;
        }
    }
    rb_wait<0>();
}

}  // namespace heat
