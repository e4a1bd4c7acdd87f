// heat_rclus.cuh -- the r-sweep of the increment form (half-step 1 of the
// Peaceman-Rachford step, Sec. 3, eq. "scheme_eq_1") for r-lines longer than
// one block holds on chip: a thread-block cluster of CL blocks holds each
// line, block c the segment of cells [c S, (c+1) S), S = 256 K (K = 8: 2048
// cells), so lines of up to 8 S = 16384 cells stay in registers.
//
// Every block of a cluster walks the same band of rows.  Within a block the
// solve is that of the register-resident r-sweep (heat_rblock.cuh): each
// thread holds K cells with the pivot-scaled coefficients of its row class,
// forms the right-hand side times the pivot, reduces its chunk to an affine
// map, scans the maps of its warp with shuffles.  The maps of the cluster's
// warps (up to 64) are then joined through distributed shared memory: lane
// 31 (forward) or lane 0 (backward) of every warp stores its warp's map into
// a slot of every block of the cluster, one cluster barrier later every
// thread combines the slots of the warps before (forward) or after
// (backward) its own, weighted by the products of the warps' multipliers in
// between (fixed per row class, computed when the class changes).  One
// cluster barrier per direction and pass; each slot array is written only
// after the barrier that follows the last read of its previous contents.
//
// REFINE (the refined FP32 path): the line is solved twice.  After the first
// solve (delta0) the residual of the increment system at delta0 is formed in
// extended precision from FP32 pairs (exact differences, FMA products; the
// same terms as the block-line r-sweep's refined mode), and the second solve
// of that residual is added: theta + (delta0 + e).  The residual of a cell
// needs delta0 of both neighbours; across a warp edge and across a block
// edge they are exchanged through (distributed) shared memory under one
// more cluster barrier, so every cell uses the stored delta0 of its
// neighbours exactly.
#pragma once

#include "heat_internal.h"

namespace heat {

// cells per thread and threads per block of the cluster r-sweep
constexpr int kRcK = 8;
constexpr int kRcThreads = 256;
constexpr int kRcSeg = kRcK * kRcThreads;  // cells per block
constexpr int kRcMaxCl = 8;                 // portable cluster size
// rows per thread's ring (a power of two): 8 in the plain form; 4 in the
// refined form, whose blocks also stage the row class's residual pairs
template <int MODE>
__host__ __device__ constexpr int rc_ring() { return MODE == MODE_REFINE ? 4 : 8; }
// dynamic shared memory of a block: the ring, and (refined) the pairs
// q, am, ap, b of its 2048 cells
template <int MODE>
constexpr size_t rc_smem_bytes()
{
    return (size_t)rc_ring<MODE>() * kRcSeg * sizeof(float) + (MODE == MODE_REFINE ? 4 * kRcSeg * sizeof(float2) : 0);
}

__device__ __forceinline__ unsigned rc_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
// all threads of every block of the cluster; release / acquire orders the
// shared-memory stores before it against the loads after it
__device__ __forceinline__ void rc_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// address of p (this block's shared memory) in block `rank` of the cluster
__device__ __forceinline__ unsigned rc_map(const void *p, unsigned rank)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    unsigned d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(d) : "r"(s), "r"(rank));
    return d;
}
__device__ __forceinline__ void rc_st(unsigned addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;\n" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ float2 rc_ld2(const float2 *p) { return __ldg(p); }

// sum over the 32 lanes of a warp, returned to every lane
__device__ __forceinline__ float rc_wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int MODE, bool EXACT>
__global__ void __launch_bounds__(kRcThreads, 2) rclus_kernel(const SweepArgs<float> *__restrict__ args, int flip)
{
    static_assert(MODE == MODE_DELTA || MODE == MODE_REFINE, "increment forms only");
    using real = float;
    constexpr int K = kRcK, NRING = rc_ring<MODE>();
    const unsigned FULL = 0xffffffffu;
    const SweepArgs<real> &A = args[0];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    const int Nr = A.Nr, Nz = A.Nz, band = A.band;
    const int CL = A.G / kRcThreads;  // blocks per line
    const int NW = CL * 8;            // warps per line
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int c = (int)rc_rank();
    const int gw = c * 8 + w;  // warp index within the line
    const int i0 = (c * kRcThreads + tid) * K;
    const int jstart = ((int)blockIdx.x / CL) * band;
    const bool vec = EXACT || (Nr & 3) == 0;
    const real bc0 = (real)A.bc.th[0], bc1 = (real)A.bc.th[1];
    const real bc2 = (real)A.bc.th[2], bc3 = (real)A.bc.th[3];
    const LineTab<real> &R = A.R, &Z = A.Z;
    const int *__restrict__ rowcls = A.rowcls;
    const int *__restrict__ colcls = A.colcls;
    pdl_launch_dependents();
    // every block of the cluster has started before anyone stores into its shared memory
    rc_sync();
    if (jstart >= Nz) return;  // the same for every block of the cluster
    const int nrow = min(band, Nz - jstart);

    extern __shared__ __align__(16) unsigned char rc_smem[];
    real *ring = reinterpret_cast<real *>(rc_smem) + tid * K;  // this thread's cells of ring row 0
    // REFINE: pairs of the class, [array q, am, ap, b][pair of cells v][thread]
    // as float4 (cells 2v, 2v+1 of the thread), so that a warp's reads of one
    // (array, v) are consecutive 16-byte words
    float4 *pairs = reinterpret_cast<float4 *>(rc_smem + (size_t)NRING * kRcSeg * sizeof(real));
    __shared__ real sFw[8 * kRcMaxCl], sHw[8 * kRcMaxCl];       // products of f / cp over each warp's cells
    __shared__ real sB[2][8 * kRcMaxCl], sG[2][8 * kRcMaxCl];   // forward / backward warp maps of the pass
    __shared__ real sLo[8], sHi[8], sEL, sER;                   // REFINE: delta0 at warp and block edges

    // this thread's K cells of row x into its ring slot (zero past the field)
    auto fetch = [&](int x) {
        real *dst = ring + (size_t)((x - jstart + 1) & (NRING - 1)) * kRcSeg;  // x >= jstart - 1
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
    // column classes of the thread's cells, as in the register-resident r-sweep:
    // zc0 (first cell), zc1 (last cell in the field), zsel (cells of zc1),
    // zmany / zany (a third class in the chunk, for some lane of the warp)
    const int zc0 = i0 < Nr ? colcls[i0] : 0;
    int zc1 = zc0;
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (i0 + k < Nr) zc1 = colcls[i0 + k];
    unsigned zsel = 0;
    bool zmany = false;
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (i0 + k < Nr) {
            const int cc = colcls[i0 + k];
            if (cc == zc1 && cc != zc0) zsel |= 1u << k;
            zmany = zmany || (cc != zc0 && cc != zc1);
        }
    const bool zany = __any_sync(FULL, zmany);
    pdl_wait();
    for (int x = jstart - 1; x <= jstart + NRING - 2; ++x) fetch(x);

    // class state: the pivot-scaled coefficients fx = xm inv (= f), cx = xp inv
    // (= cp), qi = q inv and inv; the lane multipliers of the warp scans; the
    // join weights of warps e = lane and e = lane + 32 of the line
    int acls = -1;
    real fx[K], cx[K], qi[K], iv[K];
    real m[5], n[5], Fe = real(1), He = real(1);
    real wf0 = real(0), wf1 = real(0), wh0 = real(0), wh1 = real(0);
    auto load_class = [&](int a) {
        const size_t ro = (size_t)a * Nr;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = i0 + k;
            const bool in = EXACT || i < Nr;
            iv[k] = in ? R.inv[ro + i] : real(0);
            fx[k] = in ? R.xm[ro + i] * iv[k] : real(0);
            cx[k] = in ? R.xp[ro + i] * iv[k] : real(0);
            qi[k] = in ? R.q[ro + i] * iv[k] : real(0);
        }
        if constexpr (MODE == MODE_REFINE) {
            // this thread's cells only: read back by the same thread
            const float2 *src[4] = {A.R2.q, A.R2.am, A.R2.ap, A.R2.b};
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int v = 0; v < K / 2; ++v) {
                    const int i = i0 + 2 * v;
                    const float2 a0 = (EXACT || i < Nr) ? __ldg(src[t] + ro + i) : make_float2(0.f, 0.f);
                    const float2 a1 = (EXACT || i + 1 < Nr) ? __ldg(src[t] + ro + i + 1) : make_float2(0.f, 0.f);
                    pairs[(t * (K / 2) + v) * kRcThreads + tid] = make_float4(a0.x, a0.y, a1.x, a1.y);
                }
        }
        real pf = real(1), ph = real(1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            pf *= fx[k];
            ph *= cx[k];
        }
        // m_l = prod F over lanes lane-2^l+1 .. lane (0 below 2^l),
        // n_l = prod H over lanes lane .. lane+2^l-1 (0 past the warp)
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int off = 1 << l;
            m[l] = lane >= off ? pf : real(0);
            n[l] = lane + off < 32 ? ph : real(0);
            const real pf2 = __shfl_up_sync(FULL, pf, off);
            const real ph2 = __shfl_down_sync(FULL, ph, off);
            pf = lane >= off ? pf * pf2 : pf;
            ph = lane + off < 32 ? ph * ph2 : ph;
        }
        // pf = prod F over lanes 0..lane, ph = prod H over lanes lane..31
        Fe = __shfl_up_sync(FULL, pf, 1);
        He = __shfl_down_sync(FULL, ph, 1);
        if (lane == 0) Fe = real(1);
        if (lane == 31) He = real(1);
        // every block gets every warp's products (the previous class's were
        // last read before the barriers of the pass that followed)
        if (lane == 31)
            for (int q = 0; q < CL; ++q) rc_st(rc_map(&sFw[gw], q), pf);
        if (lane == 0)
            for (int q = 0; q < CL; ++q) rc_st(rc_map(&sHw[gw], q), ph);
        rc_sync();
        // weight of warp e's forward map in this warp's carry: prod of F over
        // the warps between (e < gw); of its backward map: prod of H (e > gw)
        auto wf = [&](int e) {
            real p = real(0);
            if (e < gw) {
                p = real(1);
                for (int u = e + 1; u < gw; ++u) p *= sFw[u];
            }
            return p;
        };
        auto wh = [&](int e) {
            real p = real(0);
            if (e > gw && e < NW) {
                p = real(1);
                for (int u = gw + 1; u < e; ++u) p *= sHw[u];
            }
            return p;
        };
        wf0 = wf(lane);
        wf1 = wf(lane + 32);
        wh0 = wh(lane);
        wh1 = wh(lane + 32);
        acls = a;
    };

    // Solve the line systems of NR rows in place: d holds the right-hand
    // sides times the pivot, on return the solution (two cluster barriers).
    auto solve = [&](auto nr_tag, real(&d)[2][K]) {
        constexpr int NR = decltype(nr_tag)::value;
        // forward: chunk summaries from a zero carry, warp scans
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
                const real b2 = __shfl_up_sync(FULL, B[r], 1 << l);
                B[r] = fmad(m[l], b2, B[r]);
            }
        // the warp's inclusive maps to the blocks whose warps follow
        if (lane == 31)
            for (int q = c; q < CL; ++q)
#pragma unroll
                for (int r = 0; r < NR; ++r) rc_st(rc_map(&sB[r][gw], q), B[r]);
        real Din[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const real be = __shfl_up_sync(FULL, B[r], 1);
            Din[r] = lane == 0 ? real(0) : be;
        }
        rc_sync();
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            // only slots of warps before this one were written in this pass
            real v = lane < gw ? wf0 * sB[r][lane] : real(0);
            if (lane + 32 < gw) v = fmad(wf1, sB[r][lane + 32], v);
            Din[r] = fmad(Fe, rc_wsum(v), Din[r]);
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
                const real g2 = __shfl_down_sync(FULL, Gs[r], 1 << l);
                Gs[r] = fmad(n[l], g2, Gs[r]);
            }
        if (lane == 0)
            for (int q = 0; q <= c; ++q)
#pragma unroll
                for (int r = 0; r < NR; ++r) rc_st(rc_map(&sG[r][gw], q), Gs[r]);
        real Xin[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const real ge = __shfl_down_sync(FULL, Gs[r], 1);
            Xin[r] = lane == 31 ? real(0) : ge;
        }
        rc_sync();
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            // only slots of warps after this one were written in this pass
            real v = (lane > gw && lane < NW) ? wh0 * sG[r][lane] : real(0);
            if (lane + 32 > gw && lane + 32 < NW) v = fmad(wh1, sG[r][lane + 32], v);
            Xin[r] = fmad(He, rc_wsum(v), Xin[r]);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            real xv = Xin[r];
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                xv = fmad(cx[k], xv, d[r][k]);
                d[r][k] = xv;
            }
        }
    };

    // row r of the field from this thread's ring slot into v; ghost values
    // at the z faces (r outside the field) and past the outer r face
    auto ring_row = [&](int r, real(&v)[K]) {
        if (r < 0 || r >= Nz) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = r < 0 ? bc2 : bc3;
            return;
        }
        const real *p = ring + (size_t)((r - jstart + 1) & (NRING - 1)) * kRcSeg;
#pragma unroll
        for (int k = 0; k < K; k += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p + k);
            v[k] = q.x, v[k + 1] = q.y, v[k + 2] = q.z, v[k + 3] = q.w;
        }
        if (!EXACT && i0 + K > Nr)
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (i0 + k >= Nr) v[k] = bc1;
    };
    // theta of row jr at the chunk's outer neighbours (shuffles; across a
    // warp edge from global memory; ghosts at the r faces)
    auto row_nb = [&](int jr, const real(&xc)[K], real &nl, real &nrt) {
        nl = __shfl_up_sync(FULL, xc[K - 1], 1);
        nrt = __shfl_down_sync(FULL, xc[0], 1);
        if (lane == 0) nl = (i0 > 0 && (EXACT || i0 - 1 < Nr)) ? th[(size_t)jr * Nr + i0 - 1] : bc0;
        if (lane == 31) nrt = (i0 + K < Nr) ? th[(size_t)jr * Nr + i0 + K] : bc1;
    };
    // right-hand side of row jr times the pivot, from rows jr-1, jr, jr+1
    auto row_rhs = [&](int jr, const real(&xm)[K], const real(&xc)[K], const real(&xp)[K], real(&d)[K], real nl,
                       real nrt) {
        const size_t zo = (size_t)zc0 * Nz + jr, zo1 = (size_t)zc1 * Nz + jr;
        const real zmA = Z.xm[zo], zpA = Z.xp[zo], zmB = Z.xm[zo1], zpB = Z.xp[zo1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const real t0 = xc[k];
            const real l = k > 0 ? xc[k - 1] : nl;
            const real rr = k < K - 1 ? xc[k + 1] : nrt;
            real v = fmad(fx[k], l - t0, qi[k]);
            v = fmad(cx[k], rr - t0, v);
            const bool bsel = (zsel >> k) & 1u;
            const real zm = bsel ? zmB : zmA, zp = bsel ? zpB : zpA;
            const real zz = fmad(zp, xp[k] - t0, zm * (xm[k] - t0));
            d[k] = fmad(iv[k], zz, v);
        }
        if (zany) {
            // a chunk with a third column class: per-cell z coefficients
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                if (i < Nr && colcls[i] != zc0 && colcls[i] != zc1) {
                    const size_t zk = (size_t)colcls[i] * Nz + jr;
                    const real t0 = xc[k];
                    const real l = k > 0 ? xc[k - 1] : nl;
                    const real rr = k < K - 1 ? xc[k + 1] : nrt;
                    real v = fmad(fx[k], l - t0, qi[k]);
                    v = fmad(cx[k], rr - t0, v);
                    const real zz = fmad(Z.xp[zk], xp[k] - t0, Z.xm[zk] * (xm[k] - t0));
                    d[k] = fmad(iv[k], zz, v);
                }
            }
        }
    };
    auto store_row = [&](int jr, const real(&v)[K]) {
        real *orow = out + (size_t)jr * Nr;
        if (EXACT || (vec && i0 + K <= Nr)) {
#pragma unroll
            for (int k = 0; k < K; k += 4)
                *reinterpret_cast<float4 *>(orow + i0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (i0 + k < Nr) orow[i0 + k] = v[k];
        }
    };

    if constexpr (MODE == MODE_DELTA) {
        // one pass over rows j .. j+NR-1 (same class)
        auto pass = [&](auto nr_tag, int j) {
            constexpr int NR = decltype(nr_tag)::value;
            rb_wait<NRING - 2 - NR>();
            real x[NR + 2][K];
#pragma unroll
            for (int q = 0; q < NR + 2; ++q) ring_row(j - 1 + q, x[q]);
            real d[2][K];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                real nl, nrt;
                row_nb(j + r, x[r + 1], nl, nrt);
                row_rhs(j + r, x[r], x[r + 1], x[r + 2], d[r], nl, nrt);
            }
            solve(nr_tag, d);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
#pragma unroll
                for (int k = 0; k < K; ++k) d[r][k] = x[r + 1][k] + d[r][k];
                store_row(j + r, d[r]);
            }
            // refill the slots of rows j-1 .. j+NR-2 with rows j+NRING-1 .. j+NRING+NR-2
#pragma unroll
            for (int r = 0; r < NR; ++r) fetch(j + NRING - 1 + r);
        };
        for (int t = 0; t < nrow;) {
            const int j = jstart + t;
            const int a = rowcls[j];
            if (a != acls) load_class(a);  // the same rows, so the same decision, in every block
            if (t + 1 < nrow && rowcls[j + 1] == a) {
                pass(RbRows<2>(), j);
                t += 2;
            } else {
                pass(RbRows<1>(), j);
                t += 1;
            }
        }
    } else {
        // Refined rows, software-pipelined along the band: the correction
        // solve of row j and the first solve of row j+1 (same class) share one
        // two-row solve, so a row costs the delta0 exchange and one solve's
        // two cluster barriers.  dl0 carries delta0 of row j into its step.
        const LineTab2 &Z2 = A.Z2;
        real dl0[K];
        bool have = false;
        for (int t = 0; t < nrow; ++t) {
            const int j = jstart + t;
            const int a = rowcls[j];
            if (a != acls) load_class(a);  // no row of the previous class is in flight
            real x[3][K];
            real nl, nrt;
            if (!have) {
                // the first row of a run of one class: its first solve alone
                rb_wait<0>();
                ring_row(j - 1, x[0]);
                ring_row(j, x[1]);
                ring_row(j + 1, x[2]);
                real d[2][K];
                row_nb(j, x[1], nl, nrt);
                row_rhs(j, x[0], x[1], x[2], d[0], nl, nrt);
                solve(RbRows<1>(), d);
#pragma unroll
                for (int k = 0; k < K; ++k) dl0[k] = d[0][k];
            }
            // delta0 of the neighbours of the chunk's end cells: within the
            // warp by shuffles, across warps and blocks through shared memory
            if (lane == 0) {
                sLo[w] = dl0[0];
                if (w == 0 && c > 0) rc_st(rc_map(&sER, c - 1), dl0[0]);
            }
            if (lane == 31) {
                sHi[w] = dl0[K - 1];
                if (w == 7 && c < CL - 1) rc_st(rc_map(&sEL, c + 1), dl0[K - 1]);
            }
            real xl = __shfl_up_sync(FULL, dl0[K - 1], 1);
            real xr = __shfl_down_sync(FULL, dl0[0], 1);
            const size_t zo = (size_t)zc0 * Nz + j, zo1 = (size_t)zc1 * Nz + j;
            const float2 zmA = rc_ld2(Z2.am + zo), zpA = rc_ld2(Z2.ap + zo);
            const float2 zmB = rc_ld2(Z2.am + zo1), zpB = rc_ld2(Z2.ap + zo1);
            rc_sync();
            if (lane == 0) xl = w > 0 ? sHi[w - 1] : (c > 0 ? sEL : real(0));
            if (lane == 31) xr = w < 7 ? sLo[w + 1] : (c < CL - 1 ? sER : real(0));
            // residual of the increment system of row j at delta0, from the
            // FP64 coefficients as FP32 pairs: q + sum c (t_nb - t) - b delta0
            // + am delta0_{i-1} + ap delta0_{i+1} (the matrix's off-diagonals
            // are the couplings am, ap themselves)
            ring_row(j - 1, x[0]);
            ring_row(j, x[1]);
            ring_row(j + 1, x[2]);
            row_nb(j, x[1], nl, nrt);
            real d[2][K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                d[0][k] = real(0);
                if (!EXACT && i >= Nr) continue;
                const real t0 = x[1][k];
                const real tl = i == 0 ? t0 : (k > 0 ? x[1][k - 1] : nl);
                const real tr = i == Nr - 1 ? t0 : (k < K - 1 ? x[1][k + 1] : nrt);
                const int sv = (k >> 1) * kRcThreads + tid, hi = k & 1;
                const float4 Q4 = pairs[0 * (K / 2) * kRcThreads + sv], M4 = pairs[1 * (K / 2) * kRcThreads + sv];
                const float4 P4 = pairs[2 * (K / 2) * kRcThreads + sv], B4 = pairs[3 * (K / 2) * kRcThreads + sv];
                const float2 q2 = hi ? make_float2(Q4.z, Q4.w) : make_float2(Q4.x, Q4.y);
                const float2 am2 = hi ? make_float2(M4.z, M4.w) : make_float2(M4.x, M4.y);
                const float2 ap2 = hi ? make_float2(P4.z, P4.w) : make_float2(P4.x, P4.y);
                const float2 b2 = hi ? make_float2(B4.z, B4.w) : make_float2(B4.x, B4.y);
                Pair acc{q2.x, q2.y};
                pair_add_cdiff(acc, am2, tl, t0);
                pair_add_cdiff(acc, ap2, tr, t0);
                if (i == 0) pair_add_cdiff(acc, rc_ld2(A.R2.dl + (size_t)acls * Nr), bc0, t0);
                if (i == Nr - 1) pair_add_cdiff(acc, rc_ld2(A.R2.dh + (size_t)acls * Nr + i), bc1, t0);
                const bool bsel = (zsel >> k) & 1u;
                float2 zm = bsel ? zmB : zmA, zp = bsel ? zpB : zpA;
                size_t zk = bsel ? zo1 : zo;
                if (zany && colcls[i] != zc0 && colcls[i] != zc1) {
                    zk = (size_t)colcls[i] * Nz + j;
                    zm = rc_ld2(Z2.am + zk);
                    zp = rc_ld2(Z2.ap + zk);
                }
                pair_add_cdiff(acc, zm, x[0][k], t0);  // row j-1 (a ghost at the z face, where zm = 0)
                pair_add_cdiff(acc, zp, x[2][k], t0);
                if (j == 0) pair_add_cdiff(acc, rc_ld2(Z2.dl + zk), bc2, t0);
                if (j == Nz - 1) pair_add_cdiff(acc, rc_ld2(Z2.dh + zk), bc3, t0);
                const real xm = k > 0 ? dl0[k - 1] : xl;
                const real xp = k < K - 1 ? dl0[k + 1] : xr;
                pair_add_cx(acc, b2, -dl0[k]);
                pair_add_cx(acc, am2, xm);
                pair_add_cx(acc, ap2, xp);
                d[0][k] = __fadd_rn(acc.hi, acc.lo) * iv[k];  // the correction's right-hand side times the pivot
            }
            const bool next = t + 1 < nrow && rowcls[j + 1] == a;
            if (next) {
                // row j+1's first solve rides along: its rows j .. j+2
                rb_wait<0>();
                ring_row(j + 2, x[0]);  // rows j, j+1 are x[1], x[2]
                real nl1, nr1;
                row_nb(j + 1, x[2], nl1, nr1);
                row_rhs(j + 1, x[1], x[2], x[0], d[1], nl1, nr1);
                solve(RbRows<2>(), d);
            } else {
                solve(RbRows<1>(), d);
            }
            // row j: theta + (delta0 + e)
            ring_row(j, x[1]);
#pragma unroll
            for (int k = 0; k < K; ++k) x[1][k] = x[1][k] + (dl0[k] + d[0][k]);
            store_row(j, x[1]);
            if (next) {
#pragma unroll
                for (int k = 0; k < K; ++k) dl0[k] = d[1][k];
            }
            have = next;
            fetch(j + NRING - 1);  // row j+3 into the slot of row j-1
        }
    }
    rb_wait<0>();
    // no block leaves while another may still address its shared memory
    rc_sync();
}

}  // namespace heat
