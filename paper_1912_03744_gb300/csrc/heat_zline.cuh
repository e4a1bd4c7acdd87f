// heat_zline.cuh -- the z-sweep (half-step 2 of the Peaceman-Rachford step,
// Sec. 3, eq. "scheme_eq_2"; the line matrix is the axial operator of
// eq. "Lambda_z" plus the mass term) in the literal and increment forms.
//
// Columns are strided, so lanes own columns: a warp owns up to 32 V adjacent
// columns (V per lane, one 16-byte segment of a row, so each row access of
// the warp is one contiguous run) and one chunk of Rc rows, and every lane
// walks its chunk row by row (interleaved Thomas).  The column partition and
// its carry algebra are those of ZPart (heat_internal.h):
//   zsum   : each (column, chunk) walked forward from a zero carry; the
//            results go to the output buffer, the carry summaries B (the
//            last of them) and G0 = sum r wG (r = right-hand side) to scratch;
//   zcarry : the carry recurrences of every column over its chunks;
//   zsolve : each chunk walked back from its carries, correcting every
//            forward result by the carry-in times a prefix product of f.
// A warp's columns are a column tile (zl_tile): 32 V columns from column 0,
// or, where the instance has a tile table, the columns of one column class
// (lanes start at the V-aligned column below the tile and store only its
// columns), so that no warp straddles a layer interface.  A batch's warps
// take their (instance, chunk, tile) from a work list (zl_work, ITEMS).
// Rows are fetched ZQ at a time and double-buffered: the loads of the next
// ZQ rows (and of the warp's left / right halo columns) are in flight while
// the current ZQ rows are computed.  The chunk's table rows are staged in
// shared memory before the walk (all loads in flight together): zsum stages
// them for a warp of one column class, zsolve its (P, cp) rows for up to ZNC
// classes; other warps read them per row and column through the read-only
// cache.  Full chunks (a multiple of 2 ZQ rows, away from the z faces, one
// row class) take lean walks with running row pointers.
#pragma once

#include <type_traits>

#include "heat_internal.h"

namespace heat {

constexpr int ZQ = 4;  // rows per fetch group

template <typename real, int V>
struct ZVec;
template <>
struct ZVec<float, 4> {
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
struct ZVec<double, 2> {
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

// The 8 packed table values {inv, f, cp, e0, e1, e2, wB, wG} of (class, row).
template <typename real>
__device__ __forceinline__ void zl_tab(const real *__restrict__ pkA, const real *__restrict__ pkB, size_t o,
                                       real (&e)[8])
{
    if constexpr (sizeof(real) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(pkA + 4 * o));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(pkB + 4 * o));
        e[0] = a.x, e[1] = a.y, e[2] = a.z, e[3] = a.w, e[4] = b.x, e[5] = b.y, e[6] = b.z, e[7] = b.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(pkA + 4 * o + u));
            const double2 b = __ldg(reinterpret_cast<const double2 *>(pkB + 4 * o + u));
            e[u] = a.x, e[u + 1] = a.y, e[4 + u] = b.x, e[5 + u] = b.y;
        }
    }
}

// Column classes staged per warp by the solve pass.
constexpr int ZNC = 4;

// The distinct column classes of the columns the warp stores (bits of
// smask), in order of discovery, into slot[0 .. ns-1]; false when there are
// more than ZNC.  slot[] and ns come out the same in every lane.
template <int V>
__device__ __forceinline__ bool zl_classes(const int (&b)[V], unsigned smask, int (&slot)[ZNC], int &ns)
{
#pragma unroll
    for (int s = 0; s < ZNC; ++s) slot[s] = -1;
    ns = 0;
#pragma unroll
    for (int round = 0; round <= ZNC; ++round) {
        int mine = -1;
#pragma unroll
        for (int q = V - 1; q >= 0; --q) {
            bool known = false;
#pragma unroll
            for (int s = 0; s < ZNC; ++s) known = known || b[q] == slot[s];
            if (((smask >> q) & 1u) && !known) mine = b[q];
        }
        const unsigned bal = __ballot_sync(HEAT_FULL_MASK, mine >= 0);
        if (bal == 0) return true;
        if (round == ZNC) return false;
        slot[round] = __shfl_sync(HEAT_FULL_MASK, mine, __ffs(bal) - 1);
        ns = round + 1;
    }
    return false;
}
// slot of each of the lane's columns (0 for those it does not store)
template <int V>
__device__ __forceinline__ void zl_slots(const int (&b)[V], unsigned smask, const int (&slot)[ZNC], int (&sq)[V])
{
#pragma unroll
    for (int q = 0; q < V; ++q) {
        sq[q] = 0;
#pragma unroll
        for (int s = 1; s < ZNC; ++s)
            if (((smask >> q) & 1u) && b[q] == slot[s]) sq[q] = s;
    }
}

// The column tile of warp grp of an instance: its lanes' first column wb and
// the columns [lo, hi) it stores (the instance's tile table, else warps of
// 32 V columns from column 0); false past the last tile.
template <typename real, int V>
__device__ __forceinline__ bool zl_tile(const SweepArgs<real> &A, int grp, int &wb, int &lo, int &hi)
{
    if (A.n_ztile > 0) {
        if (grp >= A.n_ztile) return false;
        const int4 t = A.ztile[grp];
        wb = t.x, lo = t.y, hi = t.z;
        return true;
    }
    wb = grp * 32 * V;
    lo = wb, hi = min(A.Nr, wb + 32 * V);
    return wb < A.Nr;
}
// The work of warp grp: instance mi, chunk c and column tile (wb, lo, hi),
// from the batch work list (ITEMS), else from the grid (chunk = blockIdx.y,
// instance = blockIdx.z); false when the warp has none.
template <typename real, int V, bool ITEMS>
__device__ __forceinline__ bool zl_work(const SweepArgs<real> *args, int grp, int &mi, int &c, int &wb, int &lo,
                                        int &hi)
{
    if constexpr (ITEMS) {
        if (grp >= args[0].n_zitem) return false;
        const int4 it = args[0].zitem[grp];
        mi = it.x & 0xffff, c = it.x >> 16, wb = it.y, lo = it.z, hi = it.w;
        return true;
    } else {
        mi = blockIdx.z, c = blockIdx.y;
        if (c >= args[mi].nch) return false;
        return zl_tile<real, V>(args[mi], grp, wb, lo, hi);
    }
}
// bits q of the lane's columns ib + q inside [lo, hi)
template <int V>
__device__ __forceinline__ unsigned zl_mask(int ib, int lo, int hi)
{
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < V; ++q)
        if (ib + q >= lo && ib + q < hi) m |= 1u << q;
    return m;
}

// Per-lane state of a z walk over rows [j0, j1) of the lane's V columns.
template <typename real, int V, int MODE>
struct ZWalk {
    static constexpr bool LIT = MODE == MODE_LIT;
    const real *__restrict__ th;
    const real *__restrict__ pkA;
    const real *__restrict__ pkB;
    const int *__restrict__ rowcls;
    int Nr, Nz, ib, lane, j0, j1;
    bool any, vec, uni, hasl, hasr, lo_edge, hi_edge;
    unsigned smask;                   // the lane's columns this walk stores (its tile's)
    bool sfull;                       // all V of them
    int b[V];
    int acur;
    real ra[V], rb[V], rc[V], rd[V];  // increment: xm, xp of the row class; literal: am, ap, ad, sd
    real bz_lo, bz_hi, br_lo, br_hi;  // ghost values beyond the outer faces
    real tm[V], t[V];                 // rows j-1 and j of the walk
    const real *stg = nullptr;        // the chunk's staged table rows [j1 - j0][8] (uniform warps)
    int bw = 0;                       // the warp's column class when it has one

    // any: the lane has columns inside the field (it reads them: they are
    // neighbours); smask: the columns of its tile [lo, hi), the ones it stores
    // and whose class counts
    __device__ __forceinline__ void init(const SweepArgs<real> &A, const real *th_, int ib_, int lane_, int j0_,
                                         int j1_, int lo, int hi)
    {
        th = th_, pkA = A.pkA, pkB = A.pkB, rowcls = A.rowcls;
        Nr = A.Nr, Nz = A.Nz, ib = ib_, lane = lane_, j0 = j0_, j1 = j1_;
        any = ib < Nr;
        vec = (Nr % V) == 0;
        smask = zl_mask<V>(ib, lo, hi);
        sfull = smask == (1u << V) - 1;
        lo_edge = ib == 0;
        hi_edge = ib < Nr && ib + V >= Nr;
        hasl = lane == 0 && ib > 0 && ib - 1 < Nr;
        hasr = lane == 31 && ib + V < Nr;
        const int i1 = smask ? ib + __ffs(smask) - 1 : 0;  // the lane's first stored column
#pragma unroll
        for (int q = 0; q < V; ++q) b[q] = A.colcls[(smask >> q) & 1u ? ib + q : i1];
        uni = true;
#pragma unroll
        for (int q = 1; q < V; ++q) uni = uni && b[q] == b[0];
        acur = -1;
        bz_lo = LIT ? real(0) : (real)A.bc.th[2];
        bz_hi = LIT ? real(0) : (real)A.bc.th[3];
        br_lo = LIT ? real(0) : (real)A.bc.th[0];
        br_hi = LIT ? real(0) : (real)A.bc.th[1];
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
    // row x of the lane's columns from src; ghost rows and columns hold theta_bc
    __device__ __forceinline__ void row(const real *__restrict__ src, int x, real (&v)[V]) const
    {
        if (x < 0 || x >= Nz) {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = x < 0 ? bz_lo : bz_hi;
            return;
        }
        const real *p = src + (size_t)x * Nr + ib;
        if (vec && any) {
            ZVec<real, V>::ld(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? p[q] : br_hi;
        }
    }
    // fetch group: rows x+1 .. x+ZQ (the row after each of rows x .. x+ZQ-1)
    // and the halo columns of rows x .. x+ZQ-1
    struct Group {
        real nx[ZQ][V];
        real hl[ZQ], hr[ZQ];
    };
    __device__ __forceinline__ void fetch(int x, Group &G) const
    {
#pragma unroll
        for (int p = 0; p < ZQ; ++p) {
            const int jr = x + p;
            if (jr < j1) {
                row(th, jr + 1, G.nx[p]);
                G.hl[p] = hasl ? th[(size_t)jr * Nr + ib - 1] : real(0);
                G.hr[p] = hasr ? th[(size_t)jr * Nr + ib + V] : real(0);
            }
        }
    }
    // True (for every lane) when every column the warp stores has lane 0's
    // column class bw (lane 0 always stores one); the other columns are then
    // computed with bw too and not stored.
    __device__ __forceinline__ bool warp_uniform()
    {
        bw = __shfl_sync(HEAT_FULL_MASK, b[0], 0);
        return __all_sync(HEAT_FULL_MASK, !smask || (uni && b[0] == bw));
    }
    // store the lane's V values at p (its tile's columns)
    __device__ __forceinline__ void put(real *p, const real (&v)[V]) const
    {
        if (vec && sfull) {
            ZVec<real, V>::st(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q)
                if ((smask >> q) & 1u) p[q] = v[q];
        }
    }
    // Stage the chunk's table rows of class bw (a uniform warp) in the warp's
    // shared-memory slice buf [j1 - j0][8]: one row per lane per pass, all
    // loads in flight together.
    __device__ __forceinline__ void stage(real *buf)
    {
        for (int r = lane; r < j1 - j0; r += 32) {
            real e[8];
            zl_tab(pkA, pkB, (size_t)bw * Nz + j0 + r, e);
            real *d = buf + (size_t)r * 8;
            if constexpr (sizeof(real) == 4) {
                *reinterpret_cast<float4 *>(d) = make_float4(e[0], e[1], e[2], e[3]);
                *reinterpret_cast<float4 *>(d + 4) = make_float4(e[4], e[5], e[6], e[7]);
            } else {
#pragma unroll
                for (int u = 0; u < 8; u += 2) *reinterpret_cast<double2 *>(d + u) = make_double2(e[u], e[u + 1]);
            }
        }
        __syncwarp();
        stg = buf;
    }
    // table values of row j: E = 1 (every column of the warp shares one class:
    // the staged rows) or E = V (per column, from the read-only cache)
    template <int E>
    __device__ __forceinline__ void tab(int j, real (&e)[E][8]) const
    {
        if constexpr (E == 1) {
            const real *p = stg + (size_t)(j - j0) * 8;
            if constexpr (sizeof(real) == 4) {
                const float4 a = *reinterpret_cast<const float4 *>(p), c = *reinterpret_cast<const float4 *>(p + 4);
                e[0][0] = a.x, e[0][1] = a.y, e[0][2] = a.z, e[0][3] = a.w;
                e[0][4] = c.x, e[0][5] = c.y, e[0][6] = c.z, e[0][7] = c.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const double2 a = *reinterpret_cast<const double2 *>(p + u);
                    e[0][u] = a.x, e[0][u + 1] = a.y;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) zl_tab(pkA, pkB, (size_t)b[q] * Nz + j, e[q]);
        }
    }
    // right-hand side of row j from its left / right neighbours tl, tr of the
    // lane's first / last column and row j+1 (then advance the row window)
    template <int E>
    __device__ __forceinline__ void rhs_core(real tl, real tr, const real (&nx)[V], const real (&e)[E][8],
                                             real (&d)[V])
    {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const real(&eq)[8] = e[E == 1 ? 0 : q];
            const real x = t[q];
            const real l = q > 0 ? t[q - 1] : tl;
            const real r = q < V - 1 ? t[q + 1] : tr;
            if constexpr (LIT) {
                // e0 = s, e1 = w: (w + ad_r) x + am_r x_{i-1} + ap_r x_{i+1} + s + sd_r
                d[q] = fmad(eq[4] + rc[q], x, fmad(ra[q], l, fmad(rb[q], r, eq[3] + rd[q])));
            } else {
                // e0 = q, e1 = xm_z, e2 = xp_z
                real v = fmad(eq[4], tm[q] - x, eq[3]);
                v = fmad(eq[5], nx[q] - x, v);
                v = fmad(ra[q], l - x, v);
                d[q] = fmad(rb[q], r - x, v);
            }
        }
#pragma unroll
        for (int q = 0; q < V; ++q) tm[q] = t[q], t[q] = nx[q];
    }
    // the neighbours of the lane's first / last column: the next lanes', a
    // halo value hl / hr at a warp edge, theta_bc past the field
    __device__ __forceinline__ void sides(real hl, real hr, real &tl, real &tr) const
    {
        tl = __shfl_up_sync(HEAT_FULL_MASK, t[V - 1], 1);
        tr = __shfl_down_sync(HEAT_FULL_MASK, t[0], 1);
        if (hasl) tl = hl;
        if (hasr) tr = hr;
        if (lo_edge) tl = br_lo;
        if (hi_edge) tr = br_hi;
    }
    template <int E>
    __device__ __forceinline__ void rhs(const Group &G, int p, const real (&e)[E][8], real (&d)[V])
    {
        real tl, tr;
        sides(G.hl[p], G.hr[p], tl, tr);
        rhs_core<E>(tl, tr, G.nx[p], e, d);
    }
    // Lean walk of a full interior chunk: rows [j0, j1) with j0 >= 1,
    // j1 < Nz, (j1 - j0) a multiple of 2 ZQ, every lane inside the field, whole
    // 16-byte row segments and one row class ucls >= 0.  No row needs a bounds
    // check, so rows are reached through running pointers, and the one halo
    // value a lane needs (lane 0: the column left of the warp, lane 31: the
    // one right of it) is one predicated load.  emit(dst, d, e) gets the
    // lane's address in row j of the output whose row j0 is at dst.
    template <int E, typename Emit>
    __device__ __forceinline__ void walk_full(int ucls, const LineTab<real> &R, real *__restrict__ dst, Emit emit)
    {
        const size_t S = (size_t)Nr;
        row_class(ucls, R);
        ZVec<real, V>::ld(th + (size_t)(j0 - 1) * S + ib, tm);
        ZVec<real, V>::ld(th + (size_t)j0 * S + ib, t);
        const bool hh = hasl || hasr;
        const real *np = th + (size_t)(j0 + 1) * S + ib;
        const real *hp = th + (size_t)j0 * S + ib + (lane == 0 ? -1 : V);
        const real *ep = stg;
        real nxA[ZQ][V], hA[ZQ], nxB[ZQ][V], hB[ZQ];
        auto fetch = [&](real(&nx)[ZQ][V], real(&h)[ZQ]) {
#pragma unroll
            for (int p = 0; p < ZQ; ++p) {
                ZVec<real, V>::ld(np + p * S, nx[p]);
                h[p] = hh ? __ldg(hp + p * S) : real(0);
            }
            np += ZQ * S;
            hp += ZQ * S;
        };
        auto proc = [&](int x, const real(&nx)[ZQ][V], const real(&h)[ZQ]) {
#pragma unroll
            for (int p = 0; p < ZQ; ++p) {
                real e[E][8], d[V];
                if constexpr (E == 1) {
                    if constexpr (sizeof(real) == 4) {
                        const float4 a = *reinterpret_cast<const float4 *>(ep);
                        const float4 c = *reinterpret_cast<const float4 *>(ep + 4);
                        e[0][0] = a.x, e[0][1] = a.y, e[0][2] = a.z, e[0][3] = a.w;
                        e[0][4] = c.x, e[0][5] = c.y, e[0][6] = c.z, e[0][7] = c.w;
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; u += 2) {
                            const double2 a = *reinterpret_cast<const double2 *>(ep + u);
                            e[0][u] = a.x, e[0][u + 1] = a.y;
                        }
                    }
                    ep += 8;
                } else {
                    tab<E>(x + p, e);
                }
                real tl, tr;
                sides(h[p], h[p], tl, tr);
                rhs_core<E>(tl, tr, nx[p], e, d);
                emit(dst, d, e);
                dst += S;
            }
        };
        fetch(nxA, hA);
#pragma unroll 1
        for (int x = j0; x < j1; x += 2 * ZQ) {
            fetch(nxB, hB);
            proc(x, nxA, hA);
            if (x + 2 * ZQ < j1) fetch(nxA, hA);
            proc(x + ZQ, nxB, hB);
        }
    }
    // Walk rows [j0, j1) calling emit(j, d, e) with the right-hand side d of
    // row j and its table values e (E = 1: shared by the lane's columns).
    // A chunk of several row classes (ucls < 0) reads the classes of 32 rows
    // at a time, one per lane, and takes row j's by a shuffle: no row waits
    // for a load of its class.
    template <int E, typename Emit>
    __device__ __forceinline__ void walk(int ucls, const LineTab<real> &R, Emit emit)
    {
        row(th, j0 - 1, tm);
        row(th, j0, t);
        if (ucls >= 0) row_class(ucls, R);
        int rcl = ucls < 0 ? rowcls[min(j0 + lane, Nz - 1)] : 0;
        Group A, B;
        auto proc = [&](int x, const Group &G) {
#pragma unroll
            for (int p = 0; p < ZQ; ++p) {
                const int j = x + p;
                if (j < j1) {
                    if (ucls < 0) {
                        const int jj = j - j0;
                        if (jj > 0 && (jj & 31) == 0) rcl = rowcls[min(j + lane, Nz - 1)];
                        row_class(__shfl_sync(HEAT_FULL_MASK, rcl, jj & 31), R);
                    }
                    real e[E][8], d[V];
                    tab<E>(j, e);
                    rhs<E>(G, p, e, d);
                    emit(j, d, e);
                }
            }
        };
        fetch(j0, A);
#pragma unroll 1
        for (int x = j0; x < j1; x += 2 * ZQ) {
            const bool h1 = x + ZQ < j1;
            if (h1) fetch(x + ZQ, B);
            proc(x, A);
            if (h1) {
                if (x + 2 * ZQ < j1) fetch(x + 2 * ZQ, A);
                proc(x + ZQ, B);
            }
        }
    }
};

// Pass 1: every (column, chunk) walked forward from a zero carry.  The
// results d0_j (the forward recurrence with a zero carry-in) are stored in the
// output field buffer -- during the z-sweep it holds the superseded field --
// and the chunk's carry summaries B = d0 at its last row and G0 = sum r wG go
// to zs[(c*2 + s)*Nr + i].  Grid (column warps / warps per block, chunks,
// instances), or with ITEMS (batch work list / warps per block).
template <typename real, int V, int MODE, bool ITEMS>
__global__ void __launch_bounds__(128, 4) zsum2_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int grp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int mi, c, wb, lo, hi;
    if (!zl_work<real, V, ITEMS>(args, grp, mi, c, wb, lo, hi)) return;  // no work (warp-uniform)
    const SweepArgs<real> &A = args[mi];
    const int Nr = A.Nr, Nz = A.Nz, Rc = A.Rc;
    const int j0 = c * Rc, j1 = min(Nz, j0 + Rc);
    real *__restrict__ d0out = flip ? A.f0 : A.f1;
    ZWalk<real, V, MODE> W;
    W.init(A, flip ? A.f1 : A.f0, wb + lane * V, lane, j0, j1, lo, hi);
    real dl[V], sg[V];
#pragma unroll
    for (int q = 0; q < V; ++q) dl[q] = sg[q] = real(0);
    auto emit = [&](int j, const real(&d)[V], const auto &e) {
        constexpr int E = sizeof(e) / sizeof(e[0]);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            dl[q] = fmad(d[q], e[E == 1 ? 0 : q][0], e[E == 1 ? 0 : q][1] * dl[q]);
            sg[q] = fmad(d[q], e[E == 1 ? 0 : q][7], sg[q]);
        }
        W.put(d0out + (size_t)j * Nr + W.ib, dl);
    };
    // the lean walk of a full interior chunk of a warp of one column class
    // (warp-uniform decision)
    auto emit_full = [&](real *dst, const real(&d)[V], const auto &e) {
        constexpr int E = sizeof(e) / sizeof(e[0]);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            dl[q] = fmad(d[q], e[E == 1 ? 0 : q][0], e[E == 1 ? 0 : q][1] * dl[q]);
            sg[q] = fmad(d[q], e[E == 1 ? 0 : q][7], sg[q]);
        }
        W.put(dst, dl);
    };
    const int ucls = A.ucls[c];
    const bool full = W.vec && ucls >= 0 && j0 >= 1 && j1 < Nz && (j1 - j0) % (2 * ZQ) == 0 &&
                      __all_sync(HEAT_FULL_MASK, W.any);
    real *dst = d0out + (size_t)j0 * Nr + W.ib;
    extern __shared__ __align__(16) unsigned char zs_smem[];
    if (W.warp_uniform()) {
        // (a work list's block may hold warps of instances with different Rc:
        // slices at the batch's largest)
        const int Rs = ITEMS ? args[0].zrc_max : Rc;
        W.stage(reinterpret_cast<real *>(zs_smem) + (size_t)(threadIdx.x >> 5) * Rs * 8);
        pdl_wait();
        if (full)
            W.template walk_full<1>(ucls, A.R, dst, emit_full);
        else
            W.template walk<1>(ucls, A.R, emit);
    } else {
        pdl_wait();
        W.template walk<V>(ucls, A.R, emit);  // (a lean walk here would spill)
    }
    real *__restrict__ zs = A.zs;
    W.put(zs + ((size_t)c * 2) * Nr + W.ib, dl);
    W.put(zs + ((size_t)c * 2 + 1) * Nr + W.ib, sg);
}

// Pass 3: every (column, chunk) walked back from its carries: with
// D = the forward carry into the chunk and X = the backward carry from above,
//   d'_j = d0_j + P_j D   (P_j = prod f from the chunk's first row to j),
//   x_j  = d'_j + cp_j x_{j+1},
// and the new field is theta + x (increment form) or x (literal form).  Rows
// of d0 and theta are fetched ZQ at a time, double-buffered.
// OUT (increment form, the refined z-sweep): ZOUT_DELTA0 stores x itself in
// the rho buffer (delta0 of the first solve); ZOUT_CORR stores
// theta + (delta0 + x) with delta0 read from the rho buffer (x the correction).
enum { ZOUT_FIELD = 0, ZOUT_DELTA0 = 1, ZOUT_CORR = 2 };
template <typename real, int V, int MODE, bool ITEMS, int OUT = ZOUT_FIELD>
__global__ void __launch_bounds__(128, ITEMS ? 4 : 1) zsolve2_kernel(const SweepArgs<real> *__restrict__ args, int flip)
{
    pdl_launch_dependents();
    constexpr bool LIT = MODE == MODE_LIT || OUT == ZOUT_DELTA0;  // no theta to add
    static_assert(OUT == ZOUT_FIELD || MODE == MODE_DELTA, "refined outputs are increment forms");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = blockIdx.x * (blockDim.x >> 5) + w;
    int mi, c, wb, lo, hi;
    if (!zl_work<real, V, ITEMS>(args, grp, mi, c, wb, lo, hi)) return;  // no work (warp-uniform)
    const SweepArgs<real> &A = args[mi];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;  // holds d0 on entry
    real *__restrict__ dst = OUT == ZOUT_DELTA0 ? A.rho : out;
    const real *__restrict__ dl0 = A.rho;  // ZOUT_CORR: delta0
    const int Nr = A.Nr, Nz = A.Nz, Rc = A.Rc;
    const int j0 = c * Rc, j1 = min(Nz, j0 + Rc);
    const int ib = wb + lane * V;
    // any: columns inside the field (read); smask: the tile's (stored)
    const bool any = ib < Nr, vec = (Nr % V) == 0;
    const unsigned smask = zl_mask<V>(ib, lo, hi);
    const bool sfull = smask == (1u << V) - 1;
    const real *__restrict__ pkA = A.pkA;
    const real *__restrict__ pkB = A.pkB;
    int b[V];
    const int i1 = smask ? ib + __ffs(smask) - 1 : 0;  // the lane's first stored column
#pragma unroll
    for (int q = 0; q < V; ++q) b[q] = A.colcls[(smask >> q) & 1u ? ib + q : i1];
    bool uni = true;
#pragma unroll
    for (int q = 1; q < V; ++q) uni = uni && b[q] == b[0];
    const int bw = __shfl_sync(HEAT_FULL_MASK, b[0], 0);
    const bool wuni = __all_sync(HEAT_FULL_MASK, !smask || (uni && b[0] == bw));
    auto put = [&](real *p, const real(&v)[V]) {
        if (vec && sfull) {
            ZVec<real, V>::st(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q)
                if ((smask >> q) & 1u) p[q] = v[q];
        }
    };
    // staged (P_j, cp_j) of the chunk's rows for each of the warp's (at most
    // ZNC) column classes, [slot][Rc][2]; slot 0 is bw in a warp of one class
    int slot[ZNC], ns;
    const bool few = zl_classes(b, smask, slot, ns);
    extern __shared__ __align__(16) unsigned char zl_smem[];
    const int Rs = ITEMS ? args[0].zrc_max : Rc;  // slice stride (see zsum2)
    real *stg = reinterpret_cast<real *>(zl_smem) + (size_t)w * ZNC * Rs * 2;
    int off[V];
    if (few) {
        for (int u = lane; u < ns * (j1 - j0); u += 32) {
            const int s = u / (j1 - j0), r = u - s * (j1 - j0);
            int cs = slot[0];
#pragma unroll
            for (int k = 1; k < ZNC; ++k)
                if (s == k) cs = slot[k];
            const size_t o = (size_t)cs * Nz + j0 + r;
            stg[((size_t)s * Rc + r) * 2] = __ldg(pkB + 4 * o + 2);
            stg[((size_t)s * Rc + r) * 2 + 1] = __ldg(pkA + 4 * o + 2);
        }
        __syncwarp();
        int sq[V];
        zl_slots(b, smask, slot, sq);
#pragma unroll
        for (int q = 0; q < V; ++q) off[q] = sq[q] * Rc * 2;
    }
    pdl_wait();
    const real *__restrict__ zc = A.zc;
    real D[V], x[V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const bool in = (smask >> q) & 1u;
        D[q] = in ? zc[((size_t)c * 2) * Nr + ib + q] : real(0);
        x[q] = in ? zc[((size_t)c * 2 + 1) * Nr + ib + q] : real(0);
    }
    auto ldrow = [&](const real *__restrict__ src, int j, real (&v)[V]) {
        const real *p = src + (size_t)j * Nr + ib;
        if (vec && any) {
            ZVec<real, V>::ld(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? p[q] : real(0);
        }
    };
    auto fetch = [&](int x0, real (&dz)[ZQ][V], real (&bs)[ZQ][V], real (&ds)[ZQ][V]) {
#pragma unroll
        for (int p = 0; p < ZQ; ++p) {
            const int j = x0 - p;
            if (j >= j0) {
                ldrow(out, j, dz[p]);
                if constexpr (!LIT) ldrow(th, j, bs[p]);
                if constexpr (OUT == ZOUT_CORR) ldrow(dl0, j, ds[p]);
            }
        }
    };
    auto proc = [&](int x0, const real (&dz)[ZQ][V], const real (&bs)[ZQ][V], const real (&ds)[ZQ][V]) {
#pragma unroll
        for (int p = 0; p < ZQ; ++p) {
            const int j = x0 - p;
            if (j >= j0) {
                real Pj[V], cpj[V];
                if (wuni) {
                    const real pv = stg[2 * (j - j0)], cv = stg[2 * (j - j0) + 1];
#pragma unroll
                    for (int q = 0; q < V; ++q) Pj[q] = pv, cpj[q] = cv;
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        const size_t o = (size_t)b[q] * Nz + j;
                        Pj[q] = __ldg(pkB + 4 * o + 2);
                        cpj[q] = __ldg(pkA + 4 * o + 2);
                    }
                }
                real o[V];
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    x[q] = fmad(cpj[q], x[q], fmad(Pj[q], D[q], dz[p][q]));
                    o[q] = LIT ? x[q] : OUT == ZOUT_CORR ? bs[p][q] + (ds[p][q] + x[q]) : bs[p][q] + x[q];
                }
                put(dst + (size_t)j * Nr + ib, o);
            }
        }
    };
    real da[ZQ][V], ba[ZQ][V], db[ZQ][V], bb[ZQ][V];
    real sa[ZQ][V], sb[ZQ][V];  // ZOUT_CORR: delta0 rows
    if (few && (j1 - j0) % (2 * ZQ) == 0) {
        // a full chunk: no row needs a bounds check; running row pointers.
        // TM = 1: one class (one staged (P, cp) pair per row), else per
        // column; VEC: whole 16-byte row segments, else per column with
        // range checks
        const size_t S = (size_t)Nr;
        const size_t o1 = (size_t)(j1 - 1) * S + ib;
        auto lean = [&](auto tm_tag, auto vec_tag) {
            constexpr int TM = decltype(tm_tag)::value;
            constexpr bool VEC = decltype(vec_tag)::value;
            const real *dp = out + o1, *tp = th + o1, *lp = dl0 + o1;
            real *op = dst + o1;
            int ro = 2 * (j1 - 1 - j0);
            auto ld = [&](const real *p, real(&v)[V]) {
                if constexpr (VEC) {
                    if (any) {
                        ZVec<real, V>::ld(p, v);
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) v[q] = real(0);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? __ldg(p + q) : real(0);
                }
            };
            auto fetchf = [&](real(&dz)[ZQ][V], real(&bs)[ZQ][V], real(&ds)[ZQ][V]) {
#pragma unroll
                for (int p = 0; p < ZQ; ++p) {
                    ld(dp - p * S, dz[p]);
                    if constexpr (!LIT) ld(tp - p * S, bs[p]);
                    if constexpr (OUT == ZOUT_CORR) ld(lp - p * S, ds[p]);
                }
                dp -= ZQ * S;
                tp -= ZQ * S;
                lp -= ZQ * S;
            };
            auto procf = [&](const real(&dz)[ZQ][V], const real(&bs)[ZQ][V], const real(&ds)[ZQ][V]) {
#pragma unroll
                for (int p = 0; p < ZQ; ++p) {
                    real Pj[V], cpj[V];
                    if constexpr (TM == 1) {
                        const real pv = stg[ro], cv = stg[ro + 1];
#pragma unroll
                        for (int q = 0; q < V; ++q) Pj[q] = pv, cpj[q] = cv;
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) Pj[q] = stg[off[q] + ro], cpj[q] = stg[off[q] + ro + 1];
                    }
                    ro -= 2;
                    real o[V];
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        x[q] = fmad(cpj[q], x[q], fmad(Pj[q], D[q], dz[p][q]));
                        o[q] = LIT ? x[q] : OUT == ZOUT_CORR ? bs[p][q] + (ds[p][q] + x[q]) : bs[p][q] + x[q];
                    }
                    put(op, o);
                    op -= S;
                }
            };
            fetchf(da, ba, sa);
#pragma unroll 1
            for (int x0 = j1 - 1; x0 >= j0; x0 -= 2 * ZQ) {
                fetchf(db, bb, sb);
                procf(da, ba, sa);
                if (x0 - 2 * ZQ >= j0) fetchf(da, ba, sa);
                procf(db, bb, sb);
            }
        };
        using One = std::integral_constant<int, 1>;
        using Many = std::integral_constant<int, ZNC>;
        using Vec = std::integral_constant<bool, true>;
        using Sca = std::integral_constant<bool, false>;
        if (ns == 1) {
            if (vec)
                lean(One(), Vec());
            else
                lean(One(), Sca());
        } else {
            if (vec)
                lean(Many(), Vec());
            else
                lean(Many(), Sca());
        }
        return;
    }
    fetch(j1 - 1, da, ba, sa);
#pragma unroll 1
    for (int x0 = j1 - 1; x0 >= j0; x0 -= 2 * ZQ) {
        const bool h1 = x0 - ZQ >= j0;
        if (h1) fetch(x0 - ZQ, db, bb, sb);
        proc(x0, da, ba, sa);
        if (h1) {
            if (x0 - 2 * ZQ >= j0) fetch(x0 - 2 * ZQ, da, ba, sa);
            proc(x0 - ZQ, db, bb, sb);
        }
    }
}

// Summary pass of the refined z-sweep's correction: zsum2 with the residual
// rho_j (stored in the output buffer by zres_kernel) as the right-hand side
// of row j; the forward results d0 replace it in place (each lane reads its
// stored columns before writing them).
template <int V, bool ITEMS>
__global__ void __launch_bounds__(128, 4) zsumc_kernel(const SweepArgs<float> *__restrict__ args, int flip)
{
    using real = float;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int grp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int mi, c, wb, lo, hi;
    if (!zl_work<real, V, ITEMS>(args, grp, mi, c, wb, lo, hi)) return;  // no work (warp-uniform)
    const SweepArgs<real> &A = args[mi];
    const int Nr = A.Nr, Nz = A.Nz, Rc = A.Rc;
    const int j0 = c * Rc, j1 = min(Nz, j0 + Rc);
    real *__restrict__ io = flip ? A.f0 : A.f1;
    ZWalk<real, V, MODE_DELTA> W;
    W.init(A, flip ? A.f1 : A.f0, wb + lane * V, lane, j0, j1, lo, hi);
    real dl[V], sg[V];
#pragma unroll
    for (int q = 0; q < V; ++q) dl[q] = sg[q] = real(0);
    extern __shared__ __align__(16) unsigned char zc_smem[];
    const bool one = W.warp_uniform();
    if (one) {
        const int Rs = ITEMS ? args[0].zrc_max : Rc;
        W.stage(reinterpret_cast<real *>(zc_smem) + (size_t)(threadIdx.x >> 5) * Rs * 8);
    }
    pdl_wait();
    auto run = [&](auto e_tag) {
        constexpr int E = decltype(e_tag)::value;
        real ra[ZQ][V], rb[ZQ][V];
        auto fetch = [&](int x, real(&r)[ZQ][V]) {
#pragma unroll
            for (int p = 0; p < ZQ; ++p)
                if (x + p < j1) W.row(io, x + p, r[p]);
        };
        auto proc = [&](int x, const real(&r)[ZQ][V]) {
#pragma unroll
            for (int p = 0; p < ZQ; ++p) {
                const int j = x + p;
                if (j < j1) {
                    real e[E][8];
                    W.template tab<E>(j, e);
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        dl[q] = fmad(r[p][q], e[E == 1 ? 0 : q][0], e[E == 1 ? 0 : q][1] * dl[q]);
                        sg[q] = fmad(r[p][q], e[E == 1 ? 0 : q][7], sg[q]);
                    }
                    W.put(io + (size_t)j * Nr + W.ib, dl);
                }
            }
        };
        fetch(j0, ra);
#pragma unroll 1
        for (int x = j0; x < j1; x += 2 * ZQ) {
            const bool h1 = x + ZQ < j1;
            if (h1) fetch(x + ZQ, rb);
            proc(x, ra);
            if (h1) {
                if (x + 2 * ZQ < j1) fetch(x + 2 * ZQ, ra);
                proc(x + ZQ, rb);
            }
        }
    };
    if (one)
        run(std::integral_constant<int, 1>());
    else
        run(std::integral_constant<int, V>());
    real *__restrict__ zs = A.zs;
    W.put(zs + ((size_t)c * 2) * Nr + W.ib, dl);
    W.put(zs + ((size_t)c * 2 + 1) * Nr + W.ib, sg);
}

// Residual of the refined z-sweep's line systems at delta0 (the first
// solve's increment, in the rho buffer), for every cell, into the output
// buffer: rho = q + sum over the four neighbours of c (theta_nb - theta)
// - b delta0 + am delta0_{j-1} + ap delta0_{j+1}, the z-couplings (am, ap,
// b, q) of the cell's column class and the r-couplings of its row class
// from the FP64 tables as FP32 pairs, with exact differences and FMA
// products (Pair in heat_kernels.cuh).  Dirichlet faces enter as couplings
// (dl, dh) to the ghost value theta_bc.  A warp owns 32 V adjacent columns
// and walks kZResRows rows, the next rows' loads in flight.
constexpr int kZResRows = 32;
template <int V>
__global__ void __launch_bounds__(128) zres_kernel(const SweepArgs<float> *__restrict__ args, int flip)
{
    using real = float;
    pdl_launch_dependents();
    const SweepArgs<real> &A = args[0];
    const real *__restrict__ th = flip ? A.f1 : A.f0;
    real *__restrict__ out = flip ? A.f0 : A.f1;
    const real *__restrict__ dz = A.rho;
    const int Nr = A.Nr, Nz = A.Nz;
    const int lane = threadIdx.x & 31;
    const int wcol = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 * V;
    if (wcol >= Nr) return;  // warp-uniform
    const int ib = wcol + lane * V;
    const int j0 = blockIdx.y * kZResRows, j1 = min(Nz, j0 + kZResRows);
    const bool any = ib < Nr, vec = (Nr % V) == 0;
    const real bz_lo = (real)A.bc.th[2], bz_hi = (real)A.bc.th[3];
    const real br_lo = (real)A.bc.th[0], br_hi = (real)A.bc.th[1];
    const LineTab2 &R2 = A.R2, &Z2 = A.Z2;
    int b[V];
#pragma unroll
    for (int q = 0; q < V; ++q) b[q] = ib + q < Nr ? A.colcls[ib + q] : (any ? A.colcls[ib] : 0);
    bool uni = true;
#pragma unroll
    for (int q = 1; q < V; ++q) uni = uni && b[q] == b[0];
    auto trow = [&](int j, real(&v)[V]) {
        if (j < 0 || j >= Nz) {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = j < 0 ? bz_lo : bz_hi;
            return;
        }
        const real *p = th + (size_t)j * Nr + ib;
        if (vec && any) {
            ZVec<real, V>::ld(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? p[q] : br_hi;
        }
    };
    auto drow = [&](int j, real(&v)[V]) {
        if (j < 0 || j >= Nz) {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = real(0);
            return;
        }
        const real *p = dz + (size_t)j * Nr + ib;
        if (vec && any) {
            ZVec<real, V>::ld(p, v);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = ib + q < Nr ? p[q] : real(0);
        }
    };
    pdl_wait();
    // rows j-1, j (tm, t; dm, dc) and the prefetched row j+1 (tp, dp)
    real tm[V], t[V], tp[V], dm[V], dc[V], dp[V];
    trow(j0 - 1, tm);
    trow(j0, t);
    drow(j0 - 1, dm);
    drow(j0, dc);
    trow(j0 + 1, tp);
    drow(j0 + 1, dp);
    int acur = -1;
    float2 A0[V], A1[V];
#pragma unroll
    for (int q = 0; q < V; ++q) A0[q] = A1[q] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        // the row after next in flight while this one is computed
        real tn[V], dn[V];
        trow(j + 2, tn);
        drow(j + 2, dn);
        real tl = __shfl_up_sync(HEAT_FULL_MASK, t[V - 1], 1);
        real tr = __shfl_down_sync(HEAT_FULL_MASK, t[0], 1);
        if (lane == 0) tl = ib > 0 && ib - 1 < Nr ? th[(size_t)j * Nr + ib - 1] : br_lo;
        if (lane == 31) tr = ib + V < Nr ? th[(size_t)j * Nr + ib + V] : br_hi;
        const int a = A.rowcls[j];
        if (a != acur) {
            acur = a;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int i = ib + q;
                const size_t ro = (size_t)a * Nr + i;
                A0[q] = i < Nr ? (i == 0 ? R2.dl[ro] : R2.am[ro]) : make_float2(0.f, 0.f);
                A1[q] = i < Nr ? (i == Nr - 1 ? R2.dh[ro] : R2.ap[ro]) : make_float2(0.f, 0.f);
            }
        }
        real rr[V];
        float2 cq, cm, cp, cb, fm, fp;  // z pairs of the class: q, am, ap, b; face couplings of the theta terms
        auto zload = [&](int cls) {
            const size_t zj = (size_t)cls * Nz + j;
            cq = __ldg(Z2.q + zj);
            cm = __ldg(Z2.am + zj);
            cp = __ldg(Z2.ap + zj);
            cb = __ldg(Z2.b + zj);
            fm = j == 0 ? __ldg(Z2.dl + zj) : cm;
            fp = j == Nz - 1 ? __ldg(Z2.dh + zj) : cp;
        };
        if (uni) zload(b[0]);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            if (!uni) zload(b[q]);
            const real x = t[q];
            const real l = q > 0 ? t[q - 1] : tl;
            const real r = q < V - 1 ? t[q + 1] : tr;
            Pair acc{cq.x, cq.y};
            pair_add_cdiff(acc, fm, tm[q], x);
            pair_add_cdiff(acc, fp, tp[q], x);
            pair_add_cdiff(acc, A0[q], l, x);
            pair_add_cdiff(acc, A1[q], r, x);
            pair_add_cx(acc, cb, -dc[q]);
            pair_add_cx(acc, cm, dm[q]);
            pair_add_cx(acc, cp, dp[q]);
            rr[q] = __fadd_rn(acc.hi, acc.lo);
        }
        if (any) {
            real *o = out + (size_t)j * Nr + ib;
            if (vec) {
                ZVec<real, V>::st(o, rr);
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q)
                    if (ib + q < Nr) o[q] = rr[q];
            }
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            tm[q] = t[q], t[q] = tp[q], tp[q] = tn[q];
            dm[q] = dc[q], dc[q] = dp[q], dp[q] = dn[q];
        }
    }
}

// Pass 2: chunk carries.  A block of SEG warps (segments: 4, 16 or 32, the
// fewest that cover the chunks) serves 32 columns (lane = column: every
// access is coalesced); warp s owns chunks [s m, (s+1) m),
// m = ceil(nch / SEG) <= ZMAXM, loads all their summaries and constants at
// once, composes its segment's affine maps, joins the segments through shared
// memory and writes cin_c = D_{c-1} and xin_c = X_{c+1} to zc[(c*2 + 0|1)*Nr + i].
constexpr int ZSEG2 = 32;  // segments (warps per block) for up to ZSEG2 ZMAXM chunks
constexpr int ZMAXM = 8;

template <typename real, int SEG>
__global__ void __launch_bounds__(32 * SEG) zcarry2_kernel(const SweepArgs<real> *__restrict__ args)
{
    pdl_launch_dependents();
    const SweepArgs<real> &A = args[blockIdx.y];
    const int Nr = A.Nr, nch = A.nch;
    if ((int)blockIdx.x * 32 >= Nr) return;  // past this instance (block-uniform)
    const real *__restrict__ zs = A.zs;
    real *__restrict__ zc = A.zc;
    __shared__ real sF[SEG][33], sB[SEG][33];
    const int lane = threadIdx.x & 31, sgm = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const bool col = i < Nr;
    const real *__restrict__ chb = A.chk + (size_t)(col ? A.colcls[i] : 0) * nch * 4;
    const int m = (nch + SEG - 1) / SEG;
    const int c0 = sgm * m;
    const size_t st = (size_t)2 * Nr;
    real Bv[ZMAXM], Gv[ZMAXM], Fv[ZMAXM], Hv[ZMAXM], GPv[ZMAXM];
    // the chunk constants do not change between launches: requested before
    // the wait for the summary pass, whose results (zs) are read after it
#pragma unroll
    for (int u = 0; u < ZMAXM; ++u) {
        const int c = c0 + u;
        const bool ok = col && u < m && c < nch;
        Fv[u] = ok ? chb[c * 4] : real(1);
        Hv[u] = ok ? chb[c * 4 + 1] : real(1);
        if constexpr (sizeof(real) == 4) GPv[u] = ok ? chb[c * 4 + 2] : real(0);  // (FP64: no registers left)
    }
    pdl_wait();
#pragma unroll
    for (int u = 0; u < ZMAXM; ++u) {
        const int c = c0 + u;
        const bool ok = col && u < m && c < nch;
        Bv[u] = ok ? zs[c * st + i] : real(0);
        Gv[u] = ok ? zs[c * st + Nr + i] : real(0);
    }
    // forward: D_c = B_c + F_c D_{c-1}
    real F = real(1), B = real(0);
#pragma unroll
    for (int u = 0; u < ZMAXM; ++u) {
        B = fmad(Fv[u], B, Bv[u]);
        F *= Fv[u];
    }
    sF[sgm][lane] = F;
    sB[sgm][lane] = B;
    __syncthreads();
    real D = real(0);
    for (int v = 0; v < sgm; ++v) D = fmad(sF[v][lane], D, sB[v][lane]);
    // Gv becomes G0_c + GP_c D_{c-1}, the backward map's constant term
#pragma unroll
    for (int u = 0; u < ZMAXM; ++u) {
        const int c = c0 + u;
        const bool ok = col && u < m && c < nch;
        if (ok) {
            zc[c * st + i] = D;
            if constexpr (sizeof(real) == 4)
                Gv[u] = fmad(GPv[u], D, Gv[u]);
            else
                Gv[u] = fmad(chb[c * 4 + 2], D, Gv[u]);
        }
        D = fmad(Fv[u], D, Bv[u]);
    }
    // backward: X_c = (G0_c + GP_c D_{c-1}) + H_c X_{c+1}
    real H = real(1), Gm = real(0);
#pragma unroll
    for (int u = ZMAXM - 1; u >= 0; --u) {
        Gm = fmad(Hv[u], Gm, Gv[u]);
        H *= Hv[u];
    }
    __syncthreads();
    sF[sgm][lane] = H;
    sB[sgm][lane] = Gm;
    __syncthreads();
    real X = real(0);
    for (int v = SEG - 1; v > sgm; --v) X = fmad(sF[v][lane], X, sB[v][lane]);
#pragma unroll
    for (int u = ZMAXM - 1; u >= 0; --u) {
        if (col && u < m && c0 + u < nch) zc[(c0 + u) * st + Nr + i] = X;
        X = fmad(Hv[u], X, Gv[u]);
    }
}

}  // namespace heat
