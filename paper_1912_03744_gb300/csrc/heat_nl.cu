// heat_nl.cu -- the paper's full method on the GPU (FP64): temperature-
// dependent coefficients with the simple iteration, adaptive tau and the
// pulsed source, on the paper's own non-rectangular layout (declared in
// include/heat.h, the heat_nl_* entry points).
//
//   Sec. 3, eq. "iter_scheme_eq_1": half-step 1 iterates T^s -> T^{s+1}; per
//       r-line a tridiagonal system whose mass term C(T^s)/(tau/2), source
//       X(T^s) and r-couplings (conductivities at T^s) change every
//       iteration, with the z-operator applied explicitly to the old layer T
//       (its conductivities at T).
//   Sec. 3, eq. "iter_scheme_eq_2": half-step 2 iterates per z-line with the
//       z-couplings at T^s; C, X and the explicit r-operator at Tbar.
//   Sec. 3, eq. "iter_cond": an iteration ends when max |T^{s+1} - T^s| < eps.
//   Sec. 3 / Sec. 4: s_max iterations without meeting it halve tau and restart
//       the step from the old layer; each step starts from the estimate
//       t_trs/1000 inside a transition of the source, t_src/100 elsewhere
//       (the caller passes both); the last step is shortened to end at t_end,
//       and a step outside a transition to end at the next switch.
//   Sec. 2, eqs. "source", "unit_model", "trans_model": X = chi(T) j^2 p(t),
//       p evaluated at t + tau/2.
//   Sec. 3, eq. "grid": row j holds the cells i = 0 .. N_j - 1 and column i
//       the cells j = 0 .. M_i - 1: the domain r <= r_max(z), z <= z_max(r)
//       is not a rectangle, and the field is stored that way.
// Material laws are per-region tables at temperature knots, read by linear
// interpolation (flat beyond the end knots); face conductivities are the
// harmonic (or arithmetic) means of the two cells' own conductivities, as in
// the constant case.
//
// Layout.  Row j is stored up to its last active cell (N_j cells; void cells
// before it stay, as identity rows), rows one after the other ("row-packed",
// the layout of half-step 1); the same for columns ("column-packed", M_i cells
// per column, the layout of half-step 2, so that its lines are contiguous
// too).  Void cells past the last active cell of their line are not stored.
// Between the half-steps the half layer is carried from the row-packed to the
// column-packed layout, and the new layer back, by 32 x 32 tiles through
// shared memory (coalesced on both sides); the kernel that builds half-step
// 2's fixed terms does the first transpose on the way.
//
// Kernels.  The coefficients change every iteration, so nothing is
// factorised ahead.  Per half-step, one kernel forms what stays fixed during
// its iteration (half-step 1: the explicit z-operator on the old layer;
// half-step 2: the mass term C(Tbar)/(tau/2) and the right-hand side with
// the explicit r-operator and X at Tbar).  Each iteration is then one kernel
// that assembles and solves every line of its layout, a block of NW warps per
// line: the block assembles the line's tridiagonal system into shared memory
// (coalesced), then solves it as three chunked scans (thread t holds a chunk
// of K consecutive cells, K odd so that the threads' shared-memory rows fall
// in distinct banks):
//   pivots    the Thomas pivots m_i = b_i - a_i c'_{i-1} follow from the linear
//             recurrence (p_i, q_i) = M_i (p_{i-1}, q_{i-1}), M_i = [[0, c_i],
//             [-a_i, b_i]], as m_i = q_i / q_{i-1} and c'_i = p_i / q_i; a chunk
//             is the product of its M_i, the threads scan these 2x2 products
//             (rescaled by powers of two; warp shuffles, then the warps' totals
//             through shared memory) and each rewalks its chunk from its exact
//             incoming (p, q);
//   forward   d'_i = d_i / m_i - (a_i / m_i) d'_{i-1}: an affine map per chunk,
//             scanned, rewalked;
//   backward  x_i = d'_i - c'_i x_{i+1}: the same, from the far end.
// A GB300 SM retires two FP64 FMAs per clock, so one line per thread would
// leave most SMs idle and the FP64 pipe of the busy ones saturated: a block
// per line spreads the lines over the SMs.
// Each block folds max |T^{s+1} - T^s| of its line into the iteration's slot
// with an integer atomicMax on the bit pattern (non-negative doubles order
// like their bits).  The host launches the iterations in small batches; an
// iteration whose predecessor's slot is already below eps returns at once, so
// a batch that converges early costs only empty launches, and the host reads
// the slots once per batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "heat_internal.h"

namespace heat {
int validate(const heat_geometry *, const heat_materials *, const heat_options *, double);
void build_grid(const heat_geometry *, Grid &);
}  // namespace heat

using namespace heat;

namespace {

constexpr int kTile = 32;  // transpose tile

// Material tables and the two packed layouts.
struct NlArgs {
    int Nr, Nz, K, face_mean;
    const int *offr;             // [Nz + 1] row-packed: row j at offr[j], N_j = offr[j+1] - offr[j]
    const int *offz;             // [Nr + 1] column-packed: column i at offz[i], M_i = offz[i+1] - offz[i]
    const signed char *regr;     // region of each row-packed cell, -1 void
    const signed char *regz;     // region of each column-packed cell
    const double *dr, *dz;       // cell widths
    // geometric factors of the couplings (Sec. 3, eqs. "Lambda_r", "Lambda_z"):
    //   A-_r = gm[i] k_{i-1/2}, A+_r = gp[i] k_{i+1/2}, Dirichlet r faces 2 gm[0] k, 2 gp[Nr-1] k;
    //   A-_z = zm[j] k_{j-1/2}, A+_z = zp[j] k_{j+1/2}, Dirichlet z faces 2 zm[0] k, 2 zp[Nz-1] k
    const double *gm, *gp, *zm, *zp;
    const double *Tk;            // [R][K] knots
    const double *tab;           // [R][K][6]: k, dk/dT, C, dC/dT, chi, dchi/dT on [Tk[k], Tk[k+1])
    const double *j2;            // [R]
    int bc[4];
    double Tbc[4];
};

// One direction's lines: line l is stored at off[l] .. off[l+1]-1; position p
// along it is cell p of the full grid axis of N cells.
struct LineSet {
    const int *off;
    const signed char *reg;
    const double *gm, *gp, *hw;  // coupling factors and half cell widths along the line (length N)
    int N;                       // full axis length (Dirichlet faces are at 0 and N - 1)
    int bc_lo, bc_hi;
    double T_lo, T_hi;
};

// A law at T: the value at the knot below plus the interval's slope times the
// distance (flat below the first and beyond the last knot).  f = 0 k, 2 C, 4 chi.
__device__ __forceinline__ double law(const NlArgs &A, int m, int f, double T)
{
    const double *tk = A.Tk + (size_t)m * A.K;
    const double *tb = A.tab + (size_t)m * A.K * 6;
    if (A.K == 1 || T <= tk[0]) return tb[f];
    if (T >= tk[A.K - 1]) return tb[(A.K - 1) * 6 + f];
    int k = 0;
    while (T >= tk[k + 1]) ++k;
    return fma(tb[k * 6 + f + 1], T - tk[k], tb[k * 6 + f]);
}

// Face conductivity between cells of conductivities ka, kb and half widths da, db.
__device__ __forceinline__ double face(double ka, double kb, double da, double db, int fm)
{
    return fm ? 0.5 * (ka + kb) : (da + db) * ka * kb / (da * kb + db * ka);
}

// Row-packed index of cell (i, j), or -1 past the row's last stored cell.
__device__ __forceinline__ int at_r(const NlArgs &A, int i, int j)
{
    const int o = A.offr[j];
    return i < A.offr[j + 1] - o ? o + i : -1;
}
// Column-packed index of cell (i, j), or -1.
__device__ __forceinline__ int at_z(const NlArgs &A, int i, int j)
{
    const int o = A.offz[i];
    return j < A.offz[i + 1] - o ? o + j : -1;
}

__device__ __forceinline__ void fold_max(unsigned long long *slot, double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
        b = x > b ? x : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(slot, b);
}

__device__ __forceinline__ bool converged_before(const unsigned long long *slots, int s, double eps)
{
    return s > 0 && __longlong_as_double((long long)slots[s - 1]) < eps;
}

// Half-step 1, fixed part: the explicit z-operator of eq. "iter_scheme_eq_1"
// on the old layer T (row-packed), conductivities at T (0 on void cells).
// Block (128): a stretch of one row.
__global__ void nl_zexp_kernel(NlArgs A, const double *__restrict__ T, double *__restrict__ E)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = at_r(A, i, j);
    if (c < 0) return;
    const int m = A.regr[c];
    double lz = 0.0;
    if (m >= 0) {
        const int Nz = A.Nz;
        const double t = T[c], k = law(A, m, 0, t);
        const int cm = j > 0 ? at_r(A, i, j - 1) : -1, cp = j < Nz - 1 ? at_r(A, i, j + 1) : -1;
        if (cm >= 0 && A.regr[cm] >= 0)
            lz += A.zm[j] * face(law(A, A.regr[cm], 0, T[cm]), k, 0.5 * A.dz[j - 1], 0.5 * A.dz[j], A.face_mean) *
                  (T[cm] - t);
        if (cp >= 0 && A.regr[cp] >= 0)
            lz += A.zp[j] * face(k, law(A, A.regr[cp], 0, T[cp]), 0.5 * A.dz[j], 0.5 * A.dz[j + 1], A.face_mean) *
                  (T[cp] - t);
        if (j == 0 && A.bc[2] == HEAT_BC_DIRICHLET) lz += 2.0 * A.zm[0] * k * (A.Tbc[2] - t);
        if (j == Nz - 1 && A.bc[3] == HEAT_BC_DIRICHLET) lz += 2.0 * A.zp[Nz - 1] * k * (A.Tbc[3] - t);
    }
    E[c] = lz;
}

// Half-step 2, fixed part, and the transpose to the column-packed layout:
// from Tbar (row-packed) forms, for every column-packed cell, Tbar itself,
// W = C(Tbar)/(tau/2) and F = W Tbar + Lambda_r[Tbar] + X(Tbar) of eq.
// "iter_scheme_eq_2" (conductivities of the explicit r-operator at Tbar;
// W = 1, F = Tbar on void).  A 32 x 32 tile of (i, j) per block (32 x 8
// threads): Tbar of columns i0-1 .. i0+32 is read along rows, the results are
// written along columns.
__global__ void __launch_bounds__(256) nl_rexp_kernel(NlArgs A, const double *__restrict__ Tb, double w2, double pt,
                                                      double *__restrict__ Tz, double *__restrict__ W,
                                                      double *__restrict__ F)
{
    __shared__ double sT[kTile][kTile + 3];   // [j][i - i0 + 1]
    __shared__ signed char sR[kTile][kTile + 3];
    __shared__ double sW[kTile][kTile + 1], sF[kTile][kTile + 1];  // [i][j]
    const int Nr = A.Nr, Nz = A.Nz;
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int jj = ty; jj < kTile; jj += 8) {
        const int j = j0 + jj;
        for (int ii = tx; ii < kTile + 2; ii += 32) {
            const int i = i0 + ii - 1;
            int c = -1;
            if (j < Nz && i >= 0 && i < Nr) c = at_r(A, i, j);
            sT[jj][ii] = c >= 0 ? Tb[c] : 0.0;
            sR[jj][ii] = c >= 0 ? A.regr[c] : (signed char)-1;
        }
    }
    __syncthreads();
    for (int jj = ty; jj < kTile; jj += 8) {
        const int j = j0 + jj, i = i0 + tx;
        if (j >= Nz || i >= Nr) continue;
        const int m = sR[jj][tx + 1];
        const double t = sT[jj][tx + 1];
        double w = 1.0, f = t;
        if (m >= 0) {
            const double k = law(A, m, 0, t);
            double lr = 0.0;
            if (sR[jj][tx] >= 0)
                lr += A.gm[i] * face(law(A, sR[jj][tx], 0, sT[jj][tx]), k, 0.5 * A.dr[i - 1], 0.5 * A.dr[i],
                                     A.face_mean) * (sT[jj][tx] - t);
            if (sR[jj][tx + 2] >= 0)
                lr += A.gp[i] * face(k, law(A, sR[jj][tx + 2], 0, sT[jj][tx + 2]), 0.5 * A.dr[i], 0.5 * A.dr[i + 1],
                                     A.face_mean) * (sT[jj][tx + 2] - t);
            if (i == 0 && A.bc[0] == HEAT_BC_DIRICHLET) lr += 2.0 * A.gm[0] * k * (A.Tbc[0] - t);
            if (i == Nr - 1 && A.bc[1] == HEAT_BC_DIRICHLET) lr += 2.0 * A.gp[Nr - 1] * k * (A.Tbc[1] - t);
            w = law(A, m, 2, t) * w2;
            const double xs = A.j2[m] != 0.0 ? law(A, m, 4, t) * A.j2[m] * pt : 0.0;
            f = w * t + lr + xs;
        }
        sW[tx][jj] = w;
        sF[tx][jj] = f;
    }
    __syncthreads();
    for (int ii = ty; ii < kTile; ii += 8) {
        const int i = i0 + ii, j = j0 + tx;
        if (i >= Nr || j >= Nz) continue;
        const int c = at_z(A, i, j);
        if (c < 0) continue;
        Tz[c] = sT[tx][ii + 1];
        W[c] = sW[ii][tx];
        F[c] = sF[ii][tx];
    }
}

// The new layer from the column-packed to the row-packed layout (32 x 32
// tiles).  Row-packed cells with no column-packed twin are void cells past
// their column's last active cell: they keep their value.
__global__ void __launch_bounds__(256) nl_zr_transpose_kernel(NlArgs A, const double *__restrict__ Tz,
                                                              double *__restrict__ Tr)
{
    __shared__ double s[kTile][kTile + 1];  // [i][j]
    __shared__ bool ok[kTile][kTile + 1];
    const int Nr = A.Nr, Nz = A.Nz;
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int ii = ty; ii < kTile; ii += 8) {
        const int i = i0 + ii, j = j0 + tx;
        const int c = (i < Nr && j < Nz) ? at_z(A, i, j) : -1;
        ok[ii][tx] = c >= 0;
        s[ii][tx] = c >= 0 ? Tz[c] : 0.0;
    }
    __syncthreads();
    for (int jj = ty; jj < kTile; jj += 8) {
        const int j = j0 + jj, i = i0 + tx;
        if (i >= Nr || j >= Nz || !ok[tx][jj]) continue;
        const int c = at_r(A, i, j);
        if (c >= 0) Tr[c] = s[tx][jj];
    }
}

// 2^-e for the exponent e of |x|, to rescale a 2x2 product (x = 0: 2^1023).
__device__ __forceinline__ double pow2_inv_scale(double x)
{
    const long long b = __double_as_longlong(x) & 0x7ff0000000000000LL;
    const long long e = b >> 52;   // biased exponent of |x|
    const long long k = 2046 - e;  // biased exponent of 2^-(e - 1023)
    return __longlong_as_double((k < 1 ? 1 : (k > 2046 ? 2046 : k)) << 52);
}

struct Mat2 {
    double a, b, c, d;  // [[a, b], [c, d]]
};
// x y, rescaled by a power of two (only the ratios of the second column matter)
__device__ __forceinline__ Mat2 mul_scaled(const Mat2 &x, const Mat2 &y)
{
    Mat2 r{fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c), fma(x.c, y.b, x.d * y.d)};
    const double s = pow2_inv_scale(fabs(r.d) > fabs(r.c) ? r.d : r.c);
    return {r.a * s, r.b * s, r.c * s, r.d * s};
}
__device__ __forceinline__ Mat2 shfl_up_mat(const Mat2 &x, int o)
{
    return {__shfl_up_sync(0xffffffffu, x.a, o), __shfl_up_sync(0xffffffffu, x.b, o),
            __shfl_up_sync(0xffffffffu, x.c, o), __shfl_up_sync(0xffffffffu, x.d, o)};
}

// One iteration of a half-step for every line of a layout: block (NW warps)
// = line blockIdx.x.  KIND 1: eq. "iter_scheme_eq_1" on the row-packed
// r-lines, fix0 = the old layer T, fix1 = its explicit z-operator, mass term
// and source at the iterate.  KIND 2: eq. "iter_scheme_eq_2" on the
// column-packed z-lines, fix0 = W, fix1 = F.  Ts: T^s, Tn: T^{s+1} (same
// layout).  Shared memory: five rows of the longest line (a, b, c, d and the
// face conductivities) and the warps' scan totals.
template <int KIND>
__global__ void __launch_bounds__(256) nl_line_kernel(NlArgs A, LineSet Ls, const double *__restrict__ fix0,
                                                      const double *__restrict__ fix1, const double *__restrict__ Ts,
                                                      double *__restrict__ Tn, int Lmax, double w2, double pt,
                                                      double eps, unsigned long long *slots, int s)
{
    if (converged_before(slots, s, eps)) return;
    const int off = Ls.off[blockIdx.x], L = Ls.off[blockIdx.x + 1] - off;
    if (L == 0) return;  // (block-uniform)
    extern __shared__ double sm[];
    double *sa = sm, *sb = sm + Lmax, *sc = sm + 2 * Lmax, *sd = sm + 3 * Lmax, *sf = sm + 4 * Lmax;
    double *tot = sm + 5 * Lmax;  // [NW][4]
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, NW = nt >> 5;
    const signed char *rg = Ls.reg + off;
    const double *ts = Ts + off;
    // conductivities at the iterate, then the faces p+1/2 (0 next to void)
    for (int p = tid; p < L; p += nt) sa[p] = rg[p] >= 0 ? law(A, rg[p], 0, ts[p]) : 0.0;
    __syncthreads();
    for (int p = tid; p < L - 1; p += nt)
        sf[p] = (rg[p] >= 0 && rg[p + 1] >= 0) ? face(sa[p], sa[p + 1], Ls.hw[p], Ls.hw[p + 1], A.face_mean) : 0.0;
    __syncthreads();
    // the line system a x_{p-1} + b x_p + c x_{p+1} = d (identity rows on void)
    for (int p = tid; p < L; p += nt) {
        const int m = rg[p];
        const double f0 = fix0[off + p], f1 = fix1[off + p];
        double a = 0.0, b = 1.0, c = 0.0, d = KIND == 1 ? f0 : f1;
        if (m >= 0) {
            const double am = p > 0 ? Ls.gm[p] * sf[p - 1] : 0.0;
            const double ap = p < L - 1 ? Ls.gp[p] * sf[p] : 0.0;
            const double dlo = (p == 0 && Ls.bc_lo == HEAT_BC_DIRICHLET) ? 2.0 * Ls.gm[0] * sa[p] : 0.0;
            const double dhi = (p == Ls.N - 1 && Ls.bc_hi == HEAT_BC_DIRICHLET) ? 2.0 * Ls.gp[p] * sa[p] : 0.0;
            double wm;
            if (KIND == 1) {
                wm = law(A, m, 2, ts[p]) * w2;
                const double xs = A.j2[m] != 0.0 ? law(A, m, 4, ts[p]) * A.j2[m] * pt : 0.0;
                d = wm * f0 + f1 + xs;
            } else {
                wm = f0;
                d = f1;
            }
            a = -am;
            c = -ap;
            b = wm + am + ap + dlo + dhi;
            d += dlo * Ls.T_lo + dhi * Ls.T_hi;
        }
        sa[p] = a, sb[p] = b, sc[p] = c, sd[p] = d;  // each thread rewrites only its own cells
    }
    __syncthreads();
    int K = (L + nt - 1) / nt;
    K |= 1;  // odd: the threads' rows of K doubles fall in distinct bank pairs
    const int p0 = min(tid * K, L), p1 = min(p0 + K, L);

    // ---- pivots: chunk product P = M_{p1-1} ... M_{p0}, M_p = [[0, c_p], [-a_p, b_p]]
    Mat2 P{1.0, 0.0, 0.0, 1.0};
    for (int p = p0; p < p1; ++p) P = mul_scaled(Mat2{0.0, sc[p], -sa[p], sb[p]}, P);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // inclusive within the warp, later chunks on the left
        const Mat2 Q = shfl_up_mat(P, o);
        if (lane >= o) P = mul_scaled(P, Q);
    }
    if (lane == 31) tot[w * 4 + 0] = P.a, tot[w * 4 + 1] = P.b, tot[w * 4 + 2] = P.c, tot[w * 4 + 3] = P.d;
    __syncthreads();
    // (p, q) entering the chunk: the earlier warps' totals, then the earlier
    // lanes' product, applied to (0, 1)
    double pp = 0.0, qq = 1.0;
    for (int v = 0; v < w; ++v) {
        const double np = fma(tot[v * 4 + 0], pp, tot[v * 4 + 1] * qq);
        const double nq = fma(tot[v * 4 + 2], pp, tot[v * 4 + 3] * qq);
        const double sc2 = pow2_inv_scale(nq);
        pp = np * sc2, qq = nq * sc2;
    }
    {
        const Mat2 E = shfl_up_mat(P, 1);
        if (lane > 0) {
            const double np = fma(E.a, pp, E.b * qq), nq = fma(E.c, pp, E.d * qq);
            pp = np, qq = nq;
        }
    }
    __syncthreads();  // tot is reused below
    // rewalk: 1/m_p -> sb, c'_p -> sc; forward map of the chunk (G, H): d'_out = G + H d'_in
    double G = 0.0, H = 1.0;
    for (int p = p0; p < p1; ++p) {
        const double a = sa[p], b = sb[p], c = sc[p];
        const double pn = c * qq, qn = fma(b, qq, -a * pp);
        const double r = 1.0 / qn;
        const double inv_m = qq * r;
        sb[p] = inv_m;
        sc[p] = pn * r;
        G = fma(-a * inv_m, G, sd[p] * inv_m);
        H = -a * inv_m * H;
        const double sc2 = pow2_inv_scale(qn);
        pp = pn * sc2, qq = qn * sc2;
    }
    // ---- forward substitution: scan of the affine maps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double g2 = __shfl_up_sync(0xffffffffu, G, o), h2 = __shfl_up_sync(0xffffffffu, H, o);
        if (lane >= o) G = fma(H, g2, G), H = H * h2;
    }
    if (lane == 31) tot[w * 2 + 0] = G, tot[w * 2 + 1] = H;
    __syncthreads();
    double dp = 0.0;
    for (int v = 0; v < w; ++v) dp = fma(tot[v * 2 + 1], dp, tot[v * 2]);
    {
        const double ge = __shfl_up_sync(0xffffffffu, G, 1), he = __shfl_up_sync(0xffffffffu, H, 1);
        if (lane > 0) dp = fma(he, dp, ge);
    }
    __syncthreads();
    for (int p = p0; p < p1; ++p) {
        dp = fma(-sa[p] * sb[p], dp, sd[p] * sb[p]);
        sd[p] = dp;
    }
    // ---- backward substitution x_p = d'_p - c'_p x_{p+1}: chunk map x_{p0} = G + H x_{p1}
    G = 0.0, H = 1.0;
    for (int p = p1 - 1; p >= p0; --p) {
        G = fma(-sc[p], G, sd[p]);
        H = -sc[p] * H;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double g2 = __shfl_down_sync(0xffffffffu, G, o), h2 = __shfl_down_sync(0xffffffffu, H, o);
        if (lane + o < 32) G = fma(H, g2, G), H = H * h2;
    }
    if (lane == 0) tot[w * 2 + 0] = G, tot[w * 2 + 1] = H;
    __syncthreads();
    double x = 0.0;
    for (int v = NW - 1; v > w; --v) x = fma(tot[v * 2 + 1], x, tot[v * 2]);
    {
        const double ge = __shfl_down_sync(0xffffffffu, G, 1), he = __shfl_down_sync(0xffffffffu, H, 1);
        if (lane < 31) x = fma(he, x, ge);
    }
    for (int p = p1 - 1; p >= p0; --p) {
        x = fma(-sc[p], x, sd[p]);
        sa[p] = x;
    }
    __syncthreads();
    double diff = 0.0;
    for (int p = tid; p < L; p += nt) {
        const double v = sa[p];
        Tn[off + p] = v;
        diff = fmax(diff, fabs(v - ts[p]));
    }
    fold_max(slots + s, diff);
}

__global__ void nl_fill_kernel(double *__restrict__ T, size_t n, double v)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) T[c] = v;
}

int cuda_st(cudaError_t e)
{
    if (e == cudaSuccess) return HEAT_OK;
    return e == cudaErrorMemoryAllocation ? HEAT_ERR_OOM : HEAT_ERR_CUDA;
}

// Warps per line block: about 16 cells per thread, 1..8 warps.
int warps_for(int Lmax)
{
    int nw = 1;
    while (nw < 8 && 32 * nw * 16 < Lmax) nw *= 2;
    return nw;
}

}  // namespace

struct heat_nl {
    cudaStream_t stream = nullptr;
    int device = -1;
    Grid g;
    NlArgs A{};
    LineSet rl{}, zl{};           // r-lines (row-packed), z-lines (column-packed)
    int Lr_max = 0, Lz_max = 0;   // longest row / column
    int nw_r = 1, nw_z = 1;       // warps per line block
    long long n_rows_packed = 0, n_cols_packed = 0;
    std::vector<int> offr, offz;  // host copies of the layouts
    heat_pulse pulse{};
    heat_nl_options opt{};
    double T_init = 0.0;
    double t = 0.0;
    // device buffers: row-packed T, Tbar, iterates, explicit z-operator;
    // column-packed Tbar, W, F, iterates
    double *d_T = nullptr, *d_Tbar = nullptr, *d_it[2] = {nullptr, nullptr}, *d_E = nullptr;
    double *d_Tz = nullptr, *d_W = nullptr, *d_F = nullptr, *d_itz[2] = {nullptr, nullptr};
    unsigned long long *d_slots = nullptr;
    unsigned long long *h_slots = nullptr;  // pinned
    std::vector<void *> owned;              // every other device allocation
    long long launches = 0;
};

namespace {

// p(t) of eq. "unit_model" (model 1) or eq. "trans_model" (model 2); 1 for model 0.
double pulse_at(const heat_pulse &P, double t)
{
    if (P.model == HEAT_PULSE_CONST) return 1.0;
    int last = (int)std::floor(t / P.t_per) + 1;  // later pulses add exact zeros
    if (last < 0) last = 0;
    double s = 0.0;
    for (int n = 0; n <= last; ++n) {
        const double on = t - n * P.t_per, off = on - P.t_src;
        if (P.model == HEAT_PULSE_RECT)
            s += (on >= 0.0 ? 1.0 : 0.0) - (off >= 0.0 ? 1.0 : 0.0);
        else
            s += 0.5 * (std::erf(P.xi * (P.zeta * on / P.t_trs - 1.0)) - std::erf(P.xi * (P.zeta * off / P.t_trs - 1.0)));
    }
    return s;
}

template <typename T>
int upload(heat_nl *s, const std::vector<T> &h, const T **out)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, h.size()) * sizeof(T));
    if (e != cudaSuccess) return cuda_st(e);
    s->owned.push_back(p);
    if (!h.empty() && (e = cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream)) !=
                          cudaSuccess)
        return cuda_st(e);
    *out = static_cast<const T *>(p);
    return HEAT_OK;
}

void free_nl(heat_nl *s)
{
    if (!s) return;
    for (void *p : {(void *)s->d_T, (void *)s->d_Tbar, (void *)s->d_it[0], (void *)s->d_it[1], (void *)s->d_E,
                    (void *)s->d_Tz, (void *)s->d_W, (void *)s->d_F, (void *)s->d_itz[0], (void *)s->d_itz[1],
                    (void *)s->d_slots})
        if (p) cudaFree(p);
    for (void *p : s->owned) cudaFree(p);
    if (s->h_slots) cudaFreeHost(s->h_slots);
    delete s;
}

constexpr int kBatch = 3;  // iterations launched between two reads of the slots
constexpr int kNlMaxN = HEAT_NL_MAX_N;  // a line's five rows of doubles fit one block's shared memory

size_t line_smem(int Lmax, int nw) { return (5 * (size_t)Lmax + 4 * (size_t)nw) * sizeof(double); }

// One half-step's iteration (dir 0: eq. "iter_scheme_eq_1" from T on the
// row-packed layout; dir 1: eq. "iter_scheme_eq_2" from Tbar on the
// column-packed layout).  Returns the number of iterations used (the result
// is then in the layout's iterate buffer (used - 1) % 2), 0 if s_max were
// not enough, or a negative status.
int run_half(heat_nl *s, int dir, double tau, double pt)
{
    const int s_max = s->opt.s_max;
    const double w2 = 2.0 / tau;
    const NlArgs &A = s->A;
    cudaError_t e = cudaMemsetAsync(s->d_slots, 0, sizeof(unsigned long long) * s_max, s->stream);
    if (e != cudaSuccess) return cuda_st(e);
    const dim3 tiles((A.Nr + kTile - 1) / kTile, (A.Nz + kTile - 1) / kTile), tile_block(32, 8);
    if (dir == 0)
        nl_zexp_kernel<<<dim3((s->Lr_max + 127) / 128, A.Nz), 128, 0, s->stream>>>(A, s->d_T, s->d_E);
    else
        nl_rexp_kernel<<<tiles, tile_block, 0, s->stream>>>(A, s->d_Tbar, w2, pt, s->d_Tz, s->d_W, s->d_F);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_st(e);
    ++s->launches;
    const int nw = dir == 0 ? s->nw_r : s->nw_z, Lmax = dir == 0 ? s->Lr_max : s->Lz_max;
    const size_t smem = line_smem(Lmax, nw);
    const int lines = dir == 0 ? A.Nz : A.Nr;
    for (int s0 = 0; s0 < s_max; s0 += kBatch) {
        const int nb = std::min(kBatch, s_max - s0);
        for (int b = 0; b < nb; ++b) {
            const int it = s0 + b;
            if (dir == 0) {
                const double *Ts = it == 0 ? s->d_T : s->d_it[(it - 1) % 2];
                nl_line_kernel<1><<<lines, 32 * nw, smem, s->stream>>>(A, s->rl, s->d_T, s->d_E, Ts, s->d_it[it % 2],
                                                                       Lmax, w2, pt, s->opt.eps, s->d_slots, it);
            } else {
                const double *Ts = it == 0 ? s->d_Tz : s->d_itz[(it - 1) % 2];
                nl_line_kernel<2><<<lines, 32 * nw, smem, s->stream>>>(A, s->zl, s->d_W, s->d_F, Ts, s->d_itz[it % 2],
                                                                       Lmax, w2, pt, s->opt.eps, s->d_slots, it);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_st(e);
            ++s->launches;
        }
        if ((e = cudaMemcpyAsync(s->h_slots + s0, s->d_slots + s0, nb * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
            return cuda_st(e);
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_st(e);
        for (int b = 0; b < nb; ++b) {
            double v;
            std::memcpy(&v, &s->h_slots[s0 + b], sizeof(v));
            if (v < s->opt.eps) return s0 + b + 1;
        }
    }
    return 0;
}

// One step of length tau from s->t without halving: HEAT_OK (field advanced,
// time not), HEAT_ERR_NOCONV (field unchanged), or an error.
int try_step(heat_nl *s, double tau, int *it1, int *it2)
{
    const double pt = pulse_at(s->pulse, s->t + 0.5 * tau);
    *it1 = *it2 = 0;
    int u = run_half(s, 0, tau, pt);
    if (u < 0) return u;
    if (u == 0) return HEAT_ERR_NOCONV;
    *it1 = u;
    std::swap(s->d_Tbar, s->d_it[(u - 1) % 2]);
    u = run_half(s, 1, tau, pt);
    if (u < 0) return u;
    if (u == 0) return HEAT_ERR_NOCONV;
    *it2 = u;
    // the new layer back to the row-packed layout
    const dim3 tiles((s->A.Nr + kTile - 1) / kTile, (s->A.Nz + kTile - 1) / kTile);
    nl_zr_transpose_kernel<<<tiles, dim3(32, 8), 0, s->stream>>>(s->A, s->d_itz[(u - 1) % 2], s->d_T);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_st(e);
    ++s->launches;
    return HEAT_OK;
}

}  // namespace

extern "C" {

int heat_nl_create(const heat_geometry *geom, const heat_nl_materials *mat, const heat_pulse *pulse,
                   const heat_nl_options *opt, void *stream, heat_nl **out)
{
    if (!out) return HEAT_ERR_ARG;
    *out = nullptr;
    if (!geom || !mat || !pulse || !opt) return HEAT_ERR_ARG;
    const int R = mat->n_regions, K = mat->n_knots;
    if (R < 1 || R > 127 || K < 1 || K > 1024 || !mat->T_knots || !mat->k || !mat->C || !mat->chi || !mat->j2)
        return HEAT_ERR_ARG;
    for (int m = 0; m < R; ++m) {
        for (int k = 0; k < K; ++k) {
            const size_t x = (size_t)m * K + k;
            if (!std::isfinite(mat->T_knots[x]) || !(mat->k[x] > 0.0) || !(mat->C[x] > 0.0) ||
                !std::isfinite(mat->k[x]) || !std::isfinite(mat->C[x]) || !std::isfinite(mat->chi[x]))
                return HEAT_ERR_ARG;
            if (k > 0 && !(mat->T_knots[x] > mat->T_knots[x - 1])) return HEAT_ERR_ARG;
        }
        if (!std::isfinite(mat->j2[m])) return HEAT_ERR_ARG;
    }
    if (pulse->model < HEAT_PULSE_CONST || pulse->model > HEAT_PULSE_ERF) return HEAT_ERR_ARG;
    if (pulse->model != HEAT_PULSE_CONST &&
        !(pulse->t_per > 0.0 && pulse->t_src > 0.0 && pulse->t_src <= pulse->t_per && pulse->t_trs > 0.0 &&
          std::isfinite(pulse->xi) && std::isfinite(pulse->zeta)))
        return HEAT_ERR_ARG;
    if (!(opt->eps > 0.0) || opt->s_max < 1 || opt->s_max > 4096 || !(opt->tau_base > 0.0) ||
        !(opt->tau_trs > 0.0) || !(opt->tau_min > 0.0) ||
        (opt->face_mean != HEAT_HARMONIC && opt->face_mean != HEAT_ARITH))
        return HEAT_ERR_ARG;
    // the geometry checks of heat_create, with stand-in constant materials
    std::vector<double> one(R, 1.0), zero(R, 0.0);
    const heat_materials cm{R, one.data(), one.data(), zero.data(), mat->T_init};
    const heat_options co{HEAT_FP64, opt->face_mean};
    int st = validate(geom, &cm, &co, 1.0);
    if (st != HEAT_OK) return st;
    {
        long long Nr = 0, Nz = 0;
        for (int l = 0; l < geom->n_r_layers; ++l) Nr += geom->r_cells[l];
        for (int l = 0; l < geom->n_z_layers; ++l) Nz += geom->z_cells[l];
        if (Nr > kNlMaxN || Nz > kNlMaxN) return HEAT_ERR_ARG;
    }

    heat_nl *s = new (std::nothrow) heat_nl();
    if (!s) return HEAT_ERR_OOM;
    s->stream = static_cast<cudaStream_t>(stream);
    s->pulse = *pulse;
    s->opt = *opt;
    s->T_init = mat->T_init;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_st(e);
    }
    build_grid(geom, s->g);
    const Grid &g = s->g;
    const int Nr = g.Nr, Nz = g.Nz;
    auto fail = [&](int x) {
        free_nl(s);
        return x;
    };
    // region of each cell: the first box whose closed rectangle holds its centre
    std::vector<signed char> reg((size_t)Nr * Nz);
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nr; ++i) {
            int r = -1;
            for (int b = 0; b < geom->n_boxes && r < 0; ++b) {
                const heat_box &bx = geom->boxes[b];
                if (g.rc[i] >= bx.r0 && g.rc[i] <= bx.r1 && g.zc[j] >= bx.z0 && g.zc[j] <= bx.z1) r = bx.region;
            }
            reg[(size_t)j * Nr + i] = (signed char)r;
        }
    // the packed layouts: N_j = 1 + last active i of row j, M_i = 1 + last active j of column i
    std::vector<int> Nj(Nz, 0), Mi(Nr, 0);
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nr; ++i)
            if (reg[(size_t)j * Nr + i] >= 0) Nj[j] = i + 1, Mi[i] = std::max(Mi[i], j + 1);
    s->offr.assign(Nz + 1, 0);
    s->offz.assign(Nr + 1, 0);
    for (int j = 0; j < Nz; ++j) s->offr[j + 1] = s->offr[j] + Nj[j];
    for (int i = 0; i < Nr; ++i) s->offz[i + 1] = s->offz[i] + Mi[i];
    s->n_rows_packed = s->offr[Nz];
    s->n_cols_packed = s->offz[Nr];
    s->Lr_max = *std::max_element(Nj.begin(), Nj.end());
    s->Lz_max = *std::max_element(Mi.begin(), Mi.end());
    if (s->n_rows_packed == 0) return fail(HEAT_ERR_ARG);  // no active cell
    std::vector<signed char> regr(s->n_rows_packed), regz(s->n_cols_packed);
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nj[j]; ++i) regr[s->offr[j] + i] = reg[(size_t)j * Nr + i];
    for (int i = 0; i < Nr; ++i)
        for (int j = 0; j < Mi[i]; ++j) regz[s->offz[i] + j] = reg[(size_t)j * Nr + i];
    // tables: value and slope on each knot interval
    std::vector<double> tk(mat->T_knots, mat->T_knots + (size_t)R * K), tab((size_t)R * K * 6, 0.0);
    for (int m = 0; m < R; ++m)
        for (int k = 0; k < K; ++k) {
            const size_t x = (size_t)m * K + k;
            const double *v[3] = {mat->k, mat->C, mat->chi};
            for (int f = 0; f < 3; ++f) {
                tab[x * 6 + 2 * f] = v[f][x];
                tab[x * 6 + 2 * f + 1] = k + 1 < K ? (v[f][x + 1] - v[f][x]) / (tk[x + 1] - tk[x]) : 0.0;
            }
        }
    std::vector<double> j2(mat->j2, mat->j2 + R);
    // the couplings' geometric factors: r_{i-1/2} / (r_i hbar_i h_i), r_{i+1/2} / (r_i hbar_i h_{i+1}),
    // 1 / (etabar_j eta_j), 1 / (etabar_j eta_{j+1}); half widths
    std::vector<double> gm(Nr), gp(Nr), zm(Nz), zp(Nz), hr(Nr), hz(Nz);
    for (int i = 0; i < Nr; ++i) {
        gm[i] = g.rf[i] / (g.rc[i] * g.hbar[i] * g.h[i]);
        gp[i] = g.rf[i + 1] / (g.rc[i] * g.hbar[i] * g.h[i + 1]);
        hr[i] = 0.5 * g.dr[i];
    }
    for (int j = 0; j < Nz; ++j) {
        zm[j] = 1.0 / (g.etabar[j] * g.eta[j]);
        zp[j] = 1.0 / (g.etabar[j] * g.eta[j + 1]);
        hz[j] = 0.5 * g.dz[j];
    }
    NlArgs &A = s->A;
    A.Nr = Nr, A.Nz = Nz, A.K = K, A.face_mean = opt->face_mean;
    for (int f = 0; f < 4; ++f) A.bc[f] = geom->bc[f], A.Tbc[f] = geom->T_bc[f];
    const double *hrd = nullptr, *hzd = nullptr;
    if ((st = upload(s, s->offr, &A.offr)) != HEAT_OK || (st = upload(s, s->offz, &A.offz)) != HEAT_OK ||
        (st = upload(s, regr, &A.regr)) != HEAT_OK || (st = upload(s, regz, &A.regz)) != HEAT_OK ||
        (st = upload(s, g.dr, &A.dr)) != HEAT_OK || (st = upload(s, g.dz, &A.dz)) != HEAT_OK ||
        (st = upload(s, gm, &A.gm)) != HEAT_OK || (st = upload(s, gp, &A.gp)) != HEAT_OK ||
        (st = upload(s, zm, &A.zm)) != HEAT_OK || (st = upload(s, zp, &A.zp)) != HEAT_OK ||
        (st = upload(s, tk, &A.Tk)) != HEAT_OK || (st = upload(s, tab, &A.tab)) != HEAT_OK ||
        (st = upload(s, j2, &A.j2)) != HEAT_OK || (st = upload(s, hr, &hrd)) != HEAT_OK ||
        (st = upload(s, hz, &hzd)) != HEAT_OK)
        return fail(st);
    s->rl = LineSet{A.offr, A.regr, A.gm, A.gp, hrd, Nr, geom->bc[0], geom->bc[1], geom->T_bc[0], geom->T_bc[1]};
    s->zl = LineSet{A.offz, A.regz, A.zm, A.zp, hzd, Nz, geom->bc[2], geom->bc[3], geom->T_bc[2], geom->T_bc[3]};
    s->nw_r = warps_for(s->Lr_max);
    s->nw_z = warps_for(s->Lz_max);
    const size_t smem = std::max(line_smem(s->Lr_max, s->nw_r), line_smem(s->Lz_max, s->nw_z));
    if (smem > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(nl_line_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(nl_line_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
            return fail(cuda_st(e));
    }
    double **rbufs[5] = {&s->d_T, &s->d_Tbar, &s->d_it[0], &s->d_it[1], &s->d_E};
    double **zbufs[5] = {&s->d_Tz, &s->d_W, &s->d_F, &s->d_itz[0], &s->d_itz[1]};
    for (double **b : rbufs)
        if ((e = cudaMalloc(b, s->n_rows_packed * sizeof(double))) != cudaSuccess) return fail(cuda_st(e));
    for (double **b : zbufs)
        if ((e = cudaMalloc(b, s->n_cols_packed * sizeof(double))) != cudaSuccess) return fail(cuda_st(e));
    if ((e = cudaMalloc(&s->d_slots, opt->s_max * sizeof(unsigned long long))) != cudaSuccess) return fail(cuda_st(e));
    if ((e = cudaMallocHost(&s->h_slots, opt->s_max * sizeof(unsigned long long))) != cudaSuccess)
        return fail(cuda_st(e));
    nl_fill_kernel<<<256, 256, 0, s->stream>>>(s->d_T, s->n_rows_packed, mat->T_init);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_st(e));
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return fail(cuda_st(e));
    *out = s;
    return HEAT_OK;
}

int heat_nl_step(heat_nl *s, double tau, int *it1, int *it2)
{
    if (!s || !(tau > 0.0) || !std::isfinite(tau)) return HEAT_ERR_ARG;
    int a = 0, b = 0;
    const int st = try_step(s, tau, &a, &b);
    if (it1) *it1 = a;
    if (it2) *it2 = b;
    if (st == HEAT_OK) s->t += tau;
    return st;
}

int heat_nl_advance(heat_nl *s, double t_end, long long max_steps, heat_nl_stats *stats)
{
    if (!s || !std::isfinite(t_end) || max_steps < 0) return HEAT_ERR_ARG;
    heat_nl_stats st{};
    st.tau_smallest = INFINITY;
    int status = HEAT_OK;
    const heat_pulse &P = s->pulse;
    while (s->t < t_end) {
        if (st.steps >= max_steps) break;
        bool trs = false;
        double to_switch = INFINITY;
        if (P.model != HEAT_PULSE_CONST) {
            // the phase in the period; within tol of a switch counts as at it
            const double tol = 1e-9 * P.t_per;
            double ph = std::fmod(s->t, P.t_per);
            if (P.t_per - ph < tol) ph = 0.0;
            trs = ph < P.t_trs || (ph >= P.t_src - tol && ph < P.t_src + P.t_trs);
            if (!trs) to_switch = (ph < P.t_src ? P.t_src : P.t_per) - ph;
        }
        double tau = trs ? s->opt.tau_trs : s->opt.tau_base;
        if (tau > to_switch) tau = to_switch;  // no step passes over a transition
        bool last = tau >= t_end - s->t;
        if (last) tau = t_end - s->t;
        for (;;) {
            int it1, it2;
            status = try_step(s, tau, &it1, &it2);
            if (status == HEAT_OK) {
                st.iters1 += it1;
                st.iters2 += it2;
                break;
            }
            if (status != HEAT_ERR_NOCONV) break;
            tau *= 0.5;
            last = false;
            st.halvings += 1;
            if (tau < s->opt.tau_min) break;
        }
        if (status != HEAT_OK) break;
        s->t = last ? t_end : s->t + tau;
        st.steps += 1;
        if (tau < st.tau_smallest) st.tau_smallest = tau;
    }
    if (stats) *stats = st;
    return status;
}

int heat_nl_time(heat_nl *s, double *t)
{
    if (!s || !t) return HEAT_ERR_ARG;
    *t = s->t;
    return HEAT_OK;
}

int heat_nl_set_time(heat_nl *s, double t)
{
    if (!s || !std::isfinite(t)) return HEAT_ERR_ARG;
    s->t = t;
    return HEAT_OK;
}

}  // extern "C"

namespace {

// A row-packed device field to a rectangular [Nz][Nr] array (host or device;
// cells not stored read T_init), or back (cells not stored are dropped).
int nl_to_rect(heat_nl *s, const double *packed, double *rect, int on_device)
{
    const int Nr = s->g.Nr, Nz = s->g.Nz;
    std::vector<double> host(s->n_rows_packed), full((size_t)Nr * Nz, s->T_init);
    cudaError_t e = cudaMemcpyAsync(host.data(), packed, host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_st(e);
    for (int j = 0; j < Nz; ++j)
        std::memcpy(&full[(size_t)j * Nr], &host[s->offr[j]], (s->offr[j + 1] - s->offr[j]) * sizeof(double));
    if (!on_device) {
        std::memcpy(rect, full.data(), full.size() * sizeof(double));
        return HEAT_OK;
    }
    e = cudaMemcpyAsync(rect, full.data(), full.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_st(e);
}

int nl_from_rect(heat_nl *s, const double *rect, double *packed, int on_device)
{
    const int Nr = s->g.Nr, Nz = s->g.Nz;
    std::vector<double> host(s->n_rows_packed), full;
    const double *src = rect;
    cudaError_t e;
    if (on_device) {
        full.resize((size_t)Nr * Nz);
        e = cudaMemcpyAsync(full.data(), rect, full.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_st(e);
        src = full.data();
    }
    for (int j = 0; j < Nz; ++j)
        std::memcpy(&host[s->offr[j]], src + (size_t)j * Nr, (s->offr[j + 1] - s->offr[j]) * sizeof(double));
    e = cudaMemcpyAsync(packed, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_st(e);
}

}  // namespace

extern "C" {

int heat_nl_field(heat_nl *s, double *out, size_t n, int on_device)
{
    if (!s || !out || n != (size_t)s->g.Nr * s->g.Nz) return HEAT_ERR_ARG;
    return nl_to_rect(s, s->d_T, out, on_device);
}

int heat_nl_half_field(heat_nl *s, double *out, size_t n, int on_device)
{
    if (!s || !out || n != (size_t)s->g.Nr * s->g.Nz) return HEAT_ERR_ARG;
    return nl_to_rect(s, s->d_Tbar, out, on_device);
}

int heat_nl_set_field(heat_nl *s, const double *in, size_t n, int on_device)
{
    if (!s || !in || n != (size_t)s->g.Nr * s->g.Nz) return HEAT_ERR_ARG;
    return nl_from_rect(s, in, s->d_T, on_device);
}

int heat_nl_layout(heat_nl *s, int *N_j, int *M_i, long long *stored)
{
    if (!s) return HEAT_ERR_ARG;
    if (N_j)
        for (int j = 0; j < s->g.Nz; ++j) N_j[j] = s->offr[j + 1] - s->offr[j];
    if (M_i)
        for (int i = 0; i < s->g.Nr; ++i) M_i[i] = s->offz[i + 1] - s->offz[i];
    if (stored) *stored = s->n_rows_packed;
    return HEAT_OK;
}

int heat_nl_field_packed(heat_nl *s, double *out, size_t n, int on_device)
{
    if (!s || !out || n != (size_t)s->n_rows_packed) return HEAT_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(out, s->d_T, n * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
    return cuda_st(e);
}

int heat_nl_info(heat_nl *s, int *Nr, int *Nz, long long *launches)
{
    if (!s) return HEAT_ERR_ARG;
    if (Nr) *Nr = s->g.Nr;
    if (Nz) *Nz = s->g.Nz;
    if (launches) *launches = s->launches;
    return HEAT_OK;
}

void heat_nl_destroy(heat_nl *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_nl(s);
}

}  // extern "C"
