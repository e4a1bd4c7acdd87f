// heat_nl.cu -- the paper's full method on the GPU (FP64): temperature-
// dependent coefficients with the simple iteration, adaptive tau and the
// pulsed source (declared in include/heat.h, the heat_nl_* entry points).
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
// Material laws are per-region tables at temperature knots, read by linear
// interpolation (flat beyond the end knots); face conductivities are the
// harmonic (or arithmetic) means of the two cells' own conductivities, as in
// the constant case.
//
// Kernels.  The coefficients change every iteration, so nothing is
// factorised ahead.  Per half-step, one kernel first forms what stays fixed
// during its iteration (half-step 1: the explicit z-operator on the old
// layer; half-step 2: the mass term C(Tbar)/(tau/2) and the right-hand side
// with the explicit r-operator and X at Tbar), per cell and coalesced.  Each
// iteration is then one kernel that assembles and solves every line of its
// direction:
//   r-lines: one warp per line.  The warp assembles the line's tridiagonal
//   system into shared memory with coalesced loads, then solves it as three
//   chunked scans (lane l holds a chunk of K consecutive cells, K odd so
//   that the lanes' shared-memory rows fall in distinct banks):
//     pivots      the Thomas pivots m_i = b_i - a_i c_{i-1}/m_{i-1} follow
//                 from the linear recurrence (p_i, q_i) = M_i (p_{i-1}, q_{i-1}),
//                 M_i = [[0, c_i], [-a_i, b_i]], as m_i = q_i / q_{i-1} and
//                 c'_i = p_i / q_i; a chunk is the product of its M_i, the lanes
//                 scan these 2x2 products (rescaled by powers of two) and each
//                 rewalks its chunk from its exact incoming (p, q);
//     forward     d'_i = d_i / m_i - (a_i / m_i) d'_{i-1}: an affine map per
//                 chunk, scanned, rewalked;
//     backward    x_i = d'_i - c'_i x_{i+1}: the same, from the far end.
//   A GB300 SM retires two FP64 FMAs per clock, so a line per thread leaves
//   most of the chip idle and the FP64 pipe of the few busy SMs saturated;
//   a warp per line spreads the lines over the SMs.
//   z-lines: one thread per column (neighbouring threads read neighbouring
//   columns, so every row access of a warp is contiguous), Thomas with c'
//   and d' in a scratch field.
// Each line folds max |T^{s+1} - T^s| into the iteration's slot with an
// integer atomicMax on the bit pattern (non-negative doubles order like
// their bits).  The host launches the iterations in small batches; an
// iteration whose predecessor's slot is already below eps returns at once,
// so a batch that converges early costs only empty launches, and the host
// reads the slots once per batch.
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

struct NlArgs {
    int Nr, Nz, K, face_mean;
    const signed char *region;  // [Nz][Nr], -1 void
    const double *dr, *dz;      // cell widths
    // geometric factors of the couplings (Sec. 3, eqs. "Lambda_r", "Lambda_z"):
    //   A-_r = gm[i] k_{i-1/2}, A+_r = gp[i] k_{i+1/2}, Dirichlet r faces 2 gm[0] k, 2 gp[Nr-1] k;
    //   A-_z = zm[j] k_{j-1/2}, A+_z = zp[j] k_{j+1/2}, Dirichlet z faces 2 zm[0] k, 2 zp[Nz-1] k
    const double *gm, *gp, *zm, *zp;
    const double *Tk;           // [R][K] knots
    const double *tab;          // [R][K][6]: k, dk/dT, C, dC/dT, chi, dchi/dT on [Tk[k], Tk[k+1])
    const double *j2;           // [R]
    int bc[4];
    double Tbc[4];
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
// on the old layer T, conductivities at T (0 on void cells).
__global__ void nl_zexp_kernel(NlArgs A, const double *__restrict__ T, double *__restrict__ E)
{
    const int Nr = A.Nr, Nz = A.Nz;
    const size_t n = (size_t)Nr * Nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int m = A.region[c];
        double lz = 0.0;
        if (m >= 0) {
            const int j = (int)(c / Nr);
            const double t = T[c], k = law(A, m, 0, t);
            if (j > 0 && A.region[c - Nr] >= 0)
                lz += A.zm[j] * face(law(A, A.region[c - Nr], 0, T[c - Nr]), k, 0.5 * A.dz[j - 1], 0.5 * A.dz[j],
                                     A.face_mean) * (T[c - Nr] - t);
            if (j < Nz - 1 && A.region[c + Nr] >= 0)
                lz += A.zp[j] * face(k, law(A, A.region[c + Nr], 0, T[c + Nr]), 0.5 * A.dz[j], 0.5 * A.dz[j + 1],
                                     A.face_mean) * (T[c + Nr] - t);
            if (j == 0 && A.bc[2] == HEAT_BC_DIRICHLET) lz += 2.0 * A.zm[0] * k * (A.Tbc[2] - t);
            if (j == Nz - 1 && A.bc[3] == HEAT_BC_DIRICHLET) lz += 2.0 * A.zp[Nz - 1] * k * (A.Tbc[3] - t);
        }
        E[c] = lz;
    }
}

// Half-step 2, fixed part: W = C(Tbar)/(tau/2) and the right-hand side
// F = W Tbar + Lambda_r[Tbar] + X(Tbar) of eq. "iter_scheme_eq_2"
// (conductivities of the explicit r-operator at Tbar; F = Tbar, W = 1 on void).
__global__ void nl_rexp_kernel(NlArgs A, const double *__restrict__ Tb, double w2, double pt,
                               double *__restrict__ W, double *__restrict__ F)
{
    const int Nr = A.Nr, Nz = A.Nz;
    const size_t n = (size_t)Nr * Nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int m = A.region[c];
        const double t = Tb[c];
        if (m < 0) {
            W[c] = 1.0;
            F[c] = t;
            continue;
        }
        const int i = (int)(c % Nr);
        const double k = law(A, m, 0, t);
        double lr = 0.0;
        if (i > 0 && A.region[c - 1] >= 0)
            lr += A.gm[i] * face(law(A, A.region[c - 1], 0, Tb[c - 1]), k, 0.5 * A.dr[i - 1], 0.5 * A.dr[i],
                                 A.face_mean) * (Tb[c - 1] - t);
        if (i < Nr - 1 && A.region[c + 1] >= 0)
            lr += A.gp[i] * face(k, law(A, A.region[c + 1], 0, Tb[c + 1]), 0.5 * A.dr[i], 0.5 * A.dr[i + 1],
                                 A.face_mean) * (Tb[c + 1] - t);
        if (i == 0 && A.bc[0] == HEAT_BC_DIRICHLET) lr += 2.0 * A.gm[0] * k * (A.Tbc[0] - t);
        if (i == Nr - 1 && A.bc[1] == HEAT_BC_DIRICHLET) lr += 2.0 * A.gp[Nr - 1] * k * (A.Tbc[1] - t);
        const double w = law(A, m, 2, t) * w2;
        const double xs = A.j2[m] != 0.0 ? law(A, m, 4, t) * A.j2[m] * pt : 0.0;
        W[c] = w;
        F[c] = w * t + lr + xs;
    }
}

// 2^-e for the exponent e of |x| (x != 0), to rescale a 2x2 product.
__device__ __forceinline__ double pow2_inv_scale(double x)
{
    const long long b = __double_as_longlong(x) & 0x7ff0000000000000LL;
    const long long e = b >> 52;  // biased exponent of |x|
    const long long k = 2046 - e; // biased exponent of 2^-(e - 1023)
    return __longlong_as_double((k < 1 ? 1 : (k > 2046 ? 2046 : k)) << 52);
}

// One iteration of eq. "iter_scheme_eq_1" for every r-line: warp = row j.
// Told: the old layer T; E: its explicit z-operator; Ts: T^s; Tn: T^{s+1}.
// Shared memory: five rows of Nr doubles (a, b, c, d, face conductivities).
__global__ void __launch_bounds__(32) nl_rline_kernel(NlArgs A, const double *__restrict__ Told,
                                                       const double *__restrict__ E, const double *__restrict__ Ts,
                                                       double *__restrict__ Tn, double w2, double pt, double eps,
                                                       unsigned long long *slots, int s)
{
    if (converged_before(slots, s, eps)) return;
    extern __shared__ double sm[];
    const int Nr = A.Nr, j = blockIdx.x, lane = threadIdx.x;
    const size_t row = (size_t)j * Nr;
    const signed char *rg = A.region + row;
    double *sa = sm, *sb = sm + Nr, *sc = sm + 2 * Nr, *sd = sm + 3 * Nr, *sf = sm + 4 * Nr;
    // conductivities at the iterate, then the faces i+1/2 (0 next to void)
    for (int i = lane; i < Nr; i += 32) sa[i] = rg[i] >= 0 ? law(A, rg[i], 0, Ts[row + i]) : 0.0;
    __syncwarp();
    for (int i = lane; i < Nr - 1; i += 32)
        sf[i] = (rg[i] >= 0 && rg[i + 1] >= 0) ? face(sa[i], sa[i + 1], 0.5 * A.dr[i], 0.5 * A.dr[i + 1], A.face_mean)
                                               : 0.0;
    __syncwarp();
    // the line system a x_{i-1} + b x_i + c x_{i+1} = d (identity rows on void)
    for (int i = lane; i < Nr; i += 32) {
        const int m = rg[i];
        const double t = Told[row + i];
        double a = 0.0, b = 1.0, c = 0.0, d = t;
        if (m >= 0) {
            const double arm = i > 0 ? A.gm[i] * sf[i - 1] : 0.0;
            const double arp = i < Nr - 1 ? A.gp[i] * sf[i] : 0.0;
            const double drl = (i == 0 && A.bc[0] == HEAT_BC_DIRICHLET) ? 2.0 * A.gm[0] * sa[i] : 0.0;
            const double drh = (i == Nr - 1 && A.bc[1] == HEAT_BC_DIRICHLET) ? 2.0 * A.gp[Nr - 1] * sa[i] : 0.0;
            const double ts = Ts[row + i];
            const double w = law(A, m, 2, ts) * w2;
            const double xs = A.j2[m] != 0.0 ? law(A, m, 4, ts) * A.j2[m] * pt : 0.0;
            a = -arm;
            c = -arp;
            b = w + arm + arp + drl + drh;
            d = w * t + E[row + i] + xs + drl * A.Tbc[0] + drh * A.Tbc[1];
        }
        sa[i] = a, sb[i] = b, sc[i] = c, sd[i] = d;  // each lane rewrites only its own cells
    }
    __syncwarp();
    int K = (Nr + 31) / 32;
    K |= 1;  // odd: lane rows of K doubles fall in distinct bank pairs
    const int i0 = min(lane * K, Nr), i1 = min(i0 + K, Nr);
    // pivots: chunk product P = M_{i1-1} ... M_{i0} of M_i = [[0, c_i], [-a_i, b_i]]
    double p11 = 1.0, p12 = 0.0, p21 = 0.0, p22 = 1.0;
    for (int i = i0; i < i1; ++i) {
        const double a = sa[i], b = sb[i], c = sc[i];
        const double n11 = c * p21, n12 = c * p22;
        const double n21 = fma(b, p21, -a * p11), n22 = fma(b, p22, -a * p12);
        const double sc2 = pow2_inv_scale(fabs(n22) > fabs(n21) ? n22 : n21);
        p11 = n11 * sc2, p12 = n12 * sc2, p21 = n21 * sc2, p22 = n22 * sc2;
    }
    // inclusive scan of the products over the lanes (later chunks on the left)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double q11 = __shfl_up_sync(0xffffffffu, p11, o), q12 = __shfl_up_sync(0xffffffffu, p12, o);
        const double q21 = __shfl_up_sync(0xffffffffu, p21, o), q22 = __shfl_up_sync(0xffffffffu, p22, o);
        if (lane >= o) {
            const double n11 = fma(p11, q11, p12 * q21), n12 = fma(p11, q12, p12 * q22);
            const double n21 = fma(p21, q11, p22 * q21), n22 = fma(p21, q12, p22 * q22);
            const double sc2 = pow2_inv_scale(fabs(n22) > fabs(n21) ? n22 : n21);
            p11 = n11 * sc2, p12 = n12 * sc2, p21 = n21 * sc2, p22 = n22 * sc2;
        }
    }
    // (p, q) entering the chunk: the previous lane's product applied to (0, 1)
    double pp = __shfl_up_sync(0xffffffffu, p12, 1), qq = __shfl_up_sync(0xffffffffu, p22, 1);
    if (lane == 0) pp = 0.0, qq = 1.0;
    // rewalk: 1/m_i -> sb, c'_i -> sc; forward map of the chunk (G, H): d'_out = G + H d'_in
    double G = 0.0, H = 1.0;
    for (int i = i0; i < i1; ++i) {
        const double a = sa[i], b = sb[i], c = sc[i];
        const double pn = c * qq, qn = fma(b, qq, -a * pp);
        const double r = 1.0 / qn;
        const double inv_m = qq * r;
        sb[i] = inv_m;
        sc[i] = pn * r;
        const double g = sd[i] * inv_m, h = -a * inv_m;
        G = fma(h, G, g);
        H = h * H;
        const double sc2 = pow2_inv_scale(qn);
        pp = pn * sc2, qq = qn * sc2;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double g2 = __shfl_up_sync(0xffffffffu, G, o), h2 = __shfl_up_sync(0xffffffffu, H, o);
        if (lane >= o) G = fma(H, g2, G), H = H * h2;
    }
    double dp = __shfl_up_sync(0xffffffffu, G, 1);
    if (lane == 0) dp = 0.0;
    for (int i = i0; i < i1; ++i) {
        dp = fma(-sa[i] * sb[i], dp, sd[i] * sb[i]);
        sd[i] = dp;
    }
    // backward: x_i = d'_i - c'_i x_{i+1}; chunk map x_{i0} = G + H x_{i1}
    G = 0.0, H = 1.0;
    for (int i = i1 - 1; i >= i0; --i) {
        G = fma(-sc[i], G, sd[i]);
        H = -sc[i] * H;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double g2 = __shfl_down_sync(0xffffffffu, G, o), h2 = __shfl_down_sync(0xffffffffu, H, o);
        if (lane + o < 32) G = fma(H, g2, G), H = H * h2;
    }
    double x = __shfl_down_sync(0xffffffffu, G, 1);
    if (lane == 31) x = 0.0;
    for (int i = i1 - 1; i >= i0; --i) {
        x = fma(-sc[i], x, sd[i]);
        sa[i] = x;
    }
    __syncwarp();
    double diff = 0.0;
    for (int i = lane; i < Nr; i += 32) {
        const double v = sa[i];
        Tn[row + i] = v;
        diff = fmax(diff, fabs(v - Ts[row + i]));
    }
    fold_max(slots + s, diff);
}

// One iteration of eq. "iter_scheme_eq_2" for every z-line: thread = column i.
// W, F: the fixed mass term and right-hand side; Ts: T^s; Tn: T^{s+1}.
__global__ void __launch_bounds__(32) nl_zline_kernel(NlArgs A, const double *__restrict__ W,
                                                       const double *__restrict__ F, const double *__restrict__ Ts,
                                                       double *__restrict__ Tn, double *__restrict__ cw,
                                                       double *__restrict__ dw, double eps, unsigned long long *slots,
                                                       int s)
{
    if (converged_before(slots, s, eps)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int Nr = A.Nr, Nz = A.Nz;
    double diff = 0.0;
    if (i < Nr) {
        double cprev = 0.0, dprev = 0.0;
        double k_cur = A.region[i] >= 0 ? law(A, A.region[i], 0, Ts[i]) : 0.0, fl = 0.0;
        for (int j = 0; j < Nz; ++j) {
            const size_t c0 = (size_t)j * Nr + i;
            const int m = A.region[c0];
            const bool up = j + 1 < Nz && A.region[c0 + Nr] >= 0;
            const double k_next = up ? law(A, A.region[c0 + Nr], 0, Ts[c0 + Nr]) : 0.0;
            double a = 0.0, b = 1.0, c = 0.0, d = F[c0];
            double fr = 0.0;
            if (m >= 0) {
                const double azm = A.zm[j] * fl;
                if (up) fr = face(k_cur, k_next, 0.5 * A.dz[j], 0.5 * A.dz[j + 1], A.face_mean);
                const double azp = A.zp[j] * fr;
                const double dzl = (j == 0 && A.bc[2] == HEAT_BC_DIRICHLET) ? 2.0 * A.zm[0] * k_cur : 0.0;
                const double dzh = (j == Nz - 1 && A.bc[3] == HEAT_BC_DIRICHLET) ? 2.0 * A.zp[Nz - 1] * k_cur : 0.0;
                a = -azm;
                c = -azp;
                b = W[c0] + azm + azp + dzl + dzh;
                d += dzl * A.Tbc[2] + dzh * A.Tbc[3];
            }
            const double r = 1.0 / (b - a * cprev);
            cprev = c * r;
            dprev = (d - a * dprev) * r;
            cw[c0] = cprev;
            dw[c0] = dprev;
            fl = fr;
            k_cur = k_next;
        }
        double x = dprev;
        const size_t last = (size_t)(Nz - 1) * Nr + i;
        Tn[last] = x;
        diff = fabs(x - Ts[last]);
        for (int j = Nz - 2; j >= 0; --j) {
            const size_t c0 = (size_t)j * Nr + i;
            x = dw[c0] - cw[c0] * x;
            Tn[c0] = x;
            diff = fmax(diff, fabs(x - Ts[c0]));
        }
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

}  // namespace

struct heat_nl {
    cudaStream_t stream = nullptr;
    int device = -1;
    Grid g;
    NlArgs A{};
    heat_pulse pulse{};
    heat_nl_options opt{};
    double t = 0.0;
    // device buffers
    double *d_T = nullptr, *d_Tbar = nullptr, *d_it[2] = {nullptr, nullptr}, *d_cw = nullptr, *d_dw = nullptr;
    double *d_fix = nullptr;  // half-step 1: the explicit z-operator; half-step 2: the right-hand side F
    double *d_Wz = nullptr;   // half-step 2: the mass term W
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
    for (void *p : {(void *)s->d_T, (void *)s->d_Tbar, (void *)s->d_it[0], (void *)s->d_it[1], (void *)s->d_cw,
                    (void *)s->d_dw, (void *)s->d_fix, (void *)s->d_Wz, (void *)s->d_slots})
        if (p) cudaFree(p);
    for (void *p : s->owned) cudaFree(p);
    if (s->h_slots) cudaFreeHost(s->h_slots);
    delete s;
}

constexpr int kBatch = 3;  // iterations launched between two reads of the slots
constexpr int kNlMaxNr = HEAT_NL_MAX_NR;  // an r-line's five rows of doubles fit one block's shared memory

constexpr int kFixBlocks = 4 * 152;  // grid of the per-cell kernels (a few waves of the 152 SMs)

// One half-step's iteration (dir 0: eq. "iter_scheme_eq_1" from T; dir 1:
// eq. "iter_scheme_eq_2" from Tbar).  Returns the number of iterations used
// (the result is then in d_it[(used - 1) % 2]), 0 if s_max were not enough,
// or a negative status.
int run_half(heat_nl *s, int dir, double tau, double pt)
{
    const int s_max = s->opt.s_max;
    const double *Tfix = dir == 0 ? s->d_T : s->d_Tbar;
    const double w2 = 2.0 / tau;
    cudaError_t e = cudaMemsetAsync(s->d_slots, 0, sizeof(unsigned long long) * s_max, s->stream);
    if (e != cudaSuccess) return cuda_st(e);
    if (dir == 0)
        nl_zexp_kernel<<<kFixBlocks, 256, 0, s->stream>>>(s->A, Tfix, s->d_fix);
    else
        nl_rexp_kernel<<<kFixBlocks, 256, 0, s->stream>>>(s->A, Tfix, w2, pt, s->d_Wz, s->d_fix);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_st(e);
    ++s->launches;
    const size_t smem = 5 * (size_t)s->g.Nr * sizeof(double);
    for (int s0 = 0; s0 < s_max; s0 += kBatch) {
        const int nb = std::min(kBatch, s_max - s0);
        for (int b = 0; b < nb; ++b) {
            const int it = s0 + b;
            const double *Ts = it == 0 ? Tfix : s->d_it[(it - 1) % 2];
            double *Tn = s->d_it[it % 2];
            if (dir == 0)
                nl_rline_kernel<<<s->g.Nz, 32, smem, s->stream>>>(s->A, Tfix, s->d_fix, Ts, Tn, w2, pt, s->opt.eps,
                                                                  s->d_slots, it);
            else
                nl_zline_kernel<<<(s->g.Nr + 31) / 32, 32, 0, s->stream>>>(s->A, s->d_Wz, s->d_fix, Ts, Tn, s->d_cw,
                                                                           s->d_dw, s->opt.eps, s->d_slots, it);
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
    std::swap(s->d_T, s->d_it[(u - 1) % 2]);
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
    if (R < 1 || K < 1 || K > 1024 || !mat->T_knots || !mat->k || !mat->C || !mat->chi || !mat->j2) return HEAT_ERR_ARG;
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

    heat_nl *s = new (std::nothrow) heat_nl();
    if (!s) return HEAT_ERR_OOM;
    s->stream = static_cast<cudaStream_t>(stream);
    s->pulse = *pulse;
    s->opt = *opt;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_st(e);
    }
    build_grid(geom, s->g);
    const Grid &g = s->g;
    const int Nr = g.Nr, Nz = g.Nz;
    const size_t ncell = (size_t)Nr * Nz;
    auto fail = [&](int x) {
        free_nl(s);
        return x;
    };
    // region of each cell: the first box whose closed rectangle holds its centre
    std::vector<signed char> reg(ncell);
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nr; ++i) {
            int r = -1;
            for (int b = 0; b < geom->n_boxes && r < 0; ++b) {
                const heat_box &bx = geom->boxes[b];
                if (g.rc[i] >= bx.r0 && g.rc[i] <= bx.r1 && g.zc[j] >= bx.z0 && g.zc[j] <= bx.z1) r = bx.region;
            }
            reg[(size_t)j * Nr + i] = (signed char)r;
        }
    if (R > 127 || Nr > kNlMaxNr) return fail(HEAT_ERR_ARG);
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
    NlArgs &A = s->A;
    A.Nr = Nr, A.Nz = Nz, A.K = K, A.face_mean = opt->face_mean;
    for (int f = 0; f < 4; ++f) A.bc[f] = geom->bc[f], A.Tbc[f] = geom->T_bc[f];
    // the couplings' geometric factors: r_{i-1/2} / (r_i hbar_i h_i), r_{i+1/2} / (r_i hbar_i h_{i+1}),
    // 1 / (etabar_j eta_j), 1 / (etabar_j eta_{j+1})
    std::vector<double> gm(Nr), gp(Nr), zm(Nz), zp(Nz);
    for (int i = 0; i < Nr; ++i) {
        gm[i] = g.rf[i] / (g.rc[i] * g.hbar[i] * g.h[i]);
        gp[i] = g.rf[i + 1] / (g.rc[i] * g.hbar[i] * g.h[i + 1]);
    }
    for (int j = 0; j < Nz; ++j) {
        zm[j] = 1.0 / (g.etabar[j] * g.eta[j]);
        zp[j] = 1.0 / (g.etabar[j] * g.eta[j + 1]);
    }
    if ((st = upload(s, reg, &A.region)) != HEAT_OK || (st = upload(s, g.dr, &A.dr)) != HEAT_OK ||
        (st = upload(s, g.dz, &A.dz)) != HEAT_OK || (st = upload(s, gm, &A.gm)) != HEAT_OK ||
        (st = upload(s, gp, &A.gp)) != HEAT_OK || (st = upload(s, zm, &A.zm)) != HEAT_OK ||
        (st = upload(s, zp, &A.zp)) != HEAT_OK || (st = upload(s, tk, &A.Tk)) != HEAT_OK ||
        (st = upload(s, tab, &A.tab)) != HEAT_OK || (st = upload(s, j2, &A.j2)) != HEAT_OK)
        return fail(st);
    const size_t smem = 5 * (size_t)Nr * sizeof(double);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(nl_rline_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return fail(cuda_st(e));
    double **bufs[8] = {&s->d_T, &s->d_Tbar, &s->d_it[0], &s->d_it[1], &s->d_cw, &s->d_dw, &s->d_fix, &s->d_Wz};
    for (double **b : bufs)
        if ((e = cudaMalloc(b, ncell * sizeof(double))) != cudaSuccess) return fail(cuda_st(e));
    if ((e = cudaMalloc(&s->d_slots, opt->s_max * sizeof(unsigned long long))) != cudaSuccess) return fail(cuda_st(e));
    if ((e = cudaMallocHost(&s->h_slots, opt->s_max * sizeof(unsigned long long))) != cudaSuccess)
        return fail(cuda_st(e));
    nl_fill_kernel<<<256, 256, 0, s->stream>>>(s->d_T, ncell, mat->T_init);
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

static int nl_copy(heat_nl *s, double *dst, const double *src, size_t n, int on_device, cudaMemcpyKind dev_kind,
                   cudaMemcpyKind host_kind)
{
    const size_t ncell = (size_t)s->g.Nr * s->g.Nz;
    if (n != ncell) return HEAT_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(dst, src, ncell * sizeof(double), on_device ? dev_kind : host_kind, s->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
    return cuda_st(e);
}

int heat_nl_field(heat_nl *s, double *out, size_t n, int on_device)
{
    if (!s || !out) return HEAT_ERR_ARG;
    return nl_copy(s, out, s->d_T, n, on_device, cudaMemcpyDeviceToDevice, cudaMemcpyDeviceToHost);
}

int heat_nl_half_field(heat_nl *s, double *out, size_t n, int on_device)
{
    if (!s || !out) return HEAT_ERR_ARG;
    return nl_copy(s, out, s->d_Tbar, n, on_device, cudaMemcpyDeviceToDevice, cudaMemcpyDeviceToHost);
}

int heat_nl_set_field(heat_nl *s, const double *in, size_t n, int on_device)
{
    if (!s || !in) return HEAT_ERR_ARG;
    return nl_copy(s, s->d_T, in, n, on_device, cudaMemcpyDeviceToDevice, cudaMemcpyHostToDevice);
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
