// heat_internal.h -- data structures shared by the host setup, the C ABI and
// the CUDA kernels of libheat.so.
//
// Line classes.  The region map of a layered cell is a function of two masks:
// the set of boxes whose r-range contains the radial centre r_i (maskR[i]) and
// the set whose z-range contains the axial centre z_j (maskZ[j]).  Every row j
// with the same maskZ therefore has the same region vector over i, hence the
// same tridiagonal r-line matrix (Sec. 3, eq. "scheme_eq_1"); every column
// with the same maskR has the same z-line matrix (eq. "scheme_eq_2").  The
// library builds one coefficient table per row class (length Nr) and one per
// column class (length Nz) instead of per-cell coefficient arrays, so the
// sweeps read O(Nr + Nz) table entries, not O(Nr Nz), and the Thomas
// factorization (pivots) of each class is computed once per dt.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "heat.h"

namespace heat {

constexpr double kPi = 3.14159265358979323846;

#ifdef __CUDACC__
// Programmatic dependent launch: the sweep kernels are launched so that a
// kernel may start while its predecessor in the stream finishes.  Each
// kernel lets its successor be scheduled at once (launch_dependents) and,
// before it touches anything a predecessor writes (the fields, the z-pass
// scratch), waits until the predecessor grid has completed and its writes are
// visible (wait).  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
#endif

// One direction's per-class tables, structure of arrays, [n_class][N].
//   inv, f, cp : factorization of the implicit line matrix
//                -m_i x_{i-1} + b_i x_i - p_i x_{i+1} = d_i  (m, p >= 0):
//                den_0 = b_0, den_i = b_i - m_i cp_{i-1}, inv = 1/den,
//                f = m/den, cp = p/den, so the Thomas recurrences are
//                d'_i = d_i inv_i + f_i d'_{i-1},  x_i = d'_i + cp_i x_{i+1}.
//   w, s       : right-hand side of this direction's implicit half-step in
//                the literal form: mass term 2C/tau (1 on void) and the
//                source q + D_face theta_bc of this direction's Dirichlet faces.
//   am, ap, ad, sd : this direction's operator applied explicitly by the
//                other half-step:  am x_{-} + ap x_{+} + ad x + sd
//                (ad = -(m + p + D), sd = D theta_bc).
//   dl, dh, q  : Dirichlet coefficient of the low / high outer face (0 off the
//                face) and the volumetric source (0 on void), used by the
//                increment form.
//   xm, xp     : the couplings of the increment form with each outer
//                Dirichlet face folded in: at the first cell xm = D_lo (the
//                ghost neighbour then holds theta_bc), at the last cell
//                xp = D_hi; elsewhere xm = am, xp = ap.
//   m, b, p    : the matrix itself (FP64 only; residuals of the refined path).
//   cap, dsum, dbc : FP64 energy/flux weights: C (0 on void), sum of the
//                Dirichlet coefficients D of this direction and D theta_bc.
template <typename real>
struct LineTab {
    const real *inv, *f, *cp, *w, *s, *am, *ap, *ad, *sd, *dl, *dh, *q, *xm, *xp;
};

struct LineTab64 {
    const double *m, *b, *p, *w, *s, *am, *ap, *ad, *sd, *dl, *dh, *q;
    const double *cap, *dsum, *dbc;
};

// The FP64 tables the refined path's residual reads, each value v as the
// pair (hi, lo) of FP32 numbers with hi = fl32(v), lo = fl32(v - hi): v to
// about 2^-48 relative (see Pair in heat_kernels.cuh).
struct LineTab2 {
    const float2 *am, *ap, *dl, *dh, *q, *b, *m, *p;
};

// Tables of the line-team r-sweep (heat_rline.cuh) for chunks of K cells,
// teams of LW lanes and nseg segments of LW*K cells per line (Npad = nseg LW K
// cells, the padding cells having all-zero entries).  Per row class:
//   tA [Npad][4]  increment form {xm, xp, q, inv}, literal form {w, s, 0, inv}
//   tB [Npad][2]  {f, wB}: wB_k = inv_k prod_{m=k+1}^{e} f_m (e = chunk end)
//   tD [Npad][2]  {cp, wC}: wC_k = prod_{m=c0}^{k-1} cp_m (c0 = chunk start)
//   tC [Npad/K][12] per chunk c (lane t = c mod LW of its segment):
//        m_l = prod of F over chunks c-2^l+1..c (0 if t < 2^l), l = 0..4,
//        Fe  = prod of F over the segment's chunks before c,
//        n_l = prod of H over chunks c..c+2^l-1 (0 if t + 2^l >= LW),
//        He  = prod of H over the segment's chunks after c,
//      with F, H the products of f, cp over a chunk.
// zcl [Npad/K]: column class shared by every cell of chunk c, or -1.
// Cells per lane chunk of the line-team r-sweep: 8 (FP32), 4 (FP64).
template <typename real>
constexpr int rline_K() { return sizeof(real) == 4 ? 8 : 4; }
// Largest per-team shared-memory buffer (one line's forward results).
constexpr size_t kRLineMaxBuf = 16 * 1024;

template <typename real>
struct RLine {
    const real *tA, *tB, *tD, *tC;
    const int *zcl, *unit;  // unit [n_units]: j0 | (rows << 16), runs of up to kRLineR
                            // consecutive rows of one row class, in order
    int LW, nseg, n_units;
};
// Rows a line team solves together (one unit).
constexpr int kRLineR = 2;
// rows a team of the line-team r-sweep solves together: 2 in FP32; 1 in FP64,
// where the per-team buffer of forward results (8 bytes a cell) would
// otherwise hold the SM to 6 resident warps of an FP64-bound kernel
constexpr int rline_rows(bool fp64) { return fp64 ? 1 : kRLineR; }

// theta_bc of the faces r_lo, r_hi, z_lo, z_hi
struct BcVals {
    double th[4];
};

constexpr int kMaxRun = 16;  // row-class runs kept in the sweep arguments

// Everything a sweep kernel needs about one problem instance.  Kernels take
// a device array of these and pick their instance from a grid index, so one
// launch serves one problem or a whole batch.  The field ping-pongs between
// f0 and f1: with flip = 0 a sweep reads f0 and writes f1, with flip = 1 the
// reverse.
template <typename real>
struct SweepArgs {
    int Nr, Nz;
    int G, band;              // r-sweep: threads per line, rows per line slot
    int Rc, nch;              // z partition
    const int *rowcls, *colcls;
    LineTab<real> R, Z;
    LineTab64 R64, Z64;
    LineTab2 R2, Z2;          // refined path: the residual's coefficients as FP32 pairs
    RLine<real> rl;           // line-team r-sweep tables (tA == nullptr: not built)
    BcVals bc;
    const real *pkA, *pkB, *chk;
    const int *ucls;
    const int4 *ztile;        // z-sweep column tiles {wb, lo, hi, 0} (n_ztile of them; 0: warps of 32 V columns)
    int n_ztile;
    // batch work list of the lean z passes, the same in every instance's
    // arguments: {instance | chunk << 16, wb, lo, hi} per warp (n_zitem of
    // them; 0: grid (column warps, chunks, instances))
    const int4 *zitem;
    int n_zitem;
    int zrc_max;              // with a work list: the most chunk rows of any instance (the
                              // stride of a warp's shared-memory slice: a block mixes instances)
    real *zs, *zc, *rho;
    real *f0, *f1;
    // walk r-sweep (FP32 increment form, heat_rwalk.cuh): per row class the
    // coefficients {f, cp, q inv, inv} of cell l K + k at [class][k][lane],
    // the column class of each cell at [k][lane], the number of column classes
    const float4 *rw_tab;
    const signed char *rw_cc;
    int rw_K, rw_ncc;
    int rw_stall;             // failure-detection test: the walk's first wait runs out
    int *status;              // device status word: bit 0 = a bounded wait gave up
    // row-class runs of the instance: run r is rows [run_lo[r], run_lo[r+1])
    // of one row class (n_run = 0: more than kMaxRun runs).  The register-
    // resident r-sweep of a single instance splits each run into bands of
    // `band` rows, run r owning slots [run_slot[r], run_slot[r+1]); rb_runs = 0:
    // uniform bands of the whole height
    int n_run, rb_runs;
    int run_lo[kMaxRun + 1], run_slot[kMaxRun + 1], run_cls[kMaxRun];
};

// One kernel launch of a sweep.  Every sweep kernel takes a device array of
// SweepArgs, and all but the carry pass also the flip flag.
struct Launch {
    const void *fn = nullptr;
    dim3 grid, block;
    size_t smem = 0;
    bool flip = false;
    int cluster = 1;  // blocks per thread-block cluster along x (1: no cluster)
    bool pdl = true;  // launched with programmatic stream serialization
    // kernels with a third parameter, the first instance's arguments by value
    // (__grid_constant__: read from the constant bank, so a band's first
    // loads do not wait for a fetch of the arguments).  A plan builder marks
    // such a launch with a non-empty pargs; plan_mode then stores in it the
    // bytes of the first instance's final arguments, which run_plan passes
    std::vector<unsigned char> pargs;
};

// Launch schedule of both half-steps for one set of instances (one problem,
// or a batch sharing precision), with the tunables it was built from.
struct Tuning {
    int rK = 0;    // r-sweep: 1 = line-team kernel; 4, 8, 16, 32 = block-line kernel with rK
                   // cells per thread; 0 = default rule (line teams where every instance has tables)
    int band = 0;  // r-sweep consecutive rows per line slot; 0 = default rule
    int zwpb = 0;  // z-solve warps per block (1 or 2); 0 = default rule
};
struct SweepPlan {
    std::vector<Launch> dir[2];
    Tuning used;   // the values the plan resolved to
};

// Host FP64 master of one direction's tables.
struct HostTab {
    int n_class = 0, N = 0;
    std::vector<double> inv, f, cp, w, s, am, ap, ad, sd, dl, dh, q, xm, xp, m, b, p, cap, dsum, dbc;
    std::vector<double> ssum;  // sum of all couplings (for tau_exp)
    void resize(int nc, int n);
};

// Device copy of one direction's tables (FP64 always; FP32 copy when needed).
struct DevTab {
    double *buf64 = nullptr;  // 20 fields x n_class x N doubles
    float *buf32 = nullptr;   // 14 fields x n_class x N floats
    float2 *buf2 = nullptr;   // refined path: 8 fields x n_class x N FP32 pairs
    LineTab<double> t64{};
    LineTab<float> t32{};
    LineTab64 full{};
    LineTab2 t2{};
};

// Column partition of the z-sweep.  Every column is cut into chunks of Rc
// rows (the last one may be shorter).  For a chunk [r0, r1) of a column class
// with factorization (inv, f, cp) and right-hand side r:
//   forward summary   B = d'_{r1-1} with zero carry-in   = sum_j r_j wB_j,
//                     wB_j = inv_j prod_{m=j+1}^{r1-1} f_m
//   backward summary  G0 = x_{r0} with zero carries       = sum_j r_j wG_j,
//                     wG_j = inv_j S_j,  S_j = C_j + f_{j+1} S_{j+1},
//                     C_k = prod_{m=r0}^{k-1} cp_m
//   chunk constants   F = prod_{m=r0}^{r1-1} f_m,  H = prod_{m=r0}^{r1-1} cp_m,
//                     GP = sum_k P_k C_k,  P_k = prod_{m=r0}^{k} f_m
// and the exact carries follow from D_c = B_c + F_c D_{c-1} (D_{-1} = 0) and
// X_c = G0_c + GP_c D_{c-1} + H_c X_{c+1} (X_n = 0): chunk c starts its
// forward recurrence from D_{c-1} and its backward one from X_{c+1}.
// Packed per (class, row) tables, 8 values: pkA = {inv, f, cp, e0},
// pkB = {e1, e2, s6, wG} with (e0, e1, e2) = (q, xm, xp) for the increment
// form, (s, w, 0) for the literal form, and s6 = wB on the refined path or
// P_j = prod_{m=r0}^{j} f_m (the chunk's prefix product) on the literal and
// increment paths.  Per (class, chunk): {F, H, GP, 0}.
struct ZPart {
    int Rc = 0, n_chunks = 0;
    double *pk64 = nullptr, *ch64 = nullptr;  // device
    float *pk32 = nullptr, *ch32 = nullptr;   // device (FP32 paths)
    int *ucls = nullptr;                      // device: row class of chunk c if all its rows share it, else -1
    int4 *tiles = nullptr;                    // device: column tiles of the lean z passes (see z_tiles)
    int n_tiles = 0;
};

// Column tiles of the lean z passes, one warp each: the columns [lo, hi) of
// one column class, the warp's lanes holding V-column row segments from the
// V-aligned column wb <= lo (lanes may read columns outside [lo, hi), they
// store only inside).  A warp then never straddles a layer interface, where
// it would read its tables per column.  Returned only where some warp of
// 32 V columns from column 0 would straddle one and the tiles cost at most an
// eighth more warps; else empty.  Used for single instances (a batch plan
// drops them).
std::vector<int> z_tiles(const std::vector<int> &colcls, int Nr, int V);

// Rows per z chunk (one warp walks a chunk of its columns): 32, or more
// (a multiple of 4) so that a column has at most 256 chunks.  A single
// instance whose z-sweep would then have fewer than two warps per SM (a small
// grid: every warp walks its chunk alone on an SM, and in FP64 the SM's two
// FP64 FMAs per clock bound it) takes chunks of 16 or 8 rows instead, as long
// as a column stays within 256 chunks; batch members keep 32 (the batch's
// work list spreads their warps already).
inline int z_chunk_rows(int precision, int Nr, int Nz, bool spread)
{
    if (Nz <= 32) return Nz;
    int rc = (Nz + 255) / 256;
    rc = (rc + 3) / 4 * 4;
    rc = rc < 32 ? 32 : rc;
    if (spread && rc == 32) {
        const int cols = precision == HEAT_FP64 ? 64 : 128;  // columns per warp (one 16-byte segment per lane)
        const long long col_warps = (Nr + cols - 1) / cols;
        while (rc > 8 && col_warps * ((Nz + rc - 1) / rc) < 2 * 152 && (Nz + rc / 2 - 1) / (rc / 2) <= 256) rc /= 2;
    }
    return rc;
}
// Columns per thread of the z-sweep (one 8- or 16-byte row segment).
inline int z_cols_per_thread(int) { return 2; }

struct Grid {
    int Nr = 0, Nz = 0;
    double r_lo = 0, r_hi = 0, z_lo = 0, z_hi = 0;
    std::vector<double> rc, dr, h, hbar, rf;  // radial: centres, widths, h[0..Nr], hbar, r_{i-1/2}[0..Nr]
    std::vector<double> zc, dz, eta, etabar;  // axial
    std::vector<uint32_t> maskR, maskZ;       // boxes containing each centre, per axis
    std::vector<int> rowcls, colcls;          // class of each row j / column i
    std::vector<uint32_t> rowmask, colmask;   // maskZ of each row class / maskR of each column class
};

}  // namespace heat

struct heat_ctx {
    int precision = HEAT_FP64;
    int face_mean = HEAT_HARMONIC;
    cudaStream_t stream = nullptr;
    int device = -1;               // the device current at heat_create (owns every buffer)
    heat::Grid g;
    // problem constants
    double T_ref = 0.0;        // field stored as theta = T - T_ref
    double theta_bc[4] = {0, 0, 0, 0};
    int bc[4] = {0, 0, 0, 0};
    std::vector<int> box_region;
    std::vector<double> k, C, q;
    double tau = 0.0, tau_exp = 0.0;
    double E_ref = 0.0, Q = 0.0;  // 2 pi sum C T_ref r hbar etabar; source power
    heat::HostTab R, Z;
    std::vector<double> zpk, zch;  // host z-partition tables (see ZPart): 8 per (class,row)
    heat::ZPart zp;
    float *d_zsum = nullptr;       // z-sweep chunk summaries then carries (scratch), FP32 paths
    double *d_zsum64 = nullptr;    // z-sweep chunk summaries then carries (scratch), FP64 path
    float *d_rho = nullptr;        // refined path: FP32 residual field (scratch)
    // line-team r-sweep tables (see RLine), in the field precision
    void *d_rl = nullptr;
    int *d_rlz = nullptr;
    int rl_LW = 0, rl_nseg = 0, rl_nunits = 0, rl_nchunk = 0;
    // device
    heat::DevTab dR, dZ;
    int *d_rowcls = nullptr, *d_colcls = nullptr;
    double *d_wr = nullptr, *d_wz = nullptr;  // energy weights 2 pi r_i hbar_i, etabar_j
    void *d_field[2] = {nullptr, nullptr};
    int cur = 0;                  // index of the buffer holding the current field
    int half = 0;                 // 1 after heat_sweep(ctx, 0): the current field is Tbar
    double *d_part = nullptr;     // per-block energy partials (scratch)
    double *d_res = nullptr;      // [E_theta, Phi]
    double *d_tmp64 = nullptr;    // Nr*Nz doubles for host/device transfers of FP32 fields
    int n_part = 0;
    int deferred = HEAT_OK;
    // launch plan of one sweep direction and its device argument block
    heat::SweepPlan plan;
    std::vector<unsigned char> h_args;  // one SweepArgs<real>
    void *d_args = nullptr;
    bool batch_member = false;          // owned by a heat_batch (no heat_sweep / heat_destroy)
    // walk r-sweep tables (FP32 increment form; rw_K = 0 when not built)
    void *d_rwtab = nullptr;
    signed char *d_rwcc = nullptr;
    int rw_K = 0, rw_ncc = 0;
    int rw_stall = 0;
    int *d_status = nullptr;            // bit 0: a kernel's bounded wait gave up
    int rsweep_req = 0;                 // requested r-sweep kernel (heat_set_rsweep; 0 = default rule)
    // persistent whole-step kernel of a small FP64 instance (heat_small.cu;
    // small_fn null when the instance does not qualify)
    const void *small_fn = nullptr;
    int small_blocks = 0, small_wpb = 1;
    unsigned *d_small_bar = nullptr;    // grid barrier: the launch's arrival count (and a spare word)
};
