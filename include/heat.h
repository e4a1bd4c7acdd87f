/*
 * heat.h -- C ABI of libheat.so: the per-time-step implicit (ADI) solve of the
 * axisymmetric (r,z) heat equation in a cylinder made of piecewise-constant
 * material regions, on one GB300 GPU (sm_103a).
 *
 * Method (arXiv 1912.03744, "Parallel Algorithm for Numerical Solution of Heat
 * Equation in Complex Cylindrical Domain"):
 *   Sec. 2, eq. "main_eq"     C dT/dt = (1/r) d/dr(r k dT/dr) + d/dz(k dT/dz) + X
 *                             with k, C = rho c_V and X constant per region.
 *   Sec. 2, eq. "boundcond"   dT/dn = 0 on the boundary except T = T0 on the top
 *                             face; no flux through the axis.  Here each outer
 *                             face (r_lo, r_hi, z_lo, z_hi) is Neumann or Dirichlet.
 *   Sec. 3, eq. "grid"        shifted (cell-centred) grid, uniform inside a layer.
 *   Sec. 3, eqs. "Lambda_r", "Lambda_z" and their definitions: the spatial
 *                             operators with the 1/r metric and face conductivities.
 *   Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2": one step = half-step 1 (implicit
 *                             in r, explicit in z) then half-step 2 (explicit in
 *                             r, implicit in z), each of length tau/2.
 *   Sec. 3, last paragraph before Sec. 4: every implicit system is a set of
 *                             independent tridiagonal line systems (Thomas).
 * Readings of silent or garbled points: mirror ghost cells at outer faces
 * (h_0 = 2 (r_0 - r_lo), r_{-1/2} = r_lo, zero at the axis); harmonic face
 * conductivity weighted by cell half widths (HEAT_HARMONIC, default) or the
 * literal arithmetic mean (HEAT_ARITH); Dirichlet flux k (T_bc - T)/(dx/2);
 * void cells (no box) are identity rows with insulated faces.
 *
 * Conventions for every entry point:
 *   - Return value: HEAT_OK (0) or a negative HEAT_ERR_* code; nothing throws
 *     across the ABI.  heat_strerror() names a code.
 *   - Units: SI (m, s, K, W/(m K), J/(m^3 K), W/m^3).
 *   - Field layout: row-major [Nz][Nr] doubles, index j*Nr + i, i the radial
 *     cell (fastest), j the axial cell.
 *   - Ownership: the library allocates and owns every device buffer of a
 *     context; caller buffers are only read or written during the call
 *     (host pointers) or in stream order on the context's stream (device
 *     pointers, on_device = 1).
 *   - Streams: work is enqueued on the stream given to heat_create (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *     heat_step is asynchronous; calls that return host data synchronize.
 */
#ifndef HEAT_H
#define HEAT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HEAT_OK 0
#define HEAT_ERR_ARG (-1)       /* invalid argument (sizes, ordering, dt <= 0, NULL) */
#define HEAT_ERR_CUDA (-2)      /* a CUDA runtime call or kernel launch failed      */
#define HEAT_ERR_NONFINITE (-3) /* the field holds NaN or Inf (found by heat_energy) */
#define HEAT_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up               */
#define HEAT_ERR_OOM (-5)       /* device allocation failed                         */
#define HEAT_ERR_TOO_LARGE (-6) /* size beyond a fixed capacity (heat_energy_noalloc) */
#define HEAT_ERR_NOCONV (-7)    /* the simple iteration did not converge (heat_nl_*) */

/* ---- precision of the stored field and the line solves ---- */
#define HEAT_FP64 0             /* FP64 field, FP64 line solves                     */
#define HEAT_FP32 1             /* FP32 field (offset by T_init), FP32 line solves  */
#define HEAT_FP32_REFINED 2     /* FP32 field and solves + one FP64-residual
                                   correction solve per line (iterative refinement) */

/* ---- face conductivity at a material interface (garbled in Sec. 3) ---- */
#define HEAT_HARMONIC 0
#define HEAT_ARITH 1

/* ---- boundary condition kinds ---- */
#define HEAT_BC_NEUMANN 0
#define HEAT_BC_DIRICHLET 1

typedef struct heat_ctx heat_ctx; /* opaque, library-owned */

/* Axis-aligned region box in (r,z): a cell belongs to the first box whose
 * closed rectangle contains its centre; cells in no box are void. */
typedef struct {
    double r0, r1, z0, z1;
    int region; /* index into heat_materials arrays */
} heat_box;

/* Layered geometry (Sec. 3, eq. "grid"): radial layers [r_faces[l], r_faces[l+1]]
 * of r_cells[l] uniform cells each, axial segments likewise.  r_faces[0] = 0 is
 * the symmetry axis (its face carries no flux whatever bc[0] says).
 * bc[f], T_bc[f]: kind and value on faces f = 0 r_lo, 1 r_hi, 2 z_lo, 3 z_hi. */
typedef struct {
    int n_r_layers;
    const double *r_faces; /* n_r_layers + 1, strictly increasing, >= 0 */
    const int *r_cells;    /* n_r_layers, each >= 1                      */
    int n_z_layers;
    const double *z_faces; /* n_z_layers + 1, strictly increasing        */
    const int *z_cells;    /* n_z_layers, each >= 1                      */
    int n_boxes;           /* 1..32                                       */
    const heat_box *boxes;
    int bc[4];
    double T_bc[4];
} heat_geometry;

/* Per-region constants (the paper's k(T), c_V(T), rho(r), X(T) read as constants). */
typedef struct {
    int n_regions;
    const double *k; /* conductivity > 0                 */
    const double *C; /* volumetric heat capacity > 0     */
    const double *q; /* volumetric source (any sign)     */
    double T_init;   /* uniform initial temperature (eq. "initcond") */
} heat_materials;

typedef struct {
    int precision; /* HEAT_FP64 | HEAT_FP32 | HEAT_FP32_REFINED */
    int face_mean; /* HEAT_HARMONIC | HEAT_ARITH                 */
} heat_options;

/* Build the grid, region map, per-line-class coefficient and factorization
 * tables for time step dt (> 0), allocate device buffers, set T = T_init.
 * stream: cudaStream_t as void* (NULL = legacy default stream).
 * Errors: HEAT_ERR_ARG (bad sizes, ordering, counts, dt <= 0, NULL pointers),
 * HEAT_ERR_OOM, HEAT_ERR_CUDA.  On error *out is NULL. */
int heat_create(const heat_geometry *geom, const heat_materials *mat, const heat_options *opt,
                double dt, void *stream, heat_ctx **out);

/* Change the time step (rebuilds the factorization tables).  dt > 0. */
int heat_set_dt(heat_ctx *ctx, double dt);

/* Enqueue n >= 0 ADI steps (eqs. "scheme_eq_1" then "scheme_eq_2" per step)
 * on the context stream.  Asynchronous; launch errors return HEAT_ERR_CUDA.
 * An FP64 context whose lines are at most 256 cells long in both directions
 * (with the default r-sweep rule) runs all n steps in one cooperative launch
 * whose half steps are separated by a grid barrier with a bounded wait; a
 * wait that runs out is reported by heat_sync as HEAT_ERR_TIMEOUT. */
int heat_step(heat_ctx *ctx, int n);

/* One half-step only: dir = 0 runs half-step 1 (eq. "scheme_eq_1": implicit
 * in r, explicit in z), after which the current field is the half layer
 * Tbar; dir = 1 then runs half-step 2 (eq. "scheme_eq_2") to the next layer.
 * heat_step(ctx, 1) equals heat_sweep(ctx, 0) followed by heat_sweep(ctx, 1).
 * Errors: HEAT_ERR_ARG if dir is not 0/1, if dir = 1 is called without a
 * preceding dir = 0, or if dir = 0 is called twice in a row; heat_step
 * returns HEAT_ERR_ARG while a half-step is pending. */
int heat_sweep(heat_ctx *ctx, int dir);

/* Copy the current temperature field (Nz*Nr doubles, [j][i]) to out; n must
 * equal Nr*Nz.  on_device = 0: out is host memory, the call synchronizes.
 * on_device = 1: out is device memory, the copy is stream-ordered. */
int heat_field(heat_ctx *ctx, double *out, size_t n, int on_device);

/* Replace the field (restart / resume); same layout and rules as heat_field.
 * Void cells keep whatever value is given. */
int heat_set_field(heat_ctx *ctx, const double *in, size_t n, int on_device);

/* FP64 reductions of the current field (synchronizes):
 *   E   = 2 pi sum_active C T r_i hbar_i etabar_j        (J)
 *   Phi = 2 pi sum over Dirichlet faces of r_i hbar_i etabar_j D (T_bc - T)  (W, into Omega)
 *   Q   = 2 pi sum_active q r_i hbar_i etabar_j          (W)
 * With only the top face Dirichlet, one step satisfies
 *   E(next) - E(now) = tau Q + (tau/2) (Phi(now) + Phi(next)).
 * Any pointer may be NULL.  Returns HEAT_ERR_NONFINITE if E or Phi is not finite. */
int heat_energy(heat_ctx *ctx, double *E, double *Phi, double *Q);

/* Same results as heat_energy (to rounding: the partial sums are grouped per
 * grid row instead of per block), but the call allocates no device memory and
 * uses none of the context's scratch: its partial sums live in a fixed
 * file-scope device array of 2 * HEAT_NOALLOC_MAX_ROWS + 2 doubles (128 KB),
 * one per process and device.  The paper has no counterpart; this exists for
 * callers that must not allocate at the point they ask for the heat balance
 * (a monitor under a hard device-memory budget, or one auditing a context
 * whose scratch it cannot assume idle).
 *   ctx: a live context; its device must be current.  Synchronizes ctx's stream
 *        (also when it returns an error after queueing work).
 *   E, Phi, Q: as heat_energy; any may be NULL.
 * Returns HEAT_ERR_TOO_LARGE if Nz > HEAT_NOALLOC_MAX_ROWS, HEAT_ERR_ARG for a
 * NULL ctx or when the current device is not ctx's, HEAT_ERR_CUDA if a CUDA
 * call fails, HEAT_ERR_NONFINITE as heat_energy.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) and must come before any stream capture on that
 * device.  The array keeps the last call's contents; a call rewrites every slot
 * it reads.  Calls through this entry point are serialised by a process-wide
 * lock and each drains its stream before returning, because overlapping calls
 * would race on the one array.  No claim is made for use inside a CUDA graph. */
#define HEAT_NOALLOC_MAX_ROWS 8192
int heat_energy_noalloc(heat_ctx *ctx, double *E, double *Phi, double *Q);

/* Grid and limits.  Any pointer may be NULL; r_centres holds Nr, z_centres Nz
 * doubles.  tau_exp = min over active cells of C / (sum of the cell's
 * couplings), the forward-Euler positivity limit of the assembled operator. */
int heat_info(heat_ctx *ctx, int *Nr, int *Nz, double *r_centres, double *z_centres,
              double *tau_exp);

/* The r-sweep kernel of a single context: kind 0 = the default rule; 1 =
 * line teams (a warp walks each r-line in segments); 2 = register-resident
 * lines (FP32 increment form, lines up to 2048 cells); 3 = walked lines (FP32
 * increment form, rows a multiple of 4 cells up to 2080, staged by bulk copies,
 * one warp per row); 5 = cluster lines (both FP32 precisions, lines up to
 * 16384 cells, a thread-block cluster of ceil(Nr / 2048) blocks per line,
 * the default for FP32 lines longer than 2048 cells and for every refined
 * FP32 context within that length); 4, 8, 16, 32 = block lines with kind
 * cells per thread.
 * HEAT_ERR_ARG (and the schedule unchanged) when the kind is not available
 * for this context.  heat_get_rsweep returns the kind in use.  Synchronizes. */
int heat_set_rsweep(heat_ctx *ctx, int kind);
int heat_get_rsweep(heat_ctx *ctx);

/* Number of kernel launches heat_step(ctx, 1) enqueues (for launch accounting). */
int heat_launches_per_step(heat_ctx *ctx);

/* Wait for the context stream; returns the first deferred error, if any, or
 * HEAT_ERR_TIMEOUT when a kernel's bounded wait gave up since the last call
 * (the kernel then skipped its work; the context stays usable). */
int heat_sync(heat_ctx *ctx);

/* Failure-detection test hook: with on = 1, the walked r-sweep (heat_set_rsweep
 * kind 3, the one that stages rows by bulk copies on mbarriers) first waits,
 * with a 2 ms limit, on a barrier nothing completes, records the time-out and
 * skips the sweep; the persistent step kernel of a small FP64 instance
 * (lines up to 256 cells each way, heat_step with the default r-sweep rule)
 * waits at its first grid barrier for one block more than it has, gives up
 * after 1 s, records the time-out and ends.  heat_sync then returns
 * HEAT_ERR_TIMEOUT.  on = 0 restores normal operation.  No GPU fault is
 * involved.  Synchronizes. */
int heat_test_stall(heat_ctx *ctx, int on);

void heat_destroy(heat_ctx *ctx);

/* ---- batched ensemble ----
 * n independent problems of one precision and face mean, each on its own
 * grid with its own materials and dt, advanced in lockstep (the ensemble of
 * parameter variations the paper's method is run over, Sec. 5).  Each member
 * is an ordinary context; every stage of a step is one kernel launch over all
 * members (member index = a grid dimension), and heat_batch_step replays CUDA
 * graphs of whole steps.  Results per member are those of a single context
 * up to rounding (the batch may cut r-lines into different per-thread chunks).
 * Member limit: Nr <= HEAT_BATCH_MAX_NR (one r-line within one warp). */
typedef struct heat_batch heat_batch;
#define HEAT_BATCH_MAX_NR 1024

/* geoms[n], mats[n], dts[n]: per-member arguments as heat_create; opt shared.
 * stream: the caller's stream (NULL = legacy default stream); heat_batch_step
 * work is ordered after work already queued there, and work queued there
 * afterwards is ordered after the steps.  The batch runs on a stream of its
 * own (graph capture needs one).  1 <= n <= 65535.  Allocates every member's
 * device buffers; HEAT_ERR_ARG on bad sizes, HEAT_ERR_OOM, HEAT_ERR_CUDA. */
int heat_batch_create(int n, const heat_geometry *geoms, const heat_materials *mats,
                      const heat_options *opt, const double *dts, void *stream,
                      heat_batch **out);

/* Change every member's dt (dts[n], each > 0): rebuilds the members' tables
 * and the batch's launch plan and graphs.  Synchronizes. */
int heat_batch_set_dt(heat_batch *b, const double *dts);

/* Borrow member i's context for heat_field, heat_set_field, heat_energy,
 * heat_info (and heat_step of that member alone).  The batch owns it:
 * heat_destroy on it does nothing, heat_sweep and heat_set_dt return
 * HEAT_ERR_ARG.  Its stream is the batch's stream. */
int heat_batch_member(heat_batch *b, int i, heat_ctx **ctx);

/* Enqueue n >= 0 full steps of every member (asynchronous). */
int heat_batch_step(heat_batch *b, int n);

/* Wait for the batch stream. */
int heat_batch_sync(heat_batch *b);

/* Autotuner: time every valid schedule (r-sweep kernel and its cells per
 * thread K, rows per line slot, z-solve warps per block) for trial_steps (1..1000) steps
 * each, on the members' current fields, and keep the fastest.  The members'
 * fields are saved before and restored after, so the state does not change.
 * Allocates one temporary copy of all fields.  best_ms (may be NULL):
 * the winner's device time per step. */
int heat_batch_tune(heat_batch *b, int trial_steps, double *best_ms);

/* Set or read the schedule.  rK selects the r-sweep: 1 = line teams (a team
 * of lanes walks each r-line, 8 cells per lane in FP32, 4 in FP64; FP64 and
 * FP32 only, lines up to 4096 FP32 / 2048 FP64 cells); 2 = register-resident
 * lines (FP32 only, 8 cells per thread, lines up to 2048 cells); 4, 8, 16, 32
 * = one line per thread group with rK cells per thread; 0 = default (2 where
 * every member allows it, else 1, else 8).  band >= 0: rows per line slot (line
 * teams: rows per team when sizing the grid), 0 = default.  zwpb in
 * {0 (default), 1, 2}.  An invalid combination for these members returns
 * HEAT_ERR_ARG and keeps the current schedule. */
int heat_batch_set_tuning(heat_batch *b, int rK, int band, int zwpb);
int heat_batch_get_tuning(heat_batch *b, int *rK, int *band, int *zwpb);

/* Kernel launches one batch step enqueues (independent of n). */
int heat_batch_launches_per_step(heat_batch *b);

void heat_batch_destroy(heat_batch *b);

/* ---- the full method: temperature-dependent materials, the simple
 * iteration, adaptive tau and the pulsed source (FP64) ----
 *   Sec. 2, eq. "main_eq":   k, C = rho c_V and the source depend on T.
 *   Sec. 2, eq. "source":    X = chi(T) j^2 p(t): chi the region's resistivity,
 *                            j its current density (the printed I^2/S_C read as
 *                            (I/S_C)^2, a power per volume).
 *   Sec. 2, eqs. "unit_model", "trans_model": p(t), the rectangular pulse
 *                            train or its erf-smoothed version.
 *   Sec. 3, eqs. "iter_scheme_eq_1", "iter_scheme_eq_2", "iter_cond": each
 *                            half-step iterates T^s -> T^{s+1} until
 *                            max |T^{s+1} - T^s| < eps.  Half-step 1: C, X and
 *                            the r-couplings at T^s, the explicit z-operator at
 *                            the old layer.  Half-step 2: the z-couplings at
 *                            T^s, C, X and the explicit r-operator at Tbar.
 *   Sec. 3 (last paragraph) and Sec. 4: s_max iterations without convergence
 *                            halve tau and restart the step; every step starts
 *                            from the estimate t_trs/1000 inside a transition
 *                            of the source, t_src/100 elsewhere.
 * Readings: material laws are per-region tables at temperature knots, linear
 * between knots and flat beyond the ends (the paper's laws are cited, not
 * printed); face conductivities are the harmonic (or arithmetic) means of the
 * two cells' own conductivities; the source is taken at t + tau/2; theta(0) = 1
 * in u(t); a transition is t mod t_per in [0, t_trs) or [t_src, t_src + t_trs);
 * heat_nl_advance shortens a step outside a transition to end at the next
 * switch (n t_per or n t_per + t_src; a phase within 1e-9 t_per of a switch
 * counts as at it), and its last step to end at t_end.
 * Geometry, boundary conditions, layout ([Nz][Nr] doubles), ownership and
 * stream rules are those of heat_create; the field is FP64 and holds T. */
typedef struct heat_nl heat_nl; /* opaque, library-owned */

typedef struct {
    int n_regions, n_knots;  /* 1 <= n_knots <= 1024                         */
    const double *T_knots;   /* [n_regions][n_knots], increasing per region  */
    const double *k;         /* conductivity at the knots, > 0               */
    const double *C;         /* volumetric heat capacity at the knots, > 0   */
    const double *chi;       /* resistivity at the knots                     */
    const double *j2;        /* [n_regions] squared current density          */
    double T_init;           /* uniform initial temperature                  */
} heat_nl_materials;

#define HEAT_PULSE_CONST 0 /* p = 1                                       */
#define HEAT_PULSE_RECT 1  /* rectangular train u(t), eq. "unit_model"    */
#define HEAT_PULSE_ERF 2   /* smoothed train v(t), eq. "trans_model"      */
typedef struct {
    int model;
    double t_per, t_src, t_trs; /* period, heating time <= t_per, transition time (> 0 unless CONST) */
    double xi, zeta;            /* the smoothing constants of v(t) (the paper: 4 and 2) */
} heat_pulse;

typedef struct {
    double eps;       /* stop of the iteration: max |T^{s+1} - T^s| < eps (K), > 0     */
    int s_max;        /* iterations before tau is halved, 1..4096                      */
    double tau_base;  /* step estimate outside transitions (the paper: t_src/100)     */
    double tau_trs;   /* step estimate inside transitions (the paper: t_trs/1000)     */
    double tau_min;   /* heat_nl_advance gives up below this step                     */
    int face_mean;    /* HEAT_HARMONIC | HEAT_ARITH                                    */
} heat_nl_options;

typedef struct {
    long long steps, halvings, iters1, iters2; /* iterations summed over the steps */
    double tau_smallest;                       /* the shortest step taken          */
} heat_nl_stats;

/* Grid, regions and tables; T = T_init, time 0.  Errors: HEAT_ERR_ARG (bad
 * geometry as heat_create, Nr or Nz > HEAT_NL_MAX_N, no active cell,
 * non-increasing knots, k or C <= 0, bad options), HEAT_ERR_OOM,
 * HEAT_ERR_CUDA.  On error *out is NULL.
 * Layout (Sec. 3, eq. "grid": row j has N_j cells, column i has M_i): the
 * field is stored without void padding, row j up to its last active cell
 * (N_j = that cell's i + 1; void cells before it are kept as identity rows),
 * and a column-packed copy likewise for the z-sweep.  Void cells past the
 * last active cell of their row are not stored: heat_nl_field reports T_init
 * there and heat_nl_set_field ignores them.
 * Limit: a line is assembled and solved in one block's shared memory (five
 * rows of doubles), so Nr, Nz <= HEAT_NL_MAX_N. */
#define HEAT_NL_MAX_N 5632
int heat_nl_create(const heat_geometry *geom, const heat_nl_materials *mat, const heat_pulse *pulse,
                   const heat_nl_options *opt, void *stream, heat_nl **out);

/* One step of length tau from the current time, without halving.  it1, it2
 * (may be NULL): iterations of the two half-steps.  HEAT_ERR_NOCONV if either
 * needed more than s_max (field and time unchanged).  Synchronizes. */
int heat_nl_step(heat_nl *s, double tau, int *it1, int *it2);

/* The evolution loop of Sec. 4 from the current time to t_end (at most
 * max_steps steps; check heat_nl_time for where it stopped).  stats may be
 * NULL.  HEAT_ERR_NOCONV when a step needed tau < tau_min (the field holds the
 * last completed step).  Synchronizes. */
int heat_nl_advance(heat_nl *s, double t_end, long long max_steps, heat_nl_stats *stats);

int heat_nl_time(heat_nl *s, double *t);
int heat_nl_set_time(heat_nl *s, double t);
/* Field I/O as heat_field / heat_set_field; heat_nl_half_field returns the
 * half layer Tbar of the last completed step. */
int heat_nl_field(heat_nl *s, double *out, size_t n, int on_device);
int heat_nl_half_field(heat_nl *s, double *out, size_t n, int on_device);
int heat_nl_set_field(heat_nl *s, const double *in, size_t n, int on_device);
/* Grid size and the number of kernel launches so far. */
int heat_nl_info(heat_nl *s, int *Nr, int *Nz, long long *launches);
/* The packed layout: N_j (Nz ints), M_i (Nr ints) and the stored cell count
 * sum_j N_j (any pointer may be NULL). */
int heat_nl_layout(heat_nl *s, int *N_j, int *M_i, long long *stored);
/* The current field in the row-packed layout: n = sum_j N_j doubles, row j at
 * offset sum_{j' < j} N_j', cells i = 0 .. N_j - 1.  on_device as heat_field. */
int heat_nl_field_packed(heat_nl *s, double *out, size_t n, int on_device);
void heat_nl_destroy(heat_nl *s);

const char *heat_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* HEAT_H */
