/*
 * heat_oracle.c -- plain, slow, FP64 CPU oracle of one Peaceman-Rachford ADI
 * time step for the axisymmetric (r,z) heat equation in a cylinder made of
 * piecewise-constant material regions.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and must never be used as a fallback by it.
 *
 * What it follows (paper: "Parallel Algorithm for Numerical Solution of Heat
 * Equation in Complex Cylindrical Domain"):
 *   - Sec. 2, eq. "main_eq": C dT/dt = (1/r) d/dr(r k dT/dr) + d/dz(k dT/dz) + X,
 *     read with k, C, X piecewise constant per region (temperature independent).
 *   - Sec. 2, eq. "boundcond": insulated walls, T = T0 on the top face, no flux
 *     through the axis r = 0.  Generalised to a Neumann/Dirichlet choice on each
 *     of the four outer faces (used by the closed-form pins).
 *   - Sec. 3, eq. "grid": shifted (cell-centred) grid, uniform inside a layer,
 *     no node on a material interface.
 *   - Sec. 3, eqs. "Lambda_r", "Lambda_z" and the definitions after them:
 *     h_i = r_i - r_{i-1}, hbar_i = (h_i + h_{i+1})/2, r_{i+-1/2} = (r_i + r_{i+-1})/2,
 *     the same in z with eta, etabar.
 *   - Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2": half-step 1 implicit in r and
 *     explicit in z, half-step 2 explicit in r and implicit in z, each tau/2,
 *     the source at the half layer in both.
 *   - Sec. 3 (last paragraph of the iteration part): each implicit system is a
 *     set of independent tridiagonal line systems solved by the Thomas method.
 *
 * Readings where the paper is silent or garbled:
 *   - Boundary spacings: a mirror ghost cell beyond each outer face, so
 *     h_0 = 2 (r_0 - r_lo), h_N = 2 (r_hi - r_{N-1}), r_{-1/2} = r_lo and
 *     r_{N-1/2} = r_hi (zero at the axis), the same in z.
 *   - Face conductivity at a material interface: flux-continuous harmonic mean
 *     weighted by the half widths of the two cells (default), or the literal
 *     arithmetic mean (face_mean = 1).
 *   - Dirichlet face: ghost value 2 T_bc - T, i.e. flux k (T_bc - T) / (dx/2).
 *   - Void cells (no region box covers the centre): identity rows, zero
 *     conductance on every face touching them, excluded from energy and flux.
 *   - Energy E = 2 pi sum C T r_i hbar_i etabar_j, the weights under which the
 *     scheme telescopes; flux Phi = 2 pi sum r_i hbar_i etabar_j D (T_bc - T)
 *     over Dirichlet faces.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp heat_oracle.c -o libheat_oracle.so -lm
 * (OpenMP over independent lines only, as in the paper's Sec. 4.)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int Nr, Nz;
    double r_lo, r_hi, z_lo, z_hi;
    double *rc, *dr, *h, *hbar, *rf;   /* r: centres, widths, h[0..Nr], hbar[Nr], r_{i-1/2}[0..Nr] */
    double *zc, *dz, *eta, *etabar;    /* z: centres, widths, eta[0..Nz], etabar[Nz]            */
    int *region;                       /* [Nz*Nr], -1 = void                                    */
    double *lam, *cap, *src;           /* per cell                                              */
    double *Arm, *Arp, *Azm, *Azp;     /* per cell couplings                                    */
    double *Drl, *Drh, *Dzl, *Dzh;     /* per cell Dirichlet coefficients                       */
    int bc[4];
    double Tbc[4];
    double *T;                         /* field [Nz][Nr] */
    double *Tbar;
    struct orc_nl *nl;                 /* temperature-dependent state (orc_nl_setup), or NULL */
} orc_t;

static void orc_nl_free(struct orc_nl *n);

#define IDX(o, i, j) ((size_t)(j) * (size_t)(o)->Nr + (size_t)(i))

/* ---------------------------------------------------------------- grid */

/* Cell-centred 1D grid over layers: faces[n_l+1], cells[n_l] (eq. "grid"). */
static void build_axis(int n_l, const double *faces, const int *cells, int N,
                       double *c, double *w)
{
    int k = 0;
    for (int l = 0; l < n_l; ++l) {
        double dx = (faces[l + 1] - faces[l]) / cells[l];
        for (int m = 0; m < cells[l]; ++m) {
            c[k] = faces[l] + (m + 0.5) * dx;
            w[k] = dx;
            ++k;
        }
    }
    (void)N;
}

/* Face conductivity between two active cells with half widths da, db. */
static double face_k(double ka, double kb, double da, double db, int face_mean)
{
    if (face_mean == 1)
        return 0.5 * (ka + kb);
    return (da + db) / (da / ka + db / kb);
}

void *orc_create(int n_rl, const double *r_faces, const int *r_cells,
                 int n_zl, const double *z_faces, const int *z_cells,
                 int n_boxes, const double *boxes, const int *box_region,
                 const int *bc, const double *Tbc,
                 int n_regions, const double *k, const double *C, const double *q,
                 int face_mean, double T_init)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    int Nr = 0, Nz = 0;
    for (int l = 0; l < n_rl; ++l) Nr += r_cells[l];
    for (int l = 0; l < n_zl; ++l) Nz += z_cells[l];
    o->Nr = Nr;
    o->Nz = Nz;
    o->r_lo = r_faces[0];
    o->r_hi = r_faces[n_rl];
    o->z_lo = z_faces[0];
    o->z_hi = z_faces[n_zl];
    for (int f = 0; f < 4; ++f) {
        o->bc[f] = bc[f];
        o->Tbc[f] = Tbc[f];
    }
    size_t ncell = (size_t)Nr * Nz;
    o->rc = calloc(Nr, sizeof(double));
    o->dr = calloc(Nr, sizeof(double));
    o->h = calloc(Nr + 1, sizeof(double));
    o->hbar = calloc(Nr, sizeof(double));
    o->rf = calloc(Nr + 1, sizeof(double));
    o->zc = calloc(Nz, sizeof(double));
    o->dz = calloc(Nz, sizeof(double));
    o->eta = calloc(Nz + 1, sizeof(double));
    o->etabar = calloc(Nz, sizeof(double));
    o->region = calloc(ncell, sizeof(int));
    o->lam = calloc(ncell, sizeof(double));
    o->cap = calloc(ncell, sizeof(double));
    o->src = calloc(ncell, sizeof(double));
    o->Arm = calloc(ncell, sizeof(double));
    o->Arp = calloc(ncell, sizeof(double));
    o->Azm = calloc(ncell, sizeof(double));
    o->Azp = calloc(ncell, sizeof(double));
    o->Drl = calloc(ncell, sizeof(double));
    o->Drh = calloc(ncell, sizeof(double));
    o->Dzl = calloc(ncell, sizeof(double));
    o->Dzh = calloc(ncell, sizeof(double));
    o->T = calloc(ncell, sizeof(double));
    o->Tbar = calloc(ncell, sizeof(double));

    build_axis(n_rl, r_faces, r_cells, Nr, o->rc, o->dr);
    build_axis(n_zl, z_faces, z_cells, Nz, o->zc, o->dz);

    /* h_i = r_i - r_{i-1}; mirror ghosts at both ends. */
    o->h[0] = 2.0 * (o->rc[0] - o->r_lo);
    for (int i = 1; i < Nr; ++i) o->h[i] = o->rc[i] - o->rc[i - 1];
    o->h[Nr] = 2.0 * (o->r_hi - o->rc[Nr - 1]);
    for (int i = 0; i < Nr; ++i) o->hbar[i] = 0.5 * (o->h[i] + o->h[i + 1]);
    /* r_{i-1/2} = (r_i + r_{i-1})/2; the ghost gives r_lo and r_hi at the ends. */
    o->rf[0] = o->r_lo;
    for (int i = 1; i < Nr; ++i) o->rf[i] = 0.5 * (o->rc[i] + o->rc[i - 1]);
    o->rf[Nr] = o->r_hi;

    o->eta[0] = 2.0 * (o->zc[0] - o->z_lo);
    for (int j = 1; j < Nz; ++j) o->eta[j] = o->zc[j] - o->zc[j - 1];
    o->eta[Nz] = 2.0 * (o->z_hi - o->zc[Nz - 1]);
    for (int j = 0; j < Nz; ++j) o->etabar[j] = 0.5 * (o->eta[j] + o->eta[j + 1]);

    /* Region of each cell: the first box containing its centre. */
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nr; ++i) {
            int reg = -1;
            for (int b = 0; b < n_boxes; ++b) {
                const double *bx = boxes + 4 * b;
                if (o->rc[i] >= bx[0] && o->rc[i] <= bx[1] &&
                    o->zc[j] >= bx[2] && o->zc[j] <= bx[3]) {
                    reg = box_region[b];
                    break;
                }
            }
            if (reg >= n_regions) reg = -1;
            size_t c = IDX(o, i, j);
            o->region[c] = reg;
            if (reg >= 0) {
                o->lam[c] = k[reg];
                o->cap[c] = C[reg];
                o->src[c] = q[reg];
            }
        }

    /* Couplings of eqs. "Lambda_r" and "Lambda_z" written as
     *   Lambda_r[T]_i = Arp (T_{i+1} - T_i) - Arm (T_i - T_{i-1}) + D (T_bc - T_i). */
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nr; ++i) {
            size_t c = IDX(o, i, j);
            if (o->region[c] < 0) continue;
            double lam = o->lam[c];
            double ri = o->rc[i], hb = o->hbar[i], eb = o->etabar[j];
            if (i > 0 && o->region[IDX(o, i - 1, j)] >= 0) {
                double lf = face_k(o->lam[IDX(o, i - 1, j)], lam, 0.5 * o->dr[i - 1], 0.5 * o->dr[i], face_mean);
                o->Arm[c] = o->rf[i] * lf / (ri * hb * o->h[i]);
            }
            if (i < Nr - 1 && o->region[IDX(o, i + 1, j)] >= 0) {
                double lf = face_k(lam, o->lam[IDX(o, i + 1, j)], 0.5 * o->dr[i], 0.5 * o->dr[i + 1], face_mean);
                o->Arp[c] = o->rf[i + 1] * lf / (ri * hb * o->h[i + 1]);
            }
            if (i == 0 && o->bc[0] == 1)
                o->Drl[c] = 2.0 * o->rf[0] * lam / (ri * hb * o->h[0]);
            if (i == Nr - 1 && o->bc[1] == 1)
                o->Drh[c] = 2.0 * o->rf[Nr] * lam / (ri * hb * o->h[Nr]);
            if (j > 0 && o->region[IDX(o, i, j - 1)] >= 0) {
                double lf = face_k(o->lam[IDX(o, i, j - 1)], lam, 0.5 * o->dz[j - 1], 0.5 * o->dz[j], face_mean);
                o->Azm[c] = lf / (eb * o->eta[j]);
            }
            if (j < Nz - 1 && o->region[IDX(o, i, j + 1)] >= 0) {
                double lf = face_k(lam, o->lam[IDX(o, i, j + 1)], 0.5 * o->dz[j], 0.5 * o->dz[j + 1], face_mean);
                o->Azp[c] = lf / (eb * o->eta[j + 1]);
            }
            if (j == 0 && o->bc[2] == 1)
                o->Dzl[c] = 2.0 * lam / (eb * o->eta[0]);
            if (j == Nz - 1 && o->bc[3] == 1)
                o->Dzh[c] = 2.0 * lam / (eb * o->eta[Nz]);
        }

    for (size_t c = 0; c < ncell; ++c) o->T[c] = T_init;
    return o;
}

void orc_destroy(void *p)
{
    orc_t *o = (orc_t *)p;
    if (!o) return;
    void *bufs[] = {o->rc, o->dr, o->h, o->hbar, o->rf, o->zc, o->dz, o->eta, o->etabar,
                    o->region, o->lam, o->cap, o->src, o->Arm, o->Arp, o->Azm, o->Azp,
                    o->Drl, o->Drh, o->Dzl, o->Dzh, o->T, o->Tbar};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b) free(bufs[b]);
    orc_nl_free(o->nl);
    free(o);
}

void orc_dims(void *p, int *Nr, int *Nz)
{
    orc_t *o = (orc_t *)p;
    *Nr = o->Nr;
    *Nz = o->Nz;
}

/* Grid export: centres, hbar, etabar and region map (for tests and sampling). */
void orc_grid(void *p, double *rc, double *zc, double *hbar, double *etabar, int *region)
{
    orc_t *o = (orc_t *)p;
    memcpy(rc, o->rc, sizeof(double) * o->Nr);
    memcpy(zc, o->zc, sizeof(double) * o->Nz);
    memcpy(hbar, o->hbar, sizeof(double) * o->Nr);
    memcpy(etabar, o->etabar, sizeof(double) * o->Nz);
    memcpy(region, o->region, sizeof(int) * (size_t)o->Nr * o->Nz);
}

/* Coefficient export (per cell, [Nz][Nr]): Arm, Arp, Azm, Azp, Drl, Drh, Dzl, Dzh, C, q. */
void orc_coeffs(void *p, double *out10)
{
    orc_t *o = (orc_t *)p;
    size_t n = (size_t)o->Nr * o->Nz;
    const double *src[10] = {o->Arm, o->Arp, o->Azm, o->Azp, o->Drl, o->Drh, o->Dzl, o->Dzh, o->cap, o->src};
    for (int a = 0; a < 10; ++a) memcpy(out10 + a * n, src[a], sizeof(double) * n);
}

/* Explicit stability limit: min over active cells of C / (sum of couplings). */
double orc_tau_exp(void *p)
{
    orc_t *o = (orc_t *)p;
    double best = INFINITY;
    for (size_t c = 0; c < (size_t)o->Nr * o->Nz; ++c) {
        if (o->region[c] < 0) continue;
        double s = o->Arm[c] + o->Arp[c] + o->Azm[c] + o->Azp[c] + o->Drl[c] + o->Drh[c] + o->Dzl[c] + o->Dzh[c];
        if (s > 0.0 && o->cap[c] / s < best) best = o->cap[c] / s;
    }
    return best;
}

void orc_get_field(void *p, double *out)
{
    orc_t *o = (orc_t *)p;
    memcpy(out, o->T, sizeof(double) * (size_t)o->Nr * o->Nz);
}

void orc_set_field(void *p, const double *in)
{
    orc_t *o = (orc_t *)p;
    memcpy(o->T, in, sizeof(double) * (size_t)o->Nr * o->Nz);
}

/* ------------------------------------------------------------- Thomas */

/* Textbook Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,
 * i = 0..n-1 (a_0 and c_{n-1} unused).  cw, dw are work arrays of length n. */
void orc_thomas(int n, const double *a, const double *b, const double *c, const double *d,
                double *x, double *cw, double *dw)
{
    cw[0] = c[0] / b[0];
    dw[0] = d[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double m = b[i] - a[i] * cw[i - 1];
        cw[i] = c[i] / m;
        dw[i] = (d[i] - a[i] * dw[i - 1]) / m;
    }
    x[n - 1] = dw[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dw[i] - cw[i] * x[i + 1];
}

/* --------------------------------------------------------- one PR step */

/* Lambda_z[T] at (i,j) including Dirichlet z faces. */
static double lambda_z(const orc_t *o, const double *T, int i, int j)
{
    size_t c = IDX(o, i, j);
    double t = T[c], s = 0.0;
    if (o->Azm[c] != 0.0) s += o->Azm[c] * (T[IDX(o, i, j - 1)] - t);
    if (o->Azp[c] != 0.0) s += o->Azp[c] * (T[IDX(o, i, j + 1)] - t);
    s += o->Dzl[c] * (o->Tbc[2] - t) + o->Dzh[c] * (o->Tbc[3] - t);
    return s;
}

/* Lambda_r[T] at (i,j) including Dirichlet r faces. */
static double lambda_r(const orc_t *o, const double *T, int i, int j)
{
    size_t c = IDX(o, i, j);
    double t = T[c], s = 0.0;
    if (o->Arm[c] != 0.0) s += o->Arm[c] * (T[IDX(o, i - 1, j)] - t);
    if (o->Arp[c] != 0.0) s += o->Arp[c] * (T[IDX(o, i + 1, j)] - t);
    s += o->Drl[c] * (o->Tbc[0] - t) + o->Drh[c] * (o->Tbc[1] - t);
    return s;
}

/* One step of eqs. "scheme_eq_1" / "scheme_eq_2" with time step tau.
 * X: optional per-cell source [Nz][Nr] (evaluated at the half layer by the
 * caller); NULL uses the region source q. */
static void pr_step(orc_t *o, double tau, const double *X)
{
    const int Nr = o->Nr, Nz = o->Nz;
    const double half = 0.5 * tau;
    double *T = o->T, *Tb = o->Tbar;

    /* Half-step 1: for every row j, implicit in r, explicit Lambda_z[T]. */
#pragma omp parallel
    {
        double *a = malloc(sizeof(double) * Nr), *b = malloc(sizeof(double) * Nr);
        double *cc = malloc(sizeof(double) * Nr), *d = malloc(sizeof(double) * Nr);
        double *x = malloc(sizeof(double) * Nr), *cw = malloc(sizeof(double) * Nr);
        double *dw = malloc(sizeof(double) * Nr);
#pragma omp for schedule(static)
        for (int j = 0; j < Nz; ++j) {
            for (int i = 0; i < Nr; ++i) {
                size_t c = IDX(o, i, j);
                if (o->region[c] < 0) {
                    a[i] = 0.0; b[i] = 1.0; cc[i] = 0.0; d[i] = T[c];
                    continue;
                }
                double w = o->cap[c] / half;
                double xs = X ? X[c] : o->src[c];
                a[i] = -o->Arm[c];
                cc[i] = -o->Arp[c];
                b[i] = w + o->Arm[c] + o->Arp[c] + o->Drl[c] + o->Drh[c];
                d[i] = w * T[c] + lambda_z(o, T, i, j) + xs + o->Drl[c] * o->Tbc[0] + o->Drh[c] * o->Tbc[1];
            }
            orc_thomas(Nr, a, b, cc, d, x, cw, dw);
            for (int i = 0; i < Nr; ++i) Tb[IDX(o, i, j)] = x[i];
        }
        free(a); free(b); free(cc); free(d); free(x); free(cw); free(dw);
    }

    /* Half-step 2: for every column i, explicit Lambda_r[Tbar], implicit in z. */
#pragma omp parallel
    {
        double *a = malloc(sizeof(double) * Nz), *b = malloc(sizeof(double) * Nz);
        double *cc = malloc(sizeof(double) * Nz), *d = malloc(sizeof(double) * Nz);
        double *x = malloc(sizeof(double) * Nz), *cw = malloc(sizeof(double) * Nz);
        double *dw = malloc(sizeof(double) * Nz);
#pragma omp for schedule(static)
        for (int i = 0; i < Nr; ++i) {
            for (int j = 0; j < Nz; ++j) {
                size_t c = IDX(o, i, j);
                if (o->region[c] < 0) {
                    a[j] = 0.0; b[j] = 1.0; cc[j] = 0.0; d[j] = Tb[c];
                    continue;
                }
                double w = o->cap[c] / half;
                double xs = X ? X[c] : o->src[c];
                a[j] = -o->Azm[c];
                cc[j] = -o->Azp[c];
                b[j] = w + o->Azm[c] + o->Azp[c] + o->Dzl[c] + o->Dzh[c];
                d[j] = w * Tb[c] + lambda_r(o, Tb, i, j) + xs + o->Dzl[c] * o->Tbc[2] + o->Dzh[c] * o->Tbc[3];
            }
            orc_thomas(Nz, a, b, cc, d, x, cw, dw);
            for (int j = 0; j < Nz; ++j) T[IDX(o, i, j)] = x[j];
        }
        free(a); free(b); free(cc); free(d); free(x); free(cw); free(dw);
    }
}

/* n steps with the region sources. */
void orc_step(void *p, double tau, int n)
{
    for (int s = 0; s < n; ++s) pr_step((orc_t *)p, tau, NULL);
}

/* One step with a caller-given per-cell source (manufactured solutions). */
void orc_step_src(void *p, double tau, const double *X)
{
    pr_step((orc_t *)p, tau, X);
}

/* Half-layer field of the last step (for tests of the split). */
void orc_get_half(void *p, double *out)
{
    orc_t *o = (orc_t *)p;
    memcpy(out, o->Tbar, sizeof(double) * (size_t)o->Nr * o->Nz);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ----------------------------------------------------- energy and flux */

/* E = 2 pi sum C T r hbar etabar;  Phi = 2 pi sum r hbar etabar D (T_bc - T);
 * Q = 2 pi sum q r hbar etabar, all over active cells. */
void orc_energy(void *p, double *E, double *Phi, double *Q)
{
    orc_t *o = (orc_t *)p;
    double e = 0.0, f = 0.0, s = 0.0;
    for (int j = 0; j < o->Nz; ++j)
        for (int i = 0; i < o->Nr; ++i) {
            size_t c = IDX(o, i, j);
            if (o->region[c] < 0) continue;
            double wgt = o->rc[i] * o->hbar[i] * o->etabar[j];
            double t = o->T[c];
            e += o->cap[c] * t * wgt;
            f += wgt * (o->Drl[c] * (o->Tbc[0] - t) + o->Drh[c] * (o->Tbc[1] - t) +
                        o->Dzl[c] * (o->Tbc[2] - t) + o->Dzh[c] * (o->Tbc[3] - t));
            s += o->src[c] * wgt;
        }
    *E = 2.0 * ORC_PI * e;
    *Phi = 2.0 * ORC_PI * f;
    *Q = 2.0 * ORC_PI * s;
}

/* ====================================================================
 * Temperature-dependent coefficients, the simple iteration, adaptive tau
 * and the pulsed source: the paper's full evolution loop.
 *
 *   Sec. 2, eq. "main_eq":     k, C = rho c_V and X depend on T.  Material
 *       laws are given per region as tables of values at temperature knots,
 *       read by linear interpolation and held constant beyond the end knots
 *       (the paper's laws are cited, not printed; tests use synthetic ones).
 *   Sec. 2, eq. "source":      X = chi(T) j^2 p(t) with chi the resistivity
 *       of the region and j its current density (I / S_C; zero outside the
 *       heater) -- the printed I^2 / S_C is read as (I / S_C)^2 so that X is
 *       a power per volume.
 *   Sec. 2, eqs. "unit_model", "trans_model": p(t) is the rectangular pulse
 *       train u(t) or its erf-smoothed version v(t); model 0 is p = 1.
 *   Sec. 3, eq. "iter_scheme_eq_1": half-step 1 iterates T^s -> T^{s+1} with
 *       rho c_V, the r-operator's conductivities and X taken at the iterate
 *       T^s, the explicit z-operator at the old layer T, from T^0 = T.
 *   Sec. 3, eq. "iter_scheme_eq_2": half-step 2 iterates with the implicit
 *       z-operator's conductivities at T^s, while rho c_V, X and the explicit
 *       r-operator are taken at the converged half layer Tbar, from T^0 = Tbar.
 *   Sec. 3, eq. "iter_cond":   each iteration stops when
 *       max |T^{s+1} - T^s| < eps; the last iterate is the result.
 *   Sec. 3 (adaptive time step) and Sec. 4: when s reaches s_max without
 *       meeting the criterion, tau is halved and the step restarts from the
 *       old layer; every step starts from the estimate t_trs / 1000 inside a
 *       transition of the source and t_src / 100 elsewhere (passed in as
 *       tau_trs and tau_base).
 * Readings: face conductivities are the face means of the cells' own
 * conductivities at their temperatures (harmonic weighted by the half widths,
 * or arithmetic: the same two readings as the constant case); the source is
 * evaluated at t_k + tau/2 in both half-steps; the last step is shortened to
 * land on t_end; theta(0) = 1 in u(t); a transition is the first t_trs after
 * a switch-on (t mod t_per in [0, t_trs)) or switch-off ([t_src, t_src + t_trs));
 * a step outside a transition is shortened to end at the next switch, so that
 * no step passes over a transition (a phase within 1e-9 t_per of a switch
 * counts as at it, so that rounding of the landing time cannot leave a
 * vanishing step).
 * ==================================================================== */

typedef struct orc_nl {
    int K, n_regions;
    double *Tk, *lam, *cap, *chi; /* [n_regions][K] */
    double *jsq;                  /* [n_regions]    */
    int model;
    double t_per, t_src, t_trs, xi, zeta;
    int face_mean;
    double *Ts, *Tn, *lam_s, *lam_o, *cap_x, *X;  /* per-cell work fields */
} orc_nl_t;

static void orc_nl_free(struct orc_nl *n)
{
    if (!n) return;
    void *bufs[] = {n->Tk, n->lam, n->cap, n->chi, n->jsq, n->Ts, n->Tn, n->lam_s, n->lam_o, n->cap_x, n->X};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b) free(bufs[b]);
    free(n);
}

/* One material table at temperature T: linear between knots, constant beyond. */
static double table_at(const double *Tk, const double *v, int K, double T)
{
    if (K == 1 || T <= Tk[0]) return v[0];
    if (T >= Tk[K - 1]) return v[K - 1];
    int k = 0;
    while (T >= Tk[k + 1]) ++k;
    return v[k] + (v[k + 1] - v[k]) * (T - Tk[k]) / (Tk[k + 1] - Tk[k]);
}

/* p(t) of eq. "unit_model" (model 1) or eq. "trans_model" (model 2); model 0: 1.
 * Terms with n t_per > t + t_per are exactly zero in FP64 for the erf model
 * (both erf arguments are below -6), so the sum stops at floor(t/t_per) + 1. */
double orc_pulse(int model, double t, double t_per, double t_src, double t_trs, double xi, double zeta)
{
    if (model == 0) return 1.0;
    int nmax = (int)floor(t / t_per) + 1;
    if (nmax < 0) nmax = 0;
    double s = 0.0;
    for (int n = 0; n <= nmax; ++n) {
        double a = t - n * t_per, b = t - n * t_per - t_src;
        if (model == 1)
            s += (a >= 0.0 ? 1.0 : 0.0) - (b >= 0.0 ? 1.0 : 0.0);
        else
            s += 0.5 * (erf(xi * (zeta * a / t_trs - 1.0)) - erf(xi * (zeta * b / t_trs - 1.0)));
    }
    return s;
}

/* Attach temperature-dependent materials and the source model to an oracle
 * built by orc_create (its grid, region map and boundary conditions are
 * kept; its constant k, C, q are not used by the functions below). */
void orc_nl_setup(void *p, int n_regions, int K, const double *Tk, const double *lam, const double *cap,
                  const double *chi, const double *jsq, int model, double t_per, double t_src, double t_trs,
                  double xi, double zeta, int face_mean)
{
    orc_t *o = (orc_t *)p;
    size_t ncell = (size_t)o->Nr * o->Nz;
    orc_nl_free(o->nl);
    orc_nl_t *n = o->nl = (orc_nl_t *)calloc(1, sizeof(orc_nl_t));
    n->Ts = calloc(ncell, sizeof(double));
    n->Tn = calloc(ncell, sizeof(double));
    n->lam_s = calloc(ncell, sizeof(double));
    n->lam_o = calloc(ncell, sizeof(double));
    n->cap_x = calloc(ncell, sizeof(double));
    n->X = calloc(ncell, sizeof(double));
    n->n_regions = n_regions;
    n->K = K;
    n->model = model;
    n->t_per = t_per, n->t_src = t_src, n->t_trs = t_trs, n->xi = xi, n->zeta = zeta;
    n->face_mean = face_mean;
    size_t nt = (size_t)n_regions * K;
    n->Tk = malloc(nt * sizeof(double));
    n->lam = malloc(nt * sizeof(double));
    n->cap = malloc(nt * sizeof(double));
    n->chi = malloc(nt * sizeof(double));
    n->jsq = malloc(n_regions * sizeof(double));
    memcpy(n->Tk, Tk, nt * sizeof(double));
    memcpy(n->lam, lam, nt * sizeof(double));
    memcpy(n->cap, cap, nt * sizeof(double));
    memcpy(n->chi, chi, nt * sizeof(double));
    memcpy(n->jsq, jsq, n->n_regions * sizeof(double));
}

/* The per-region laws at one cell. */
static double lam_at(const orc_t *o, const orc_nl_t *n, size_t c, double T)
{
    int m = o->region[c];
    return table_at(n->Tk + (size_t)m * n->K, n->lam + (size_t)m * n->K, n->K, T);
}
static double cap_at(const orc_t *o, const orc_nl_t *n, size_t c, double T)
{
    int m = o->region[c];
    return table_at(n->Tk + (size_t)m * n->K, n->cap + (size_t)m * n->K, n->K, T);
}
static double src_at(const orc_t *o, const orc_nl_t *n, size_t c, double T, double pt)
{
    int m = o->region[c];
    return table_at(n->Tk + (size_t)m * n->K, n->chi + (size_t)m * n->K, n->K, T) * n->jsq[m] * pt;
}

/* Couplings of cell (i,j) (the forms of eqs. "Lambda_r", "Lambda_z", as in
 * orc_create) from a per-cell conductivity field lam:
 * out = {Arm, Arp, Azm, Azp, Drl, Drh, Dzl, Dzh}. */
static void couplings_from(const orc_t *o, const double *lam, int face_mean, int i, int j, double *out)
{
    const int Nr = o->Nr, Nz = o->Nz;
    size_t c = IDX(o, i, j);
    double l = lam[c], ri = o->rc[i], hb = o->hbar[i], eb = o->etabar[j];
    for (int a = 0; a < 8; ++a) out[a] = 0.0;
    if (i > 0 && o->region[IDX(o, i - 1, j)] >= 0)
        out[0] = o->rf[i] * face_k(lam[IDX(o, i - 1, j)], l, 0.5 * o->dr[i - 1], 0.5 * o->dr[i], face_mean) /
                 (ri * hb * o->h[i]);
    if (i < Nr - 1 && o->region[IDX(o, i + 1, j)] >= 0)
        out[1] = o->rf[i + 1] * face_k(l, lam[IDX(o, i + 1, j)], 0.5 * o->dr[i], 0.5 * o->dr[i + 1], face_mean) /
                 (ri * hb * o->h[i + 1]);
    if (j > 0 && o->region[IDX(o, i, j - 1)] >= 0)
        out[2] = face_k(lam[IDX(o, i, j - 1)], l, 0.5 * o->dz[j - 1], 0.5 * o->dz[j], face_mean) / (eb * o->eta[j]);
    if (j < Nz - 1 && o->region[IDX(o, i, j + 1)] >= 0)
        out[3] = face_k(l, lam[IDX(o, i, j + 1)], 0.5 * o->dz[j], 0.5 * o->dz[j + 1], face_mean) / (eb * o->eta[j + 1]);
    if (i == 0 && o->bc[0] == 1) out[4] = 2.0 * o->rf[0] * l / (ri * hb * o->h[0]);
    if (i == Nr - 1 && o->bc[1] == 1) out[5] = 2.0 * o->rf[Nr] * l / (ri * hb * o->h[Nr]);
    if (j == 0 && o->bc[2] == 1) out[6] = 2.0 * l / (eb * o->eta[0]);
    if (j == Nz - 1 && o->bc[3] == 1) out[7] = 2.0 * l / (eb * o->eta[Nz]);
}

static void fill_lam(const orc_t *o, const orc_nl_t *n, const double *T, double *lam)
{
    for (size_t c = 0; c < (size_t)o->Nr * o->Nz; ++c) lam[c] = o->region[c] >= 0 ? lam_at(o, n, c, T[c]) : 0.0;
}

/* max |a - b| over the grid (the C-norm of eq. "iter_cond"). */
static double cnorm_diff(const orc_t *o, const double *a, const double *b)
{
    double m = 0.0;
    for (size_t c = 0; c < (size_t)o->Nr * o->Nz; ++c) {
        double d = fabs(a[c] - b[c]);
        if (d > m) m = d;
    }
    return m;
}

/* Half-step 1 by eq. "iter_scheme_eq_1": from the old layer o->T into
 * o->Tbar.  Xext (optional, per cell) replaces chi(T) j^2 p.  Returns the
 * number of iterations used, or 0 if s_max were not enough. */
static int nl_half1(orc_t *o, orc_nl_t *n, double tau, double pt, double eps, int s_max, const double *Xext)
{
    const int Nr = o->Nr, Nz = o->Nz;
    const size_t ncell = (size_t)Nr * Nz;
    const double half = 0.5 * tau;
    double *T = o->T, *Ts = n->Ts, *Tn = n->Tn;
    memcpy(Ts, T, ncell * sizeof(double));  /* T^0 = T */
    fill_lam(o, n, T, n->lam_o);             /* the explicit z-operator at the old layer */
    int used = 0;
    for (int s = 0; s < s_max; ++s) {
        fill_lam(o, n, Ts, n->lam_s);
#pragma omp parallel
        {
        double *a = malloc(sizeof(double) * Nr), *b = malloc(sizeof(double) * Nr);
        double *cc = malloc(sizeof(double) * Nr), *d = malloc(sizeof(double) * Nr);
        double *x = malloc(sizeof(double) * Nr), *cw = malloc(sizeof(double) * Nr), *dw = malloc(sizeof(double) * Nr);
#pragma omp for schedule(static)
        for (int j = 0; j < Nz; ++j) {
            for (int i = 0; i < Nr; ++i) {
                size_t c = IDX(o, i, j);
                if (o->region[c] < 0) {
                    a[i] = 0.0; b[i] = 1.0; cc[i] = 0.0; d[i] = T[c];
                    continue;
                }
                double ks[8], ko[8];
                couplings_from(o, n->lam_s, n->face_mean, i, j, ks);  /* r-operator at T^s */
                couplings_from(o, n->lam_o, n->face_mean, i, j, ko);  /* z-operator at T   */
                double w = cap_at(o, n, c, Ts[c]) / half;
                double xs = Xext ? Xext[c] : src_at(o, n, c, Ts[c], pt);
                double t = T[c], lz = 0.0;
                if (ko[2] != 0.0) lz += ko[2] * (T[IDX(o, i, j - 1)] - t);
                if (ko[3] != 0.0) lz += ko[3] * (T[IDX(o, i, j + 1)] - t);
                lz += ko[6] * (o->Tbc[2] - t) + ko[7] * (o->Tbc[3] - t);
                a[i] = -ks[0];
                cc[i] = -ks[1];
                b[i] = w + ks[0] + ks[1] + ks[4] + ks[5];
                d[i] = w * t + lz + xs + ks[4] * o->Tbc[0] + ks[5] * o->Tbc[1];
            }
            orc_thomas(Nr, a, b, cc, d, x, cw, dw);
            for (int i = 0; i < Nr; ++i) Tn[IDX(o, i, j)] = x[i];
        }
        free(a); free(b); free(cc); free(d); free(x); free(cw); free(dw);
        }
        double diff = cnorm_diff(o, Tn, Ts);
        memcpy(Ts, Tn, ncell * sizeof(double));
        if (diff < eps) {
            used = s + 1;
            break;
        }
    }
    if (used) memcpy(o->Tbar, Ts, ncell * sizeof(double));
    return used;
}

/* Half-step 2 by eq. "iter_scheme_eq_2": from o->Tbar into n->Tn (left in
 * n->Ts as well).  Returns the iterations used, or 0. */
static int nl_half2(orc_t *o, orc_nl_t *n, double tau, double pt, double eps, int s_max, const double *Xext)
{
    const int Nr = o->Nr, Nz = o->Nz;
    const size_t ncell = (size_t)Nr * Nz;
    const double half = 0.5 * tau;
    double *Tb = o->Tbar, *Ts = n->Ts, *Tn = n->Tn;
    memcpy(Ts, Tb, ncell * sizeof(double));  /* T^0 = Tbar */
    fill_lam(o, n, Tb, n->lam_o);             /* the explicit r-operator at Tbar */
    for (size_t c = 0; c < ncell; ++c) {      /* rho c_V and X at Tbar */
        if (o->region[c] < 0) continue;
        n->cap_x[c] = cap_at(o, n, c, Tb[c]);
        n->X[c] = Xext ? Xext[c] : src_at(o, n, c, Tb[c], pt);
    }
    int used = 0;
    for (int s = 0; s < s_max; ++s) {
        fill_lam(o, n, Ts, n->lam_s);
#pragma omp parallel
        {
        double *a = malloc(sizeof(double) * Nz), *b = malloc(sizeof(double) * Nz);
        double *cc = malloc(sizeof(double) * Nz), *d = malloc(sizeof(double) * Nz);
        double *x = malloc(sizeof(double) * Nz), *cw = malloc(sizeof(double) * Nz), *dw = malloc(sizeof(double) * Nz);
#pragma omp for schedule(static)
        for (int i = 0; i < Nr; ++i) {
            for (int j = 0; j < Nz; ++j) {
                size_t c = IDX(o, i, j);
                if (o->region[c] < 0) {
                    a[j] = 0.0; b[j] = 1.0; cc[j] = 0.0; d[j] = Tb[c];
                    continue;
                }
                double ks[8], ko[8];
                couplings_from(o, n->lam_s, n->face_mean, i, j, ks);  /* z-operator at T^s   */
                couplings_from(o, n->lam_o, n->face_mean, i, j, ko);  /* r-operator at Tbar  */
                double w = n->cap_x[c] / half;
                double t = Tb[c], lr = 0.0;
                if (ko[0] != 0.0) lr += ko[0] * (Tb[IDX(o, i - 1, j)] - t);
                if (ko[1] != 0.0) lr += ko[1] * (Tb[IDX(o, i + 1, j)] - t);
                lr += ko[4] * (o->Tbc[0] - t) + ko[5] * (o->Tbc[1] - t);
                a[j] = -ks[2];
                cc[j] = -ks[3];
                b[j] = w + ks[2] + ks[3] + ks[6] + ks[7];
                d[j] = w * t + lr + n->X[c] + ks[6] * o->Tbc[2] + ks[7] * o->Tbc[3];
            }
            orc_thomas(Nz, a, b, cc, d, x, cw, dw);
            for (int j = 0; j < Nz; ++j) Tn[IDX(o, i, j)] = x[j];
        }
        free(a); free(b); free(cc); free(d); free(x); free(cw); free(dw);
        }
        double diff = cnorm_diff(o, Tn, Ts);
        memcpy(Ts, Tn, ncell * sizeof(double));
        if (diff < eps) {
            used = s + 1;
            break;
        }
    }
    return used;
}

/* One step of length tau from time t (no halving): both iterations; on
 * success the field advances and it1/it2 hold the iterations used.
 * Xext: optional per-cell source replacing chi(T) j^2 p (both half-steps).
 * Returns 1 on success, 0 if either iteration needed more than s_max. */
int orc_nl_step(void *p, double t, double tau, double eps, int s_max, const double *Xext, int *it1, int *it2)
{
    orc_t *o = (orc_t *)p;
    orc_nl_t *n = o->nl;
    if (!n) return 0;
    double pt = orc_pulse(n->model, t + 0.5 * tau, n->t_per, n->t_src, n->t_trs, n->xi, n->zeta);
    *it1 = nl_half1(o, n, tau, pt, eps, s_max, Xext);
    *it2 = 0;
    if (!*it1) return 0;
    *it2 = nl_half2(o, n, tau, pt, eps, s_max, Xext);
    if (!*it2) return 0;
    memcpy(o->T, n->Ts, sizeof(double) * (size_t)o->Nr * o->Nz);
    return 1;
}

/* The evolution loop of Sec. 4 from *t to t_end: each step starts from the
 * estimate (tau_trs inside a transition of the source, tau_base elsewhere),
 * shortened to land on t_end; a step whose iteration does not converge in
 * s_max iterations is restarted with tau / 2 (and so on, down to tau_min).
 * stats (5 doubles): steps, halvings, iterations of half-step 1, of half-step
 * 2, the smallest tau used.  Returns 0, or -1 when tau fell below tau_min
 * (the field then holds the last completed step), or -2 after max_steps. */
int orc_nl_advance(void *p, double *t, double t_end, double tau_base, double tau_trs, double eps, int s_max,
                   double tau_min, int max_steps, double *stats)
{
    orc_nl_t *n = ((orc_t *)p)->nl;
    if (!n) return -3;
    for (int a = 0; a < 5; ++a) stats[a] = 0.0;
    stats[4] = INFINITY;
    while (*t < t_end) {
        if (stats[0] >= max_steps) return -2;
        int trs = 0;
        double to_switch = INFINITY;
        if (n->model != 0) {
            /* phase in the period; within tol of a switch counts as at it */
            double tol = 1e-9 * n->t_per, ph = fmod(*t, n->t_per);
            if (n->t_per - ph < tol) ph = 0.0;
            trs = ph < n->t_trs || (ph >= n->t_src - tol && ph < n->t_src + n->t_trs);
            if (!trs) to_switch = (ph < n->t_src ? n->t_src : n->t_per) - ph;
        }
        double tau = trs ? tau_trs : tau_base;
        if (tau > to_switch) tau = to_switch; /* do not step over a transition */
        int last = tau >= t_end - *t;
        if (last) tau = t_end - *t;
        for (;;) {
            int it1, it2;
            if (orc_nl_step(p, *t, tau, eps, s_max, NULL, &it1, &it2)) {
                stats[2] += it1;
                stats[3] += it2;
                break;
            }
            tau *= 0.5;
            last = 0;
            stats[1] += 1.0;
            if (tau < tau_min) return -1;
        }
        *t = last ? t_end : *t + tau;
        stats[0] += 1.0;
        if (tau < stats[4]) stats[4] = tau;
    }
    return 0;
}
