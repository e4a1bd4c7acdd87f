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
} orc_t;

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
