// heat_setup.cpp -- host-side construction of the grid, the line classes and
// the FP64 per-class coefficient/factorization tables (done once per
// heat_create, the tables again per heat_set_dt).
//
// Grid (Sec. 3, eq. "grid"): cell-centred, uniform inside each layer.
// Spacings (Sec. 3, after eq. "Lambda_z"): h_i = r_i - r_{i-1},
// hbar_i = (h_i + h_{i+1})/2, r_{i+-1/2} = (r_i + r_{i+-1})/2, same in z.
// Outer faces use a mirror ghost cell: h_0 = 2 (r_0 - r_lo), r_{-1/2} = r_lo.
// Operators (eqs. "Lambda_r", "Lambda_z"):
//   Lambda_r[T]_i = (1/(r_i hbar_i)) [ r_{i+1/2} k_{i+1/2} (T_{i+1}-T_i)/h_{i+1}
//                                    - r_{i-1/2} k_{i-1/2} (T_i-T_{i-1})/h_i ]
//   Lambda_z[T]_j = (1/etabar_j) [ k_{j+1/2} (T_{j+1}-T_j)/eta_{j+1} - k_{j-1/2} (T_j-T_{j-1})/eta_j ]
// Dirichlet face: ghost value 2 T_bc - T, coefficient D = 2 r_face k / (r_i hbar_i h_ghost).
#include <algorithm>
#include <cmath>
#include <limits>
#include <map>

#include "heat_internal.h"

namespace heat {

void HostTab::resize(int nc, int n)
{
    n_class = nc;
    N = n;
    size_t sz = (size_t)nc * n;
    for (auto *v : {&inv, &f, &cp, &w, &s, &am, &ap, &ad, &sd, &dl, &dh, &q, &xm, &xp, &m, &b, &p, &cap, &dsum, &dbc, &ssum})
        v->assign(sz, 0.0);
}

int validate(const heat_geometry *g, const heat_materials *mt, const heat_options *o, double dt)
{
    if (!g || !mt || !o) return HEAT_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HEAT_ERR_ARG;
    if (o->precision < HEAT_FP64 || o->precision > HEAT_FP32_REFINED) return HEAT_ERR_ARG;
    if (o->face_mean != HEAT_HARMONIC && o->face_mean != HEAT_ARITH) return HEAT_ERR_ARG;
    if (g->n_r_layers < 1 || g->n_z_layers < 1 || !g->r_faces || !g->r_cells || !g->z_faces || !g->z_cells)
        return HEAT_ERR_ARG;
    if (g->n_boxes < 1 || g->n_boxes > 32 || !g->boxes) return HEAT_ERR_ARG;
    if (!(g->r_faces[0] >= 0.0)) return HEAT_ERR_ARG;
    long long Nr = 0, Nz = 0;
    for (int l = 0; l < g->n_r_layers; ++l) {
        if (!(g->r_faces[l + 1] > g->r_faces[l]) || g->r_cells[l] < 1) return HEAT_ERR_ARG;
        Nr += g->r_cells[l];
    }
    for (int l = 0; l < g->n_z_layers; ++l) {
        if (!(g->z_faces[l + 1] > g->z_faces[l]) || g->z_cells[l] < 1) return HEAT_ERR_ARG;
        Nz += g->z_cells[l];
    }
    // r-lines are solved by one block of <= 1024 threads x <= 32 cells; a
    // z chunk of <= 128 rows x 128 columns fits one block's shared memory
    if (Nr > 32768 || Nz > 32768 || Nr * Nz > (1LL << 34)) return HEAT_ERR_ARG;
    for (int f = 0; f < 4; ++f)
        if ((g->bc[f] != HEAT_BC_NEUMANN && g->bc[f] != HEAT_BC_DIRICHLET) || !std::isfinite(g->T_bc[f]))
            return HEAT_ERR_ARG;
    if (mt->n_regions < 1 || !mt->k || !mt->C || !mt->q || !std::isfinite(mt->T_init)) return HEAT_ERR_ARG;
    for (int r = 0; r < mt->n_regions; ++r)
        if (!(mt->k[r] > 0.0) || !(mt->C[r] > 0.0) || !std::isfinite(mt->k[r]) || !std::isfinite(mt->C[r]) ||
            !std::isfinite(mt->q[r]))
            return HEAT_ERR_ARG;
    for (int b = 0; b < g->n_boxes; ++b) {
        const heat_box &bx = g->boxes[b];
        if (bx.region < 0 || bx.region >= mt->n_regions) return HEAT_ERR_ARG;
        if (!(bx.r1 >= bx.r0) || !(bx.z1 >= bx.z0)) return HEAT_ERR_ARG;
    }
    return HEAT_OK;
}

// Centres and widths of a layered axis.
static void layered_axis(int nl, const double *faces, const int *cells, std::vector<double> &c,
                         std::vector<double> &w)
{
    c.clear();
    w.clear();
    for (int l = 0; l < nl; ++l) {
        const double dx = (faces[l + 1] - faces[l]) / (double)cells[l];
        for (int m = 0; m < cells[l]; ++m) {
            c.push_back(faces[l] + ((double)m + 0.5) * dx);
            w.push_back(dx);
        }
    }
}

void build_grid(const heat_geometry *geo, Grid &g)
{
    layered_axis(geo->n_r_layers, geo->r_faces, geo->r_cells, g.rc, g.dr);
    layered_axis(geo->n_z_layers, geo->z_faces, geo->z_cells, g.zc, g.dz);
    g.Nr = (int)g.rc.size();
    g.Nz = (int)g.zc.size();
    g.r_lo = geo->r_faces[0];
    g.r_hi = geo->r_faces[geo->n_r_layers];
    g.z_lo = geo->z_faces[0];
    g.z_hi = geo->z_faces[geo->n_z_layers];
    const int Nr = g.Nr, Nz = g.Nz;

    // spacing between centres with a mirror ghost beyond each outer face
    g.h.assign(Nr + 1, 0.0);
    g.h[0] = 2.0 * (g.rc[0] - g.r_lo);
    g.h[Nr] = 2.0 * (g.r_hi - g.rc[Nr - 1]);
    for (int i = 1; i < Nr; ++i) g.h[i] = g.rc[i] - g.rc[i - 1];
    g.hbar.resize(Nr);
    for (int i = 0; i < Nr; ++i) g.hbar[i] = 0.5 * (g.h[i] + g.h[i + 1]);
    g.rf.assign(Nr + 1, 0.0);  // r at face i-1/2
    g.rf[0] = g.r_lo;
    g.rf[Nr] = g.r_hi;
    for (int i = 1; i < Nr; ++i) g.rf[i] = 0.5 * (g.rc[i - 1] + g.rc[i]);

    g.eta.assign(Nz + 1, 0.0);
    g.eta[0] = 2.0 * (g.zc[0] - g.z_lo);
    g.eta[Nz] = 2.0 * (g.z_hi - g.zc[Nz - 1]);
    for (int j = 1; j < Nz; ++j) g.eta[j] = g.zc[j] - g.zc[j - 1];
    g.etabar.resize(Nz);
    for (int j = 0; j < Nz; ++j) g.etabar[j] = 0.5 * (g.eta[j] + g.eta[j + 1]);

    // box membership masks per axis
    g.maskR.assign(Nr, 0u);
    g.maskZ.assign(Nz, 0u);
    for (int b = 0; b < geo->n_boxes; ++b) {
        const heat_box &bx = geo->boxes[b];
        for (int i = 0; i < Nr; ++i)
            if (g.rc[i] >= bx.r0 && g.rc[i] <= bx.r1) g.maskR[i] |= (1u << b);
        for (int j = 0; j < Nz; ++j)
            if (g.zc[j] >= bx.z0 && g.zc[j] <= bx.z1) g.maskZ[j] |= (1u << b);
    }
    // classes: distinct masks in order of first appearance
    auto classify = [](const std::vector<uint32_t> &mask, std::vector<int> &cls, std::vector<uint32_t> &cmask) {
        std::map<uint32_t, int> id;
        cls.resize(mask.size());
        cmask.clear();
        for (size_t x = 0; x < mask.size(); ++x) {
            auto it = id.find(mask[x]);
            if (it == id.end()) {
                it = id.emplace(mask[x], (int)cmask.size()).first;
                cmask.push_back(mask[x]);
            }
            cls[x] = it->second;
        }
    };
    classify(g.maskZ, g.rowcls, g.rowmask);
    classify(g.maskR, g.colcls, g.colmask);
}

// Region of the first box in a mask, -1 if none.
static inline int first_region(uint32_t mask, const std::vector<int> &box_region)
{
    if (!mask) return -1;
    int b = __builtin_ctz(mask);
    return box_region[b];
}

static inline double face_k(double ka, double kb, double da, double db, int mean)
{
    if (mean == HEAT_ARITH) return 0.5 * (ka + kb);
    return (da + db) / (da / ka + db / kb);  // series resistance of the two half cells
}

// Fill table entries of one class from its region vector.
//   metric_c[i] : metric at the centre (r_i for r; 1 for z)
//   metric_f[i] : metric at face i-1/2 (N+1 entries; r_{i-1/2} for r; 1 for z)
//   sp[i]       : centre spacing (N+1 entries, ghosts at ends); bar[i]: hbar or etabar
//   wd[i]       : cell widths
static void fill_class(HostTab &T, int cls, const std::vector<int> &reg, const std::vector<double> &metric_c,
                       const std::vector<double> &metric_f, const std::vector<double> &sp,
                       const std::vector<double> &bar, const std::vector<double> &wd, int bc_lo, int bc_hi,
                       double th_lo, double th_hi, const heat_ctx *ctx, double tau)
{
    const int N = T.N;
    const size_t o = (size_t)cls * N;
    for (int x = 0; x < N; ++x) {
        const int r = reg[x];
        const bool act = r >= 0;
        double m = 0, p = 0, Dl = 0, Dh = 0;
        if (act) {
            const double lam = ctx->k[r];
            const double denom = metric_c[x] * bar[x];
            if (x > 0 && reg[x - 1] >= 0)
                m = metric_f[x] * face_k(ctx->k[reg[x - 1]], lam, 0.5 * wd[x - 1], 0.5 * wd[x], ctx->face_mean) /
                    (denom * sp[x]);
            if (x < N - 1 && reg[x + 1] >= 0)
                p = metric_f[x + 1] * face_k(lam, ctx->k[reg[x + 1]], 0.5 * wd[x], 0.5 * wd[x + 1], ctx->face_mean) /
                    (denom * sp[x + 1]);
            if (x == 0 && bc_lo == HEAT_BC_DIRICHLET) Dl = 2.0 * metric_f[0] * lam / (denom * sp[0]);
            if (x == N - 1 && bc_hi == HEAT_BC_DIRICHLET) Dh = 2.0 * metric_f[N] * lam / (denom * sp[N]);
        }
        const double w = act ? 2.0 * ctx->C[r] / tau : 1.0;
        T.m[o + x] = m;
        T.p[o + x] = p;
        T.w[o + x] = w;
        T.b[o + x] = act ? w + m + p + Dl + Dh : 1.0;
        T.s[o + x] = act ? ctx->q[r] + Dl * th_lo + Dh * th_hi : 0.0;
        T.am[o + x] = m;
        T.ap[o + x] = p;
        T.ad[o + x] = -(m + p + Dl + Dh);
        T.sd[o + x] = Dl * th_lo + Dh * th_hi;
        T.dl[o + x] = Dl;
        T.dh[o + x] = Dh;
        T.xm[o + x] = x == 0 ? Dl : m;
        T.xp[o + x] = x == N - 1 ? Dh : p;
        T.q[o + x] = act ? ctx->q[r] : 0.0;
        T.cap[o + x] = act ? ctx->C[r] : 0.0;
        T.dsum[o + x] = Dl + Dh;
        T.dbc[o + x] = Dl * th_lo + Dh * th_hi;
        T.ssum[o + x] = m + p + Dl + Dh;
    }
    // Thomas factorization (forward elimination of the fixed matrix)
    double cprev = 0.0;
    for (int x = 0; x < N; ++x) {
        const double den = T.b[o + x] - T.m[o + x] * cprev;
        T.inv[o + x] = 1.0 / den;
        T.f[o + x] = T.m[o + x] / den;
        T.cp[o + x] = T.p[o + x] / den;
        cprev = T.cp[o + x];
    }
}

void build_tables(heat_ctx *ctx)
{
    const Grid &g = ctx->g;
    const int Nr = g.Nr, Nz = g.Nz;
    const double tau = ctx->tau;
    std::vector<double> ones_c(std::max(Nr, Nz) + 1, 1.0);

    ctx->R.resize((int)g.rowmask.size(), Nr);
    std::vector<int> reg(Nr);
    for (int a = 0; a < (int)g.rowmask.size(); ++a) {
        for (int i = 0; i < Nr; ++i) reg[i] = first_region(g.maskR[i] & g.rowmask[a], ctx->box_region);
        fill_class(ctx->R, a, reg, g.rc, g.rf, g.h, g.hbar, g.dr, ctx->bc[0], ctx->bc[1], ctx->theta_bc[0],
                   ctx->theta_bc[1], ctx, tau);
    }
    ctx->Z.resize((int)g.colmask.size(), Nz);
    reg.assign(Nz, -1);
    for (int b = 0; b < (int)g.colmask.size(); ++b) {
        for (int j = 0; j < Nz; ++j) reg[j] = first_region(g.colmask[b] & g.maskZ[j], ctx->box_region);
        fill_class(ctx->Z, b, reg, ones_c, ones_c, g.eta, g.etabar, g.dz, ctx->bc[2], ctx->bc[3], ctx->theta_bc[2],
                   ctx->theta_bc[3], ctx, tau);
    }
}

// Packed z-sweep tables, chunk and run constants for the column partition
// (see ZPart in heat_internal.h); FP64 on the host.
static void segment_weights(const HostTab &Z, size_t o, int r0, int r1, double *wB, double *wG, double *Cout,
                            double *F, double *H, double *GP, double *Pout = nullptr)
{
    const int n = r1 - r0;
    std::vector<double> C(n + 1), P(n), S(n + 1);
    C[0] = 1.0;
    for (int k = 0; k < n; ++k) C[k + 1] = C[k] * Z.cp[o + r0 + k];
    double pp = 1.0;
    for (int k = 0; k < n; ++k) {
        pp *= Z.f[o + r0 + k];
        P[k] = pp;
    }
    double tail = 1.0;
    for (int k = n - 1; k >= 0; --k) {
        wB[k] = Z.inv[o + r0 + k] * tail;
        tail *= Z.f[o + r0 + k];
    }
    S[n] = 0.0;
    for (int k = n - 1; k >= 0; --k) {
        const double fn = k + 1 < n ? Z.f[o + r0 + k + 1] : 0.0;
        S[k] = C[k] + fn * S[k + 1];
        if (wG) wG[k] = Z.inv[o + r0 + k] * S[k];
    }
    double gp = 0.0;
    for (int k = 0; k < n; ++k) gp += P[k] * C[k];
    if (Cout)
        for (int k = 0; k < n; ++k) Cout[k] = C[k];
    if (Pout)
        for (int k = 0; k < n; ++k) Pout[k] = P[k];
    *F = P[n - 1];
    *H = C[n];
    if (GP) *GP = gp;
}

void build_zpartition(heat_ctx *ctx)
{
    const HostTab &Z = ctx->Z;
    const int Nz = Z.N, nb = Z.n_class;
    const int Rc = z_chunk_rows(ctx->precision, ctx->g.Nr, Nz, !ctx->batch_member);
    const int nch = (Nz + Rc - 1) / Rc;
    ctx->zp.Rc = Rc;
    ctx->zp.n_chunks = nch;
    ctx->zpk.assign((size_t)nb * Nz * 8, 0.0);
    ctx->zch.assign((size_t)nb * nch * 4, 0.0);
    const bool lit = ctx->precision == HEAT_FP64;
    // the refined path of a batch member (the non-lean passes) weights its
    // summary rows by wB; the literal and increment paths, and the lean
    // passes of a single refined context, take B from the zero-carry
    // recurrence itself and need the prefix products P_j = prod f from the
    // chunk's first row instead
    const bool prefix = ctx->precision != HEAT_FP32_REFINED || !ctx->batch_member;
    std::vector<double> wB(Rc), wG(Rc), Pp(Rc);
    for (int b = 0; b < nb; ++b) {
        const size_t o = (size_t)b * Nz;
        for (int c = 0; c < nch; ++c) {
            const int r0 = c * Rc, r1 = std::min(Nz, r0 + Rc);
            double *ch = &ctx->zch[((size_t)b * nch + c) * 4];
            segment_weights(Z, o, r0, r1, wB.data(), wG.data(), nullptr, &ch[0], &ch[1], &ch[2], Pp.data());
            for (int k = 0; k < r1 - r0; ++k) {
                double *e = &ctx->zpk[(o + r0 + k) * 8];
                e[6] = prefix ? Pp[k] : wB[k];
                e[7] = wG[k];
            }
        }
        for (int j = 0; j < Nz; ++j) {
            double *e = &ctx->zpk[(o + j) * 8];
            e[0] = Z.inv[o + j];
            e[1] = Z.f[o + j];
            e[2] = Z.cp[o + j];
            e[3] = lit ? Z.s[o + j] : Z.q[o + j];
            e[4] = lit ? Z.w[o + j] : Z.xm[o + j];
            e[5] = lit ? 0.0 : Z.xp[o + j];
        }
    }
}

// tau_exp, E_ref and Q.  A cell (i,j) with row class a and column class b
// has region first_region(rowmask[a] & colmask[b]) and coupling sum
// R.ssum[a][i] + Z.ssum[b][j], so each class pair is reduced separately.
void compute_limits(heat_ctx *ctx)
{
    const Grid &g = ctx->g;
    const int na = (int)g.rowmask.size(), nb = (int)g.colmask.size();
    std::vector<double> sum_rh(nb, 0.0), sum_eb(na, 0.0);
    for (int i = 0; i < g.Nr; ++i) sum_rh[g.colcls[i]] += g.rc[i] * g.hbar[i];
    for (int j = 0; j < g.Nz; ++j) sum_eb[g.rowcls[j]] += g.etabar[j];
    double tmin = std::numeric_limits<double>::infinity(), e = 0.0, qs = 0.0;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
            const int r = first_region(g.rowmask[a] & g.colmask[b], ctx->box_region);
            if (r < 0) continue;
            double mr = 0.0, mz = 0.0;
            bool any_i = false, any_j = false;
            for (int i = 0; i < g.Nr; ++i)
                if (g.colcls[i] == b) {
                    mr = std::max(mr, ctx->R.ssum[(size_t)a * g.Nr + i]);
                    any_i = true;
                }
            for (int j = 0; j < g.Nz; ++j)
                if (g.rowcls[j] == a) {
                    mz = std::max(mz, ctx->Z.ssum[(size_t)b * g.Nz + j]);
                    any_j = true;
                }
            if (!any_i || !any_j) continue;
            if (mr + mz > 0.0) tmin = std::min(tmin, ctx->C[r] / (mr + mz));
            e += ctx->C[r] * sum_rh[b] * sum_eb[a];
            qs += ctx->q[r] * sum_rh[b] * sum_eb[a];
        }
    ctx->tau_exp = tmin;
    ctx->E_ref = 2.0 * kPi * ctx->T_ref * e;
    ctx->Q = 2.0 * kPi * qs;
}

}  // namespace heat

namespace heat {

// Tables of the line-team r-sweep (see RLine in heat_internal.h) for chunks of
// K cells, from the FP64 factorization of every row class.  Returns false when
// a team's shared-memory buffer (Npad reals) would exceed max_buf_bytes, in
// which case the block-line r-sweep is used instead.
bool build_rline(const heat_ctx *ctx, int K, size_t max_buf_bytes, int &LW, int &nseg, std::vector<double> &tA,
                 std::vector<double> &tB, std::vector<double> &tD, std::vector<double> &tC, std::vector<int> &zcl)
{
    const HostTab &R = ctx->R;
    const int Nr = R.N, ncls = R.n_class;
    const bool lit = ctx->precision == HEAT_FP64;
    const size_t word = lit ? sizeof(double) : sizeof(float);
    const int nch_line = (Nr + K - 1) / K;
    LW = 4;
    while (LW < 32 && LW < nch_line) LW <<= 1;
    nseg = (nch_line + LW - 1) / LW;
    const int nchunk = nseg * LW, Npad = nchunk * K;
    if ((size_t)Npad * word > max_buf_bytes) return false;
    tA.assign((size_t)ncls * Npad * 4, 0.0);
    tB.assign((size_t)ncls * Npad * 2, 0.0);
    tD.assign((size_t)ncls * Npad * 2, 0.0);
    tC.assign((size_t)ncls * nchunk * 12, 0.0);
    std::vector<double> F(nchunk), H(nchunk);
    for (int a = 0; a < ncls; ++a) {
        const size_t o = (size_t)a * Nr;
        double *A = &tA[(size_t)a * Npad * 4], *B = &tB[(size_t)a * Npad * 2], *D = &tD[(size_t)a * Npad * 2];
        for (int c = 0; c < nchunk; ++c) {
            double inv[64], f[64], cp[64];
            for (int k = 0; k < K; ++k) {
                const int i = c * K + k;
                const bool in = i < Nr;
                inv[k] = in ? R.inv[o + i] : 0.0;
                f[k] = in ? R.f[o + i] : 0.0;
                cp[k] = in ? R.cp[o + i] : 0.0;
                if (in) {
                    double *e = &A[(size_t)i * 4];
                    e[0] = lit ? R.w[o + i] : R.xm[o + i];
                    e[1] = lit ? R.s[o + i] : R.xp[o + i];
                    e[2] = lit ? 0.0 : R.q[o + i];
                    e[3] = inv[k];
                }
            }
            double tail = 1.0;
            for (int k = K - 1; k >= 0; --k) {
                const int i = c * K + k;
                B[(size_t)i * 2] = f[k];
                B[(size_t)i * 2 + 1] = inv[k] * tail;
                tail *= f[k];
            }
            double head = 1.0;
            for (int k = 0; k < K; ++k) {
                const int i = c * K + k;
                D[(size_t)i * 2] = cp[k];
                D[(size_t)i * 2 + 1] = head;
                head *= cp[k];
            }
            F[c] = tail;
            H[c] = head;
        }
        double *C = &tC[(size_t)a * nchunk * 12];
        for (int c = 0; c < nchunk; ++c) {
            const int t = c % LW, c0 = c - t;
            double *e = &C[(size_t)c * 12];
            for (int l = 0; l < 5; ++l) {
                const int span = 1 << l;
                double m = 0.0, n = 0.0;
                if (t >= span) {
                    m = 1.0;
                    for (int u = c - span + 1; u <= c; ++u) m *= F[u];
                }
                if (t + span < LW) {
                    n = 1.0;
                    for (int u = c; u < c + span; ++u) n *= H[u];
                }
                e[l] = m;
                e[6 + l] = n;
            }
            double fe = 1.0, he = 1.0;
            for (int u = c0; u < c; ++u) fe *= F[u];
            for (int u = c + 1; u < c0 + LW; ++u) he *= H[u];
            e[5] = fe;
            e[11] = he;
        }
    }
    zcl.assign(nchunk, 0);
    const Grid &g = ctx->g;
    for (int c = 0; c < nchunk; ++c) {
        int cls = -2;
        for (int k = 0; k < K; ++k) {
            const int i = c * K + k;
            if (i >= Nr) break;
            if (cls == -2) cls = g.colcls[i];
            else if (g.colcls[i] != cls) cls = -1;
        }
        zcl[c] = cls == -2 ? 0 : cls;
    }
    return true;
}

std::vector<int> z_tiles(const std::vector<int> &colcls, int Nr, int V)
{
    const int COLS = 32 * V;
    const int plain = (Nr + COLS - 1) / COLS;
    bool straddle = false;
    for (int g = 0; g < plain && !straddle; ++g)
        for (int i = g * COLS + 1; i < std::min(Nr, (g + 1) * COLS); ++i)
            if (colcls[i] != colcls[i - 1]) {
                straddle = true;
                break;
            }
    std::vector<int> t;
    if (!straddle) return t;
    for (int s0 = 0; s0 < Nr;) {
        int s1 = s0 + 1;
        while (s1 < Nr && colcls[s1] == colcls[s0]) ++s1;
        for (int wb = s0 / V * V; wb < s1; wb += COLS) {
            t.push_back(wb);
            t.push_back(std::max(s0, wb));
            t.push_back(std::min(s1, wb + COLS));
            t.push_back(0);
        }
        s0 = s1;
    }
    if ((int)t.size() / 4 > plain + std::max(1, plain / 8)) t.clear();
    return t;
}

}  // namespace heat
