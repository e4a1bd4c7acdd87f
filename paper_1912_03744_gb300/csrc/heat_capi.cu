// heat_capi.cu -- the extern "C" entry points of libheat.so (declared and
// documented in include/heat.h).  Host-side orchestration only: every cell
// of every step is computed by the kernels in heat_sweeps.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "heat_internal.h"

namespace heat {
int validate(const heat_geometry *, const heat_materials *, const heat_options *, double);
void build_grid(const heat_geometry *, Grid &);
void build_tables(heat_ctx *);
void compute_limits(heat_ctx *);
void build_zpartition(heat_ctx *);
bool build_rline(const heat_ctx *, int, size_t, int &, int &, std::vector<double> &, std::vector<double> &,
                 std::vector<double> &, std::vector<double> &, std::vector<int> &);
cudaError_t launch_fill(heat_ctx *, int, double);
cudaError_t launch_steps(heat_ctx *, int);
cudaError_t small_setup(heat_ctx *);
cudaError_t launch_sweep(heat_ctx *, int);
cudaError_t ctx_plan(heat_ctx *);
cudaError_t launch_energy(heat_ctx *);
cudaError_t launch_theta_to_T(heat_ctx *, double *);
cudaError_t launch_T_to_theta(heat_ctx *, const double *);
int launches_per_step(const heat_ctx *);
int energy_blocks(const heat_ctx *);
int create_ctx(const heat_geometry *, const heat_materials *, const heat_options *, double, void *, bool,
               heat_ctx **);
}  // namespace heat

using namespace heat;

namespace {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return HEAT_OK;
    if (std::getenv("HEAT_DEBUG")) std::fprintf(stderr, "libheat: %s\n", cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return HEAT_ERR_OOM;
    return HEAT_ERR_CUDA;
}

#define HEAT_CHECK(call)                            \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

constexpr int kFields64 = 20;
constexpr int kFields32 = 14;

// Upload one direction's host tables: FP64 master (20 fields) and, for the
// FP32 paths, an FP32 copy of the 14 fields the sweeps use.
int upload_tab(heat_ctx *ctx, const HostTab &T, DevTab &D)
{
    const size_t n = (size_t)T.n_class * T.N;
    if (!D.buf64) HEAT_CHECK(cudaMalloc(&D.buf64, kFields64 * n * sizeof(double)));
    const std::vector<double> *src[kFields64] = {&T.inv, &T.f, &T.cp, &T.w,  &T.s,  &T.am, &T.ap,
                                                 &T.ad,  &T.sd, &T.dl, &T.dh, &T.q,  &T.xm, &T.xp,
                                                 &T.m,   &T.b,  &T.p,  &T.cap, &T.dsum, &T.dbc};
    std::vector<double> host(kFields64 * n);
    for (int a = 0; a < kFields64; ++a) std::memcpy(host.data() + a * n, src[a]->data(), n * sizeof(double));
    HEAT_CHECK(cudaMemcpyAsync(D.buf64, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream));
    double *p = D.buf64;
    auto F = [&](int a) { return (const double *)(p + a * n); };
    D.t64 = LineTab<double>{F(0), F(1), F(2), F(3), F(4), F(5), F(6), F(7), F(8), F(9), F(10), F(11), F(12), F(13)};
    D.full = LineTab64{F(14), F(15), F(16), F(3), F(4), F(5), F(6), F(7), F(8), F(9), F(10), F(11),
                       F(17), F(18), F(19)};
    if (ctx->precision != HEAT_FP64) {
        if (!D.buf32) HEAT_CHECK(cudaMalloc(&D.buf32, kFields32 * n * sizeof(float)));
        std::vector<float> h32(kFields32 * n);
        for (size_t x = 0; x < kFields32 * n; ++x) h32[x] = (float)host[x];
        HEAT_CHECK(cudaMemcpyAsync(D.buf32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice,
                                   ctx->stream));
        float *q = D.buf32;
        auto G = [&](int a) { return (const float *)(q + a * n); };
        D.t32 = LineTab<float>{G(0), G(1), G(2), G(3), G(4), G(5), G(6), G(7), G(8), G(9), G(10), G(11), G(12), G(13)};
    }
    std::vector<float2> h2;
    if (ctx->precision == HEAT_FP32_REFINED) {
        // the residual's coefficients as FP32 pairs (hi, lo): am, ap, dl, dh, q, b, m, p
        const std::vector<double> *src2[8] = {&T.am, &T.ap, &T.dl, &T.dh, &T.q, &T.b, &T.m, &T.p};
        if (!D.buf2) HEAT_CHECK(cudaMalloc(&D.buf2, 8 * n * sizeof(float2)));
        h2.resize(8 * n);
        for (int a = 0; a < 8; ++a)
            for (size_t x = 0; x < n; ++x) {
                const double v = (*src2[a])[x];
                const float hi = (float)v;
                h2[a * n + x] = make_float2(hi, (float)(v - (double)hi));
            }
        HEAT_CHECK(cudaMemcpyAsync(D.buf2, h2.data(), h2.size() * sizeof(float2), cudaMemcpyHostToDevice,
                                   ctx->stream));
        const float2 *q2 = D.buf2;
        auto P = [&](int a) { return q2 + a * n; };
        D.t2 = LineTab2{P(0), P(1), P(2), P(3), P(4), P(5), P(6), P(7)};
    }
    // host vectors are freed on return: the copies must complete first
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    return HEAT_OK;
}

// Upload the packed z-partition tables in the field precision, laid out as
// [pkA: 4 per (class,row)][pkB: 4], plus the chunk constants, and size the
// chunk scratch (summaries, then carries: 2 x n_chunks x Nr).
template <typename real>
int upload_zpart_t(heat_ctx *ctx, real *&pk, real *&ch)
{
    const size_t npk = (size_t)ctx->Z.n_class * ctx->Z.N;
    std::vector<real> h(8 * npk);
    for (size_t e = 0; e < npk; ++e) {
        const double *src = &ctx->zpk[e * 8];
        for (int f = 0; f < 4; ++f) h[e * 4 + f] = (real)src[f];
        for (int f = 0; f < 4; ++f) h[4 * npk + e * 4 + f] = (real)src[4 + f];
    }
    std::vector<real> hc(ctx->zch.begin(), ctx->zch.end());
    if (pk) cudaFree(pk), pk = nullptr;
    if (ch) cudaFree(ch), ch = nullptr;
    HEAT_CHECK(cudaMalloc(&pk, h.size() * sizeof(real)));
    HEAT_CHECK(cudaMalloc(&ch, hc.size() * sizeof(real)));
    HEAT_CHECK(cudaMemcpyAsync(pk, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_CHECK(cudaMemcpyAsync(ch, hc.data(), hc.size() * sizeof(real), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    return HEAT_OK;
}

int upload_zpart(heat_ctx *ctx)
{
    ZPart &z = ctx->zp;
    {
        std::vector<int> u(z.n_chunks);
        for (int c = 0; c < z.n_chunks; ++c) {
            const int r0 = c * z.Rc, r1 = std::min(ctx->g.Nz, r0 + z.Rc);
            int a = ctx->g.rowcls[r0];
            for (int j = r0; j < r1; ++j)
                if (ctx->g.rowcls[j] != a) a = -1;
            u[c] = a;
        }
        if (z.ucls) cudaFree(z.ucls), z.ucls = nullptr;
        HEAT_CHECK(cudaMalloc(&z.ucls, u.size() * sizeof(int)));
        HEAT_CHECK(cudaMemcpyAsync(z.ucls, u.data(), u.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    {
        // (FP32 paths only: the FP64 passes spill with the tile bookkeeping
        // and ran slower tiled)
        std::vector<int> t;
        if (ctx->precision != HEAT_FP64) t = z_tiles(ctx->g.colcls, ctx->g.Nr, 4);
        if (z.tiles) cudaFree(z.tiles), z.tiles = nullptr;
        z.n_tiles = (int)t.size() / 4;
        if (z.n_tiles) {
            HEAT_CHECK(cudaMalloc(&z.tiles, t.size() * sizeof(int)));
            HEAT_CHECK(cudaMemcpyAsync(z.tiles, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    const size_t nsum = (size_t)z.n_chunks * 4 * ctx->g.Nr;  // summaries [nch][2][Nr] + carries [nch][2][Nr]
    if (ctx->precision == HEAT_FP64) {
        int st = upload_zpart_t<double>(ctx, z.pk64, z.ch64);
        if (st != HEAT_OK) return st;
        if (!ctx->d_zsum64) HEAT_CHECK(cudaMalloc(&ctx->d_zsum64, nsum * sizeof(double)));
    } else {
        int st = upload_zpart_t<float>(ctx, z.pk32, z.ch32);
        if (st != HEAT_OK) return st;
        if (!ctx->d_zsum) HEAT_CHECK(cudaMalloc(&ctx->d_zsum, nsum * sizeof(float)));
    }
    return HEAT_OK;
}

template <typename real>
int upload_rline_t(heat_ctx *ctx, const std::vector<double> *src[4], const std::vector<int> &zcl)
{
    // zcl is followed by the row units: runs of up to kRLineR rows of one class
    size_t n = 0;
    for (int a = 0; a < 4; ++a) n += src[a]->size();
    std::vector<real> h(n);
    size_t o = 0;
    for (int a = 0; a < 4; ++a)
        for (double v : *src[a]) h[o++] = (real)v;
    if (ctx->d_rl) cudaFree(ctx->d_rl), ctx->d_rl = nullptr;
    if (ctx->d_rlz) cudaFree(ctx->d_rlz), ctx->d_rlz = nullptr;
    HEAT_CHECK(cudaMalloc(&ctx->d_rl, n * sizeof(real)));
    HEAT_CHECK(cudaMalloc(&ctx->d_rlz, zcl.size() * sizeof(int)));
    HEAT_CHECK(cudaMemcpyAsync(ctx->d_rl, h.data(), n * sizeof(real), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_CHECK(cudaMemcpyAsync(ctx->d_rlz, zcl.data(), zcl.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    return HEAT_OK;
}

// Build and upload the line-team r-sweep tables (literal and increment forms
// only; the refined path and lines too long for a team buffer keep the
// block-line r-sweep).
int upload_rline(heat_ctx *ctx)
{
    ctx->rl_LW = ctx->rl_nseg = 0;
    if (ctx->precision == HEAT_FP32_REFINED) return HEAT_OK;
    const bool f64 = ctx->precision == HEAT_FP64;
    std::vector<double> tA, tB, tD, tC;
    std::vector<int> zcl;
    int LW = 0, nseg = 0;
    if (!build_rline(ctx, f64 ? rline_K<double>() : rline_K<float>(), kRLineMaxBuf, LW, nseg, tA, tB, tD, tC, zcl))
        return HEAT_OK;
    const int nchunk = (int)zcl.size();
    const Grid &g = ctx->g;
    for (int j = 0; j < g.Nz;) {
        int n = 1;
        while (n < rline_rows(ctx->precision == HEAT_FP64) && j + n < g.Nz && g.rowcls[j + n] == g.rowcls[j]) ++n;
        zcl.push_back(j | (n << 16));
        j += n;
    }
    ctx->rl_nunits = (int)zcl.size() - nchunk;
    ctx->rl_nchunk = nchunk;
    const std::vector<double> *src[4] = {&tA, &tB, &tD, &tC};
    const int st = f64 ? upload_rline_t<double>(ctx, src, zcl) : upload_rline_t<float>(ctx, src, zcl);
    if (st != HEAT_OK) return st;
    ctx->rl_LW = LW;
    ctx->rl_nseg = nseg;
    return HEAT_OK;
}

// Walk r-sweep tables (FP32 increment form, one instance): lines whose rows
// are 16-byte multiples (bulk copies) of at most 32 x 65 cells, at most 32
// column classes.  Lane l, step k holds cell i = l K + k (K the smallest of
// 17, 33, 65 with 32 K >= Nr); cells past Nr get zeros.
int upload_rwalk(heat_ctx *ctx)
{
    ctx->rw_K = 0;
    if (ctx->precision != HEAT_FP32) return HEAT_OK;
    const int Nr = ctx->g.Nr;
    if (Nr % 4 != 0 || Nr > 32 * 65 || ctx->Z.n_class > 32) return HEAT_OK;
    const int K = Nr <= 32 * 17 ? 17 : (Nr <= 32 * 33 ? 33 : 65);
    const int ncls = ctx->R.n_class;
    const size_t per = (size_t)32 * K;
    std::vector<float4> tab(per * ncls, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<signed char> cc(per, 0);
    for (int a = 0; a < ncls; ++a)
        for (int l = 0; l < 32; ++l)
            for (int k = 0; k < K; ++k) {
                const int i = l * K + k;
                if (i >= Nr) continue;
                const size_t ro = (size_t)a * Nr + i;
                const double iv = ctx->R.inv[ro];
                tab[a * per + (size_t)k * 32 + l] =
                    make_float4((float)(ctx->R.xm[ro] * iv), (float)(ctx->R.xp[ro] * iv), (float)(ctx->R.q[ro] * iv),
                                (float)iv);
                if (a == 0) cc[(size_t)k * 32 + l] = (signed char)ctx->g.colcls[i];
            }
    if (ctx->d_rwtab) cudaFree(ctx->d_rwtab), ctx->d_rwtab = nullptr;
    if (ctx->d_rwcc) cudaFree(ctx->d_rwcc), ctx->d_rwcc = nullptr;
    HEAT_CHECK(cudaMalloc(&ctx->d_rwtab, tab.size() * sizeof(float4)));
    HEAT_CHECK(cudaMalloc(&ctx->d_rwcc, cc.size()));
    HEAT_CHECK(cudaMemcpyAsync(ctx->d_rwtab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice,
                               ctx->stream));
    HEAT_CHECK(cudaMemcpyAsync(ctx->d_rwcc, cc.data(), cc.size(), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    ctx->rw_K = K;
    ctx->rw_ncc = ctx->Z.n_class;
    return HEAT_OK;
}

void free_ctx(heat_ctx *ctx)
{
    if (!ctx) return;
    void *bufs[] = {ctx->dR.buf64, ctx->dR.buf32,   ctx->dZ.buf64,   ctx->dZ.buf32, ctx->dR.buf2, ctx->dZ.buf2, ctx->d_rowcls,
                    ctx->d_colcls, ctx->d_wr,       ctx->d_wz,       ctx->d_field[0], ctx->d_field[1],
                    ctx->d_part,   ctx->d_res,      ctx->zp.pk64,    ctx->zp.ch64,  ctx->zp.pk32,
                    ctx->zp.ch32,  ctx->d_zsum,     ctx->d_zsum64,   ctx->d_rho,    ctx->zp.ucls,
                    ctx->d_args,   ctx->d_rl,       ctx->d_rlz,      ctx->zp.tiles, ctx->d_rwtab, ctx->d_rwcc,
                    ctx->d_status, ctx->d_small_bar};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete ctx;
}

size_t elem_size(const heat_ctx *ctx) { return ctx->precision == HEAT_FP64 ? sizeof(double) : sizeof(float); }

}  // namespace

namespace heat {
// heat_set_dt without the batch-member guard (the batch re-plans afterwards).
int ctx_set_dt(heat_ctx *ctx, double dt)
{
    if (!ctx || !(dt > 0.0) || !std::isfinite(dt)) return HEAT_ERR_ARG;
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    ctx->tau = dt;
    build_tables(ctx);
    build_zpartition(ctx);
    int st = upload_tab(ctx, ctx->R, ctx->dR);
    if (st != HEAT_OK) return st;
    if ((st = upload_tab(ctx, ctx->Z, ctx->dZ)) != HEAT_OK) return st;
    if ((st = upload_zpart(ctx)) != HEAT_OK) return st;
    if ((st = upload_rline(ctx)) != HEAT_OK) return st;
    if ((st = upload_rwalk(ctx)) != HEAT_OK) return st;
    return cuda_status(ctx_plan(ctx));
}
}  // namespace heat

extern "C" {

const char *heat_strerror(int status)
{
    switch (status) {
    case HEAT_OK: return "ok";
    case HEAT_ERR_ARG: return "invalid argument";
    case HEAT_ERR_CUDA: return "CUDA error";
    case HEAT_ERR_NONFINITE: return "non-finite field";
    case HEAT_ERR_TIMEOUT: return "device wait timed out";
    case HEAT_ERR_OOM: return "device out of memory";
    case HEAT_ERR_TOO_LARGE: return "size beyond a fixed capacity";
    case HEAT_ERR_NOCONV: return "iteration did not converge";
    default: return "unknown status";
    }
}

int heat_create(const heat_geometry *geom, const heat_materials *mat, const heat_options *opt, double dt,
                void *stream, heat_ctx **out)
{
    return heat::create_ctx(geom, mat, opt, dt, stream, false, out);
}

}  // extern "C"

namespace heat {
// heat_create, for a standalone context or (member = true) a batch member.
int create_ctx(const heat_geometry *geom, const heat_materials *mat, const heat_options *opt, double dt,
               void *stream, bool member, heat_ctx **out)
{
    if (!out) return HEAT_ERR_ARG;
    *out = nullptr;
    int st = validate(geom, mat, opt, dt);
    if (st != HEAT_OK) return st;
    heat_ctx *ctx = new (std::nothrow) heat_ctx();
    if (!ctx) return HEAT_ERR_OOM;
    ctx->batch_member = member;
    ctx->precision = opt->precision;
    ctx->face_mean = opt->face_mean;
    ctx->stream = static_cast<cudaStream_t>(stream);
    {
        const cudaError_t e = cudaGetDevice(&ctx->device);
        if (e != cudaSuccess) {
            delete ctx;
            return cuda_status(e);
        }
    }
    // FP32 fields hold theta = T - T_init (precision where T varies little
    // around T_init); the FP64 field holds T itself, so a checkpoint through
    // heat_field / heat_set_field is lossless in every precision.
    ctx->T_ref = opt->precision == HEAT_FP64 ? 0.0 : mat->T_init;
    for (int f = 0; f < 4; ++f) {
        ctx->bc[f] = geom->bc[f];
        ctx->theta_bc[f] = geom->T_bc[f] - ctx->T_ref;
    }
    ctx->box_region.resize(geom->n_boxes);
    for (int b = 0; b < geom->n_boxes; ++b) ctx->box_region[b] = geom->boxes[b].region;
    ctx->k.assign(mat->k, mat->k + mat->n_regions);
    ctx->C.assign(mat->C, mat->C + mat->n_regions);
    ctx->q.assign(mat->q, mat->q + mat->n_regions);
    ctx->tau = dt;
    build_grid(geom, ctx->g);
    build_tables(ctx);
    build_zpartition(ctx);
    compute_limits(ctx);

    const Grid &g = ctx->g;
    const size_t ncell = (size_t)g.Nr * g.Nz;
    auto fail = [&](int s) {
        free_ctx(ctx);
        return s;
    };
    if ((st = upload_tab(ctx, ctx->R, ctx->dR)) != HEAT_OK) return fail(st);
    if ((st = upload_tab(ctx, ctx->Z, ctx->dZ)) != HEAT_OK) return fail(st);
    if ((st = upload_zpart(ctx)) != HEAT_OK) return fail(st);
    if ((st = upload_rline(ctx)) != HEAT_OK) return fail(st);
    if ((st = upload_rwalk(ctx)) != HEAT_OK) return fail(st);
    std::vector<double> wr(g.Nr), wz(g.Nz);
    for (int i = 0; i < g.Nr; ++i) wr[i] = 2.0 * kPi * g.rc[i] * g.hbar[i];
    for (int j = 0; j < g.Nz; ++j) wz[j] = g.etabar[j];
    cudaError_t e;
#define HEAT_TRY(call)                                   \
    if ((e = (call)) != cudaSuccess) return fail(cuda_status(e))
    HEAT_TRY(cudaMalloc(&ctx->d_rowcls, g.Nz * sizeof(int)));
    HEAT_TRY(cudaMalloc(&ctx->d_colcls, g.Nr * sizeof(int)));
    HEAT_TRY(cudaMalloc(&ctx->d_wr, g.Nr * sizeof(double)));
    HEAT_TRY(cudaMalloc(&ctx->d_wz, g.Nz * sizeof(double)));
    HEAT_TRY(cudaMalloc(&ctx->d_field[0], ncell * elem_size(ctx)));
    HEAT_TRY(cudaMalloc(&ctx->d_field[1], ncell * elem_size(ctx)));
    ctx->n_part = energy_blocks(ctx);
    HEAT_TRY(cudaMalloc(&ctx->d_part, 2 * ctx->n_part * sizeof(double)));
    HEAT_TRY(cudaMalloc(&ctx->d_res, 2 * sizeof(double)));
    HEAT_TRY(cudaMalloc(&ctx->d_status, sizeof(int)));
    HEAT_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    if (ctx->precision == HEAT_FP32_REFINED) HEAT_TRY(cudaMalloc(&ctx->d_rho, ncell * sizeof(float)));
    HEAT_TRY(cudaMemcpyAsync(ctx->d_rowcls, g.rowcls.data(), g.Nz * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_TRY(cudaMemcpyAsync(ctx->d_colcls, g.colcls.data(), g.Nr * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_TRY(cudaMemcpyAsync(ctx->d_wr, wr.data(), g.Nr * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    HEAT_TRY(cudaMemcpyAsync(ctx->d_wz, wz.data(), g.Nz * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // uniform initial field T = T_init (eq. "initcond"), stored as T - T_ref
    HEAT_TRY(launch_fill(ctx, 0, mat->T_init - ctx->T_ref));
    HEAT_TRY(launch_fill(ctx, 1, mat->T_init - ctx->T_ref));
    HEAT_TRY(ctx_plan(ctx));
    HEAT_TRY(small_setup(ctx));
    HEAT_TRY(cudaStreamSynchronize(ctx->stream));
#undef HEAT_TRY
    *out = ctx;
    return HEAT_OK;
}
}  // namespace heat

extern "C" {

int heat_set_dt(heat_ctx *ctx, double dt)
{
    if (!ctx || ctx->batch_member) return HEAT_ERR_ARG;
    return ctx_set_dt(ctx, dt);
}

int heat_sweep(heat_ctx *ctx, int dir)
{
    if (!ctx || (dir != 0 && dir != 1) || ctx->batch_member) return HEAT_ERR_ARG;
    if ((dir == 1) != (ctx->half == 1)) return HEAT_ERR_ARG;
    int st = cuda_status(launch_sweep(ctx, dir));
    if (st != HEAT_OK) return st;
    ctx->cur = 1 - ctx->cur;
    ctx->half = dir == 0 ? 1 : 0;
    return HEAT_OK;
}

int heat_step(heat_ctx *ctx, int n)
{
    if (!ctx || n < 0 || ctx->half) return HEAT_ERR_ARG;
    if (n == 0) return HEAT_OK;
    return cuda_status(launch_steps(ctx, n));
}

int heat_field(heat_ctx *ctx, double *out, size_t n, int on_device)
{
    if (!ctx || !out) return HEAT_ERR_ARG;
    const size_t ncell = (size_t)ctx->g.Nr * ctx->g.Nz;
    if (n != ncell) return HEAT_ERR_ARG;
    if (on_device) return cuda_status(launch_theta_to_T(ctx, out));
    if (ctx->precision == HEAT_FP64) {
        HEAT_CHECK(cudaMemcpyAsync(out, ctx->d_field[ctx->cur], ncell * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
        HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
        for (size_t c = 0; c < ncell; ++c) out[c] += ctx->T_ref;
    } else {
        std::vector<float> tmp(ncell);
        HEAT_CHECK(cudaMemcpyAsync(tmp.data(), ctx->d_field[ctx->cur], ncell * sizeof(float), cudaMemcpyDeviceToHost,
                                   ctx->stream));
        HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
        for (size_t c = 0; c < ncell; ++c) out[c] = (double)tmp[c] + ctx->T_ref;
    }
    return HEAT_OK;
}

int heat_set_field(heat_ctx *ctx, const double *in, size_t n, int on_device)
{
    if (!ctx || !in) return HEAT_ERR_ARG;
    const size_t ncell = (size_t)ctx->g.Nr * ctx->g.Nz;
    if (n != ncell) return HEAT_ERR_ARG;
    if (on_device) return cuda_status(launch_T_to_theta(ctx, in));
    if (ctx->precision == HEAT_FP64) {
        std::vector<double> tmp(ncell);
        for (size_t c = 0; c < ncell; ++c) tmp[c] = in[c] - ctx->T_ref;
        HEAT_CHECK(cudaMemcpyAsync(ctx->d_field[ctx->cur], tmp.data(), ncell * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
        HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    } else {
        std::vector<float> tmp(ncell);
        for (size_t c = 0; c < ncell; ++c) tmp[c] = (float)(in[c] - ctx->T_ref);
        HEAT_CHECK(cudaMemcpyAsync(ctx->d_field[ctx->cur], tmp.data(), ncell * sizeof(float), cudaMemcpyHostToDevice,
                                   ctx->stream));
        HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    return HEAT_OK;
}

int heat_energy(heat_ctx *ctx, double *E, double *Phi, double *Q)
{
    if (!ctx) return HEAT_ERR_ARG;
    HEAT_CHECK(launch_energy(ctx));
    double res[2];
    HEAT_CHECK(cudaMemcpyAsync(res, ctx->d_res, sizeof(res), cudaMemcpyDeviceToHost, ctx->stream));
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    if (E) *E = res[0] + ctx->E_ref;
    if (Phi) *Phi = res[1];
    if (Q) *Q = ctx->Q;
    if (!std::isfinite(res[0]) || !std::isfinite(res[1])) return HEAT_ERR_NONFINITE;
    return HEAT_OK;
}

int heat_info(heat_ctx *ctx, int *Nr, int *Nz, double *r_centres, double *z_centres, double *tau_exp)
{
    if (!ctx) return HEAT_ERR_ARG;
    if (Nr) *Nr = ctx->g.Nr;
    if (Nz) *Nz = ctx->g.Nz;
    if (r_centres) std::memcpy(r_centres, ctx->g.rc.data(), ctx->g.Nr * sizeof(double));
    if (z_centres) std::memcpy(z_centres, ctx->g.zc.data(), ctx->g.Nz * sizeof(double));
    if (tau_exp) *tau_exp = ctx->tau_exp;
    return HEAT_OK;
}

int heat_launches_per_step(heat_ctx *ctx) { return ctx ? launches_per_step(ctx) : HEAT_ERR_ARG; }

int heat_sync(heat_ctx *ctx)
{
    if (!ctx) return HEAT_ERR_ARG;
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    int status = 0;
    HEAT_CHECK(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        HEAT_CHECK(cudaMemset(ctx->d_status, 0, sizeof(int)));
        return HEAT_ERR_TIMEOUT;
    }
    return ctx->deferred;
}

int heat_set_rsweep(heat_ctx *ctx, int kind)
{
    if (!ctx || ctx->batch_member || kind < 0 || kind > 32) return HEAT_ERR_ARG;
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    const int old = ctx->rsweep_req;
    ctx->rsweep_req = kind;
    const cudaError_t e = ctx_plan(ctx);
    if (e == cudaErrorInvalidValue) {  // not available for this context: keep the previous schedule
        ctx->rsweep_req = old;
        const cudaError_t e2 = ctx_plan(ctx);
        return e2 == cudaSuccess ? HEAT_ERR_ARG : cuda_status(e2);
    }
    return cuda_status(e);
}

int heat_get_rsweep(heat_ctx *ctx)
{
    if (!ctx) return HEAT_ERR_ARG;
    return ctx->plan.used.rK;
}

int heat_test_stall(heat_ctx *ctx, int on)
{
    if (!ctx || ctx->batch_member) return HEAT_ERR_ARG;
    HEAT_CHECK(cudaStreamSynchronize(ctx->stream));
    ctx->rw_stall = on ? 1 : 0;
    return cuda_status(ctx_plan(ctx));
}

void heat_destroy(heat_ctx *ctx)
{
    if (!ctx || ctx->batch_member) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

}  // extern "C"
