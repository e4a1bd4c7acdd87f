// heat_sweeps.cu -- host launchers of one ADI step (dispatch by precision to
// the per-form translation units), the FP64 energy/flux reduction and the
// field conversions.  The kernels are in heat_kernels.cuh.
#include "heat_kernels.cuh"

namespace heat {

// Sweep arguments of one instance, from its context (host copy).
template <typename real>
static SweepArgs<real> make_args_t(const heat_ctx *ctx);

template <>
SweepArgs<float> make_args_t<float>(const heat_ctx *ctx)
{
    SweepArgs<float> a{};
    a.R = ctx->dR.t32;
    a.Z = ctx->dZ.t32;
    const size_t npk = (size_t)ctx->Z.n_class * ctx->g.Nz;
    a.pkA = ctx->zp.pk32;
    a.pkB = ctx->zp.pk32 + 4 * npk;
    a.chk = ctx->zp.ch32;
    a.zs = ctx->d_zsum;
    a.rho = ctx->d_rho;
    return a;
}

template <>
SweepArgs<double> make_args_t<double>(const heat_ctx *ctx)
{
    SweepArgs<double> a{};
    a.R = ctx->dR.t64;
    a.Z = ctx->dZ.t64;
    const size_t npk = (size_t)ctx->Z.n_class * ctx->g.Nz;
    a.pkA = ctx->zp.pk64;
    a.pkB = ctx->zp.pk64 + 4 * npk;
    a.chk = ctx->zp.ch64;
    a.zs = ctx->d_zsum64;
    a.rho = nullptr;
    return a;
}

template <typename real>
static void fill_args_t(const heat_ctx *ctx, void *dst)
{
    SweepArgs<real> a = make_args_t<real>(ctx);
    a.Nr = ctx->g.Nr;
    a.Nz = ctx->g.Nz;
    a.G = a.band = 0;  // set by the plan
    a.Rc = ctx->zp.Rc;
    a.nch = ctx->zp.n_chunks;
    a.rowcls = ctx->d_rowcls;
    a.colcls = ctx->d_colcls;
    a.n_run = 0;
    a.rb_runs = 0;
    for (int j = 0; j < a.Nz && a.n_run <= kMaxRun; ++j)
        if (j == 0 || ctx->g.rowcls[j] != ctx->g.rowcls[j - 1]) {
            if (a.n_run < kMaxRun) a.run_lo[a.n_run] = j;
            ++a.n_run;
        }
    if (a.n_run > kMaxRun)
        a.n_run = 0;
    else
        a.run_lo[a.n_run] = a.Nz;
    for (int r = 0; r < a.n_run; ++r) a.run_cls[r] = ctx->g.rowcls[a.run_lo[r]];
    a.R64 = ctx->dR.full;
    a.Z64 = ctx->dZ.full;
    a.R2 = ctx->dR.t2;
    a.Z2 = ctx->dZ.t2;
    for (int f = 0; f < 4; ++f) a.bc.th[f] = ctx->theta_bc[f];
    a.ucls = ctx->zp.ucls;
    a.ztile = ctx->zp.tiles;
    a.n_ztile = ctx->zp.n_tiles;
    a.zc = a.zs + (size_t)2 * a.nch * a.Nr;
    a.rl = RLine<real>{};
    if (ctx->rl_LW > 0) {
        const int K = rline_K<real>();
        const int nchunk = ctx->rl_nseg * ctx->rl_LW;
        const size_t Npad = (size_t)nchunk * K, ncls = (size_t)ctx->R.n_class;
        const real *base = static_cast<const real *>(ctx->d_rl);
        a.rl.tA = base;
        a.rl.tB = a.rl.tA + ncls * Npad * 4;
        a.rl.tD = a.rl.tB + ncls * Npad * 2;
        a.rl.tC = a.rl.tD + ncls * Npad * 2;
        a.rl.zcl = ctx->d_rlz;
        a.rl.unit = ctx->d_rlz + ctx->rl_nchunk;
        a.rl.LW = ctx->rl_LW;
        a.rl.nseg = ctx->rl_nseg;
        a.rl.n_units = ctx->rl_nunits;
    }
    a.f0 = static_cast<real *>(ctx->d_field[0]);
    a.f1 = static_cast<real *>(ctx->d_field[1]);
    a.rw_tab = static_cast<const float4 *>(ctx->d_rwtab);
    a.rw_cc = ctx->d_rwcc;
    a.rw_K = ctx->rw_K;
    a.rw_ncc = ctx->rw_ncc;
    a.rw_stall = ctx->rw_stall;
    a.status = ctx->d_status;
    *static_cast<SweepArgs<real> *>(dst) = a;
}

size_t args_bytes(int precision)
{
    return precision == HEAT_FP64 ? sizeof(SweepArgs<double>) : sizeof(SweepArgs<float>);
}

void fill_args(const heat_ctx *ctx, void *dst)
{
    if (ctx->precision == HEAT_FP64)
        fill_args_t<double>(ctx, dst);
    else
        fill_args_t<float>(ctx, dst);
}

// Plan for n instances whose host arguments are in h (G and band are filled in).
cudaError_t make_plan(int precision, void *h, int n, const Tuning &req, SweepPlan &plan)
{
    switch (precision) {
    case HEAT_FP64: return plan_fp64(static_cast<SweepArgs<double> *>(h), n, req, plan);
    case HEAT_FP32: return plan_fp32(static_cast<SweepArgs<float> *>(h), n, req, plan);
    default: return plan_fp32_refined(static_cast<SweepArgs<float> *>(h), n, req, plan);
    }
}

// Enqueue one half-step of a plan.  flip = 0 reads f0 and writes f1.  Every
// sweep kernel is launched with programmatic stream serialization (see
// pdl_wait in heat_internal.h), so its blocks can be scheduled while the
// previous kernel in the stream drains.
cudaError_t run_plan(const SweepPlan &plan, int dir, const void *d_args, int flip, cudaStream_t s)
{
    for (const Launch &L : plan.dir[dir]) {
        void *kargs[3] = {(void *)&d_args, (void *)&flip, (void *)L.pargs.data()};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = L.grid;
        cfg.blockDim = L.block;
        cfg.dynamicSmemBytes = L.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = L.pdl ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (L.cluster > 1) {
            attr[1].id = cudaLaunchAttributeClusterDimension;
            attr[1].val.clusterDim.x = (unsigned)L.cluster;
            attr[1].val.clusterDim.y = 1;
            attr[1].val.clusterDim.z = 1;
            cfg.numAttrs = 2;
        }
        cudaError_t e = cudaLaunchKernelExC(&cfg, L.fn, kargs);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Point every instance's arguments (n of them in h, of the given precision)
// at the batch work list of the lean z passes.
void set_zitems(int precision, void *h, int n, const void *items, int n_items)
{
    int rc_max = 0;
    for (int i = 0; i < n; ++i) {
        const int rc = precision == HEAT_FP64 ? static_cast<SweepArgs<double> *>(h)[i].Rc
                                              : static_cast<SweepArgs<float> *>(h)[i].Rc;
        rc_max = rc > rc_max ? rc : rc_max;
    }
    for (int i = 0; i < n; ++i) {
        if (precision == HEAT_FP64) {
            SweepArgs<double> &a = static_cast<SweepArgs<double> *>(h)[i];
            a.zitem = static_cast<const int4 *>(items), a.n_zitem = n_items, a.zrc_max = rc_max;
        } else {
            SweepArgs<float> &a = static_cast<SweepArgs<float> *>(h)[i];
            a.zitem = static_cast<const int4 *>(items), a.n_zitem = n_items, a.zrc_max = rc_max;
        }
    }
}

// (Re)build the single-instance plan of a context and upload its arguments.
cudaError_t ctx_plan(heat_ctx *ctx)
{
    ctx->h_args.assign(args_bytes(ctx->precision), 0);
    fill_args(ctx, ctx->h_args.data());
    Tuning req;
    req.rK = ctx->rsweep_req;
    cudaError_t e = make_plan(ctx->precision, ctx->h_args.data(), 1, req, ctx->plan);
    if (e != cudaSuccess) return e;
    if (!ctx->d_args && (e = cudaMalloc(&ctx->d_args, ctx->h_args.size())) != cudaSuccess) return e;
    e = cudaMemcpyAsync(ctx->d_args, ctx->h_args.data(), ctx->h_args.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(ctx->stream);
}

cudaError_t launch_sweep(heat_ctx *ctx, int dir)
{
    return run_plan(ctx->plan, dir, ctx->d_args, ctx->cur, ctx->stream);
}

cudaError_t launch_small_steps(heat_ctx *ctx, int n);

cudaError_t launch_steps(heat_ctx *ctx, int n)
{
    if (ctx->small_fn && ctx->rsweep_req == 0) return launch_small_steps(ctx, n);
    for (int s = 0; s < n; ++s) {
        cudaError_t e = run_plan(ctx->plan, 0, ctx->d_args, ctx->cur, ctx->stream);
        if (e != cudaSuccess) return e;
        e = run_plan(ctx->plan, 1, ctx->d_args, 1 - ctx->cur, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int launches_per_step(const heat_ctx *ctx)
{
    if (ctx->small_fn && ctx->rsweep_req == 0) return 1;  // (one launch runs all n steps)
    return (int)(ctx->plan.dir[0].size() + ctx->plan.dir[1].size());
}

int energy_blocks(const heat_ctx *ctx)
{
    const int nb = ctx->g.Nz < 1024 ? ctx->g.Nz : 1024;
    return nb;
}

cudaError_t launch_energy(heat_ctx *ctx)
{
    const int nb = energy_blocks(ctx);
    if (ctx->precision == HEAT_FP64)
        energy_kernel<double><<<nb, 256, 0, ctx->stream>>>(static_cast<const double *>(ctx->d_field[ctx->cur]),
                                                          ctx->g.Nr, ctx->g.Nz, ctx->d_rowcls, ctx->d_colcls,
                                                          ctx->dR.full, ctx->dZ.full, ctx->d_wr, ctx->d_wz,
                                                          ctx->d_part);
    else
        energy_kernel<float><<<nb, 256, 0, ctx->stream>>>(static_cast<const float *>(ctx->d_field[ctx->cur]),
                                                         ctx->g.Nr, ctx->g.Nz, ctx->d_rowcls, ctx->d_colcls,
                                                         ctx->dR.full, ctx->dZ.full, ctx->d_wr, ctx->d_wz,
                                                         ctx->d_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d_part, nb, ctx->d_res);
    return cudaGetLastError();
}

cudaError_t launch_theta_to_T(heat_ctx *ctx, double *T)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        theta_to_T_kernel<double><<<grid, 256, 0, ctx->stream>>>(static_cast<const double *>(ctx->d_field[ctx->cur]), T,
                                                                n, ctx->T_ref);
    else
        theta_to_T_kernel<float><<<grid, 256, 0, ctx->stream>>>(static_cast<const float *>(ctx->d_field[ctx->cur]), T,
                                                               n, ctx->T_ref);
    return cudaGetLastError();
}

cudaError_t launch_T_to_theta(heat_ctx *ctx, const double *T)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        T_to_theta_kernel<double><<<grid, 256, 0, ctx->stream>>>(T, static_cast<double *>(ctx->d_field[ctx->cur]), n,
                                                                ctx->T_ref);
    else
        T_to_theta_kernel<float><<<grid, 256, 0, ctx->stream>>>(T, static_cast<float *>(ctx->d_field[ctx->cur]), n,
                                                               ctx->T_ref);
    return cudaGetLastError();
}

cudaError_t launch_fill(heat_ctx *ctx, int buf, double value)
{
    const size_t n = (size_t)ctx->g.Nr * ctx->g.Nz;
    const int grid = kSMs * 8;
    if (ctx->precision == HEAT_FP64)
        fill_kernel<double><<<grid, 256, 0, ctx->stream>>>(static_cast<double *>(ctx->d_field[buf]), n, value);
    else
        fill_kernel<float><<<grid, 256, 0, ctx->stream>>>(static_cast<float *>(ctx->d_field[buf]), n, (float)value);
    return cudaGetLastError();
}

}  // namespace heat
