// heat_batch.cu -- the batched ensemble: n independent problems of one
// precision advanced in lockstep.
//
// Each member is an ordinary context (own grid, line-class tables, fields and
// scratch).  The batch owns one device array of the members' SweepArgs and a
// plan whose every launch covers all members: the member index is blockIdx.y
// of the r-sweep and of the carry pass and blockIdx.z of the chunk passes,
// and blocks past a member's rows, columns or chunks return at once.  One
// step is therefore a fixed 4 launches (7 on the refined path) whatever n is,
// and heat_batch_step replays CUDA graphs of whole steps captured on the
// batch's own stream, so host launch cost does not grow with n or with the
// number of steps.  No block waits on another block.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "heat_internal.h"

namespace heat {
size_t args_bytes(int precision);
void fill_args(const heat_ctx *ctx, void *dst);
void set_zitems(int precision, void *h, int n, const void *items, int n_items);
cudaError_t make_plan(int precision, void *h, int n, const Tuning &req, SweepPlan &plan);
cudaError_t run_plan(const SweepPlan &plan, int dir, const void *d_args, int flip, cudaStream_t s);
int ctx_set_dt(heat_ctx *ctx, double dt);
int create_ctx(const heat_geometry *, const heat_materials *, const heat_options *, double, void *, bool,
               heat_ctx **);
}  // namespace heat

using namespace heat;

namespace {

constexpr int kGraphSteps = 10;  // steps per graph replay (plus a one-step graph for the rest)

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return HEAT_OK;
    if (std::getenv("HEAT_DEBUG")) std::fprintf(stderr, "libheat: %s\n", cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return HEAT_ERR_OOM;
    return HEAT_ERR_CUDA;
}

}  // namespace

struct heat_batch {
    int n = 0;
    int precision = HEAT_FP32;
    std::vector<heat_ctx *> m;
    cudaStream_t s = nullptr;     // owned, non-blocking: every member's stream
    cudaStream_t user = nullptr;  // the caller's stream (0 = legacy default): ordering only
    cudaEvent_t ev = nullptr;
    std::vector<unsigned char> h_args;  // n x SweepArgs<real>
    void *d_args = nullptr;
    SweepPlan plan;
    cudaGraphExec_t g1 = nullptr, gk = nullptr;
    int4 *d_zitem = nullptr;  // work list of the lean z passes (see build_zitems)
    int n_zitem = 0;
};

namespace {

void drop_graphs(heat_batch *b)
{
    if (b->g1) cudaGraphExecDestroy(b->g1), b->g1 = nullptr;
    if (b->gk) cudaGraphExecDestroy(b->gk), b->gk = nullptr;
}

void free_batch(heat_batch *b)
{
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    drop_graphs(b);
    for (heat_ctx *c : b->m) {
        c->batch_member = false;
        heat_destroy(c);
    }
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_zitem) cudaFree(b->d_zitem);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
}

// Capture `steps` whole steps of the current plan into an executable graph.
cudaError_t capture(heat_batch *b, int steps, cudaGraphExec_t *exec)
{
    cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < steps && le == cudaSuccess; ++k) {
        le = run_plan(b->plan, 0, b->d_args, 0, b->s);
        if (le == cudaSuccess) le = run_plan(b->plan, 1, b->d_args, 1, b->s);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->s, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// The work list of the lean z passes: one warp per (member, chunk, column
// tile), the member's column tiles of one class each where z_tiles gives
// them (FP32), else its warps of 32 V columns.  With it, no warp of a z pass
// is idle: a grid over (widest member's warps, most chunks, members) leaves
// the warps and chunks the smaller members lack empty.
cudaError_t build_zitems(heat_batch *b)
{
    b->n_zitem = 0;
    if (b->n > 0xffff) return cudaSuccess;  // (the grid then serves)
    const int V = b->precision == HEAT_FP64 ? 2 : 4, COLS = 32 * V;
    std::vector<int> it;
    for (int i = 0; i < b->n; ++i) {
        const heat_ctx *c = b->m[i];
        const int Nr = c->g.Nr, nch = c->zp.n_chunks;
        std::vector<int> t;
        if (b->precision == HEAT_FP32) t = z_tiles(c->g.colcls, Nr, 4);
        if (t.empty())
            for (int g = 0; g * COLS < Nr; ++g) {
                t.push_back(g * COLS), t.push_back(g * COLS), t.push_back(std::min(Nr, (g + 1) * COLS));
                t.push_back(0);
            }
        for (int ch = 0; ch < nch; ++ch)
            for (size_t k = 0; k < t.size(); k += 4) {
                it.push_back(i | ch << 16), it.push_back(t[k]), it.push_back(t[k + 1]), it.push_back(t[k + 2]);
            }
    }
    if (b->d_zitem) cudaFree(b->d_zitem), b->d_zitem = nullptr;
    cudaError_t e = cudaMalloc(&b->d_zitem, it.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_zitem, it.data(), it.size() * sizeof(int), cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e == cudaSuccess) b->n_zitem = (int)it.size() / 4;
    return e;
}

// Build the plan for `req`, upload the arguments it filled in and capture
// the step graphs.
cudaError_t apply_tuning(heat_batch *b, const Tuning &req)
{
    cudaError_t e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return e;
    SweepPlan p;
    std::vector<unsigned char> h = b->h_args;
    if ((e = make_plan(b->precision, h.data(), b->n, req, p)) != cudaSuccess) return e;
    b->h_args.swap(h);
    b->plan = p;
    e = cudaMemcpyAsync(b->d_args, b->h_args.data(), b->h_args.size(), cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return e;
    drop_graphs(b);
    if ((e = capture(b, 1, &b->g1)) != cudaSuccess) return e;
    return capture(b, kGraphSteps, &b->gk);
}

int member_Nr(const heat_geometry *g)
{
    long long n = 0;
    for (int l = 0; l < g->n_r_layers; ++l) n += g->r_cells[l];
    return n > (1 << 30) ? (1 << 30) : (int)n;
}

}  // namespace

extern "C" {

int heat_batch_create(int n, const heat_geometry *geoms, const heat_materials *mats, const heat_options *opt,
                      const double *dts, void *stream, heat_batch **out)
{
    if (!out) return HEAT_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 65535 || !geoms || !mats || !opt || !dts) return HEAT_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!geoms[i].r_cells || geoms[i].n_r_layers < 1 || member_Nr(&geoms[i]) > HEAT_BATCH_MAX_NR)
            return HEAT_ERR_ARG;
    heat_batch *b = new (std::nothrow) heat_batch();
    if (!b) return HEAT_ERR_OOM;
    b->n = n;
    b->precision = opt->precision;
    b->user = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_status(e);
    }
    b->m.reserve(n);
    const size_t ab = args_bytes(b->precision);
    b->h_args.assign(ab * n, 0);
    for (int i = 0; i < n; ++i) {
        heat_ctx *c = nullptr;
        int st = create_ctx(&geoms[i], &mats[i], opt, dts[i], b->s, true, &c);
        if (st != HEAT_OK) {
            free_batch(b);
            return st;
        }
        b->m.push_back(c);
        fill_args(c, b->h_args.data() + ab * i);
    }
    if ((e = build_zitems(b)) == cudaSuccess)
        set_zitems(b->precision, b->h_args.data(), b->n, b->d_zitem, b->n_zitem);
    if (e != cudaSuccess || (e = cudaMalloc(&b->d_args, b->h_args.size())) != cudaSuccess ||
        (e = apply_tuning(b, Tuning())) != cudaSuccess) {
        free_batch(b);
        return cuda_status(e);
    }
    *out = b;
    return HEAT_OK;
}

int heat_batch_set_dt(heat_batch *b, const double *dts)
{
    if (!b || !dts) return HEAT_ERR_ARG;
    for (int i = 0; i < b->n; ++i)
        if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return HEAT_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t ab = args_bytes(b->precision);
    for (int i = 0; i < b->n; ++i) {
        const int st = ctx_set_dt(b->m[i], dts[i]);
        if (st != HEAT_OK) return st;
        fill_args(b->m[i], b->h_args.data() + ab * i);  // table pointers may have moved
    }
    set_zitems(b->precision, b->h_args.data(), b->n, b->d_zitem, b->n_zitem);
    return cuda_status(apply_tuning(b, b->plan.used));
}

int heat_batch_member(heat_batch *b, int i, heat_ctx **ctx)
{
    if (!b || !ctx || i < 0 || i >= b->n) return HEAT_ERR_ARG;
    *ctx = b->m[i];
    return HEAT_OK;
}

int heat_batch_step(heat_batch *b, int n)
{
    if (!b || n < 0) return HEAT_ERR_ARG;
    for (heat_ctx *c : b->m)
        if (c->half || c->cur != 0) return HEAT_ERR_ARG;
    if (n == 0) return HEAT_OK;
    cudaError_t e = cudaEventRecord(b->ev, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, b->ev, 0);
    for (int k = 0; k < n / kGraphSteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->gk, b->s);
    for (int k = 0; k < n % kGraphSteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->g1, b->s);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev, 0);
    return cuda_status(e);
}

int heat_batch_sync(heat_batch *b)
{
    if (!b) return HEAT_ERR_ARG;
    return cuda_status(cudaStreamSynchronize(b->s));
}

int heat_batch_set_tuning(heat_batch *b, int rK, int band, int zwpb)
{
    if (!b || rK < 0 || band < 0 || band > 4096 || zwpb < 0 || zwpb > 2) return HEAT_ERR_ARG;
    if (rK != 0 && rK != 1 && rK != 2 && rK != 4 && rK != 8 && rK != 16 && rK != 32) return HEAT_ERR_ARG;
    Tuning t;
    t.rK = rK;
    t.band = band;
    t.zwpb = zwpb;
    const Tuning old = b->plan.used;
    cudaError_t e = apply_tuning(b, t);
    if (e == cudaErrorInvalidValue) {  // not a valid schedule for these members: keep the old one
        apply_tuning(b, old);
        return HEAT_ERR_ARG;
    }
    return cuda_status(e);
}

int heat_batch_get_tuning(heat_batch *b, int *rK, int *band, int *zwpb)
{
    if (!b) return HEAT_ERR_ARG;
    if (rK) *rK = b->plan.used.rK;
    if (band) *band = b->plan.used.band;
    if (zwpb) *zwpb = b->plan.used.zwpb;
    return HEAT_OK;
}

int heat_batch_tune(heat_batch *b, int trial_steps, double *best_ms)
{
    if (!b || trial_steps < 1 || trial_steps > 1000) return HEAT_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return cuda_status(e);
    // save every member's field: the trials advance the state
    size_t total = 0;
    std::vector<size_t> off(b->n);
    for (int i = 0; i < b->n; ++i) {
        off[i] = total;
        const size_t bytes = (size_t)b->m[i]->g.Nr * b->m[i]->g.Nz * (b->precision == HEAT_FP64 ? 8 : 4);
        total += (bytes + 255) / 256 * 256;
    }
    unsigned char *save = nullptr;
    if ((e = cudaMalloc(&save, total)) != cudaSuccess) return cuda_status(e);
    auto copy_all = [&](bool to_save) {
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < b->n && r == cudaSuccess; ++i) {
            heat_ctx *c = b->m[i];
            const size_t bytes = (size_t)c->g.Nr * c->g.Nz * (b->precision == HEAT_FP64 ? 8 : 4);
            r = to_save ? cudaMemcpyAsync(save + off[i], c->d_field[0], bytes, cudaMemcpyDeviceToDevice, b->s)
                        : cudaMemcpyAsync(c->d_field[0], save + off[i], bytes, cudaMemcpyDeviceToDevice, b->s);
        }
        return r;
    };
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = copy_all(true);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const Tuning start = b->plan.used;
    Tuning best = start;
    float best_t = -1.f;
    const int Ks[] = {1, 2, 4, 8, 16, 32};  // 1: line teams, 2: register-resident lines
    const int bands[] = {0, 1, 2, 4, 8, 16, 32};
    for (int K : Ks)
        for (int band : bands)
            for (int w = 1; w <= 2 && e == cudaSuccess; ++w) {
                if (b->precision != HEAT_FP64 && K == 4) continue;
                if (K == 1 && band > 16) continue;
                if (K == 2 && band == 1) continue;
                Tuning t;
                t.rK = K;
                t.band = band;
                t.zwpb = w;
                cudaError_t pe = apply_tuning(b, t);
                if (pe == cudaErrorInvalidValue) continue;  // not a valid schedule here
                if ((e = pe) != cudaSuccess) break;
                e = cudaGraphLaunch(b->g1, b->s);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(t0, b->s);
                for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->g1, b->s);
                if (e == cudaSuccess) e = cudaEventRecord(t1, b->s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess && (best_t < 0.f || ms < best_t)) {
                    best_t = ms;
                    best = b->plan.used;
                }
            }
    if (e == cudaSuccess) e = copy_all(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e == cudaSuccess) e = apply_tuning(b, best);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(save);
    if (e == cudaSuccess && best_ms) *best_ms = best_t / trial_steps;
    return cuda_status(e);
}

int heat_batch_launches_per_step(heat_batch *b)
{
    return b ? (int)(b->plan.dir[0].size() + b->plan.dir[1].size()) : HEAT_ERR_ARG;
}

void heat_batch_destroy(heat_batch *b) { free_batch(b); }

}  // extern "C"
