// fno.cu -- the temperature-field surrogate (a Fourier neural operator) on
// the GPU: forward, loss, backward and Adam built from the BF16 tensor-core
// GEMM of fno_gemm.cuh and a few fused elementwise kernels, plus the
// solver-checked inference.  The network and its parameter layout are
// defined in include/surrogate.h.
//
// Spectral layer as GEMMs (per sample b and channel c; v is [Nz][Nr]):
//   A1 = v Fr^T            [Nz][2mr]   r-DFT of the kept kr (cos, -sin)
//   P2 = Fz A1             [2MZ][2mr]  z-DFT of the kept kz (cos, sin rows)
//   X  = combine(P2)       complex [MZ][mr], laid out per mode as [b][(c,re/im)]
//   Y  = X Wblk            per mode: [B][2C] x [2C][2C], Wblk the real 2x2-block
//                          form of the complex C x C weights
//   Yh = arrange(Y)        [2MZ][2mr]
//   A3 = Fz^T Yh           [Nz][2mr]   inverse z-DFT
//   S  = A3 Gr             [Nz][Nr]    inverse r-DFT (weights a_kr / (Nz Nr))
//   pre = W v + wb + S     (the pointwise GEMM adds S and the bias in its epilogue)
// The backward pass runs the transposed GEMMs in reverse order.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fno_gemm.cuh"
#include "heat_internal.h"
#include "surrogate.h"

using fno::bf16;
using fno::GemmArgs;

namespace {

constexpr double kLnKLo = -2.302585092994046;  // ln 0.1
constexpr double kLnKHi = 5.991464547107982;   // ln 400
constexpr double kQLo = 1.0e5, kQHi = 1.0e7;
constexpr double kTdMid = 300.0, kTdHalf = 50.0;
constexpr double kSQ = 0.02;
constexpr int kSplit = 16;  // split-K factor of the weight-gradient GEMMs
constexpr int kF = 16;      // input features per cell (include/surrogate.h)
constexpr double kPiD = 3.14159265358979323846;

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return HEAT_OK;
    if (std::getenv("HEAT_DEBUG")) std::fprintf(stderr, "libheat(surrogate): %s\n", cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return HEAT_ERR_OOM;
    return HEAT_ERR_CUDA;
}

#define SURR_TRY(call)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_status(e_);    \
    } while (0)

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ void features(const double *__restrict__ p, float rnorm, float znorm, float (&x)[9])
{
#pragma unroll
    for (int m = 0; m < 5; ++m) x[m] = (float)(2.0 * (log(p[m]) - kLnKLo) / (kLnKHi - kLnKLo) - 1.0);
    x[5] = (float)(2.0 * (p[5] - kQLo) / (kQHi - kQLo) - 1.0);
    x[6] = (float)((p[6] - kTdMid) / kTdHalf);
    x[7] = rnorm;
    x[8] = znorm;
}

// The 16 features of cell p of a sample whose 7 per-sample features are xs:
// xs, r, z, the one-hot region of the cell (reg[p], -1 on void), the cell's
// ln k feature and the heater source feature.
__device__ __forceinline__ void cell_features(const float (&xs)[7], float r, float z, int reg, int heater,
                                              float (&x)[kF])
{
#pragma unroll
    for (int f = 0; f < 7; ++f) x[f] = xs[f];
    x[7] = r;
    x[8] = z;
#pragma unroll
    for (int m = 0; m < 5; ++m) x[9 + m] = reg == m ? 1.f : 0.f;
    x[14] = reg >= 0 && reg < 5 ? xs[reg] : 0.f;
    x[15] = reg == heater ? xs[5] : 0.f;
}

// v0[b][c][p] = P x + pb.  Grid (chunks of p, B): the 7 features of sample
// b are formed once per block (FP64 logarithms) and shared.
__global__ void lift_kernel(const double *__restrict__ params, const float *__restrict__ rn,
                            const float *__restrict__ zn, const signed char *__restrict__ reg, int heater, int B,
                            int Nz, int Nr, int C, const float *__restrict__ Pw, const float *__restrict__ pb,
                            bf16 *__restrict__ v0)
{
    const long long P = (long long)Nz * Nr;
    const int b = blockIdx.y;
    __shared__ float sxs[7];
    if (threadIdx.x == 0) {
        float x9[9];
        features(params + 7 * b, 0.f, 0.f, x9);
        for (int f = 0; f < 7; ++f) sxs[f] = x9[f];
    }
    __syncthreads();
    float xs[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) xs[f] = sxs[f];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(p / Nr), i = (int)(p - (long long)j * Nr);
        float x[kF];
        cell_features(xs, rn[i], zn[j], reg[p], heater, x);
        bf16 *dst = v0 + (long long)b * C * P + p;
        for (int c = 0; c < C; ++c) {
            float s = pb[c];
#pragma unroll
            for (int f = 0; f < kF; ++f) s = fmaf(Pw[c * kF + f], x[f], s);
            dst[(long long)c * P] = __float2bfloat16(s);
        }
    }
}

// dP[c][f] += sum over b, p of dv0[b][c][p] x_f,  dpb[c] += sum dv0.  Block per
// (b, c): the row sums S = sum_p dv0, Sr = sum_p dv0 r_i, Sz = sum_p dv0 z_j and
// S_m = sum over the cells of region m of dv0; then the 7 per-sample features
// contribute x_f(b) S, the coordinates Sr and Sz, the one-hot channels S_m,
// the cell ln k channel sum_m x_m(b) S_m and the heater channel x_5(b) S_heater.
__global__ void lift_bwd_kernel(const double *__restrict__ params, const float *__restrict__ rn,
                                const float *__restrict__ zn, const signed char *__restrict__ reg, int heater, int B,
                                int Nz, int Nr, int C, const float *__restrict__ dv0, float *__restrict__ gP,
                                float *__restrict__ gpb)
{
    const int c = blockIdx.x, b = blockIdx.y;
    const long long P = (long long)Nz * Nr;
    const float *__restrict__ row = dv0 + ((long long)b * C + c) * P;
    float acc[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) acc[f] = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) {
        const int j = (int)(p / Nr), i = (int)(p - (long long)j * Nr);
        const float g = row[p];
        const int r = reg[p];
        acc[0] += g;
        acc[1] = fmaf(g, rn[i], acc[1]);
        acc[2] = fmaf(g, zn[j], acc[2]);
#pragma unroll
        for (int m = 0; m < 5; ++m) acc[3 + m] += r == m ? g : 0.f;
    }
    __shared__ float red[8][256];
#pragma unroll
    for (int f = 0; f < 8; ++f) red[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int f = 0; f < 8; ++f) red[f][threadIdx.x] += red[f][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float x[9];
        features(params + 7 * b, 0.f, 0.f, x);
        const float S = red[0][0];
        float* g = gP + (size_t)c * kF;
        for (int f = 0; f < 7; ++f) atomicAdd(&g[f], x[f] * S);
        atomicAdd(&g[7], red[1][0]);
        atomicAdd(&g[8], red[2][0]);
        float lnk = 0.f;
        for (int m = 0; m < 5; ++m) {
            atomicAdd(&g[9 + m], red[3 + m][0]);
            lnk = fmaf(x[m], red[3 + m][0], lnk);
        }
        atomicAdd(&g[14], lnk);
        if (heater >= 0 && heater < 5) atomicAdd(&g[15], x[5] * red[3 + heater][0]);
        atomicAdd(&gpb[c], S);
    }
}

// P2 [BC][2MZ][2mr] -> Xm [MZ*mr][B][2C]
__global__ void mix_in_kernel(const float *__restrict__ P2, int B, int C, int MZ, int mr, bf16 *__restrict__ Xm)
{
    const int W2 = 2 * mr, Z2 = 2 * MZ;
    const long long n = (long long)B * C * MZ * mr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int kr = (int)(t % mr);
        const int kzi = (int)((t / mr) % MZ);
        const long long bc = t / ((long long)mr * MZ);
        const int c = (int)(bc % C), b = (int)(bc / C);
        const float *q = P2 + bc * Z2 * W2;
        const float cr = q[(kzi * 2 + 0) * W2 + kr * 2 + 0], ci = q[(kzi * 2 + 0) * W2 + kr * 2 + 1];
        const float sr = q[(kzi * 2 + 1) * W2 + kr * 2 + 0], si = q[(kzi * 2 + 1) * W2 + kr * 2 + 1];
        const long long o = ((long long)(kzi * mr + kr) * B + b) * 2 * C + 2 * c;
        Xm[o] = __float2bfloat16(cr + si);
        Xm[o + 1] = __float2bfloat16(ci - sr);
    }
}

// Ym [MZ*mr][B][2C] -> Yh [BC][2MZ][2mr]
__global__ void mix_out_kernel(const float *__restrict__ Ym, int B, int C, int MZ, int mr, bf16 *__restrict__ Yh)
{
    const int W2 = 2 * mr, Z2 = 2 * MZ;
    const long long n = (long long)B * C * MZ * mr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int kr = (int)(t % mr);
        const int kzi = (int)((t / mr) % MZ);
        const long long bo = t / ((long long)mr * MZ);
        const int o = (int)(bo % C), b = (int)(bo / C);
        const long long s = ((long long)(kzi * mr + kr) * B + b) * 2 * C + 2 * o;
        const float yr = Ym[s], yi = Ym[s + 1];
        bf16 *q = Yh + bo * Z2 * W2;
        q[(kzi * 2 + 0) * W2 + kr * 2 + 0] = __float2bfloat16(yr);
        q[(kzi * 2 + 1) * W2 + kr * 2 + 0] = __float2bfloat16(-yi);
        q[(kzi * 2 + 0) * W2 + kr * 2 + 1] = __float2bfloat16(yi);
        q[(kzi * 2 + 1) * W2 + kr * 2 + 1] = __float2bfloat16(yr);
    }
}

// adjoint of mix_out: gYh [BC][2MZ][2mr] (FP32) -> gYm [MZ*mr][B][2C]
__global__ void mix_out_bwd_kernel(const float *__restrict__ gYh, int B, int C, int MZ, int mr,
                                   bf16 *__restrict__ gYm)
{
    const int W2 = 2 * mr, Z2 = 2 * MZ;
    const long long n = (long long)B * C * MZ * mr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int kr = (int)(t % mr);
        const int kzi = (int)((t / mr) % MZ);
        const long long bo = t / ((long long)mr * MZ);
        const int o = (int)(bo % C), b = (int)(bo / C);
        const float *q = gYh + bo * Z2 * W2;
        const float gre = q[(kzi * 2 + 0) * W2 + kr * 2 + 0] + q[(kzi * 2 + 1) * W2 + kr * 2 + 1];
        const float gim = q[(kzi * 2 + 0) * W2 + kr * 2 + 1] - q[(kzi * 2 + 1) * W2 + kr * 2 + 0];
        const long long s = ((long long)(kzi * mr + kr) * B + b) * 2 * C + 2 * o;
        gYm[s] = __float2bfloat16(gre);
        gYm[s + 1] = __float2bfloat16(gim);
    }
}

// adjoint of mix_in: gXm [MZ*mr][B][2C] (FP32) -> gP2 [BC][2MZ][2mr]
__global__ void mix_in_bwd_kernel(const float *__restrict__ gXm, int B, int C, int MZ, int mr,
                                  bf16 *__restrict__ gP2)
{
    const int W2 = 2 * mr, Z2 = 2 * MZ;
    const long long n = (long long)B * C * MZ * mr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int kr = (int)(t % mr);
        const int kzi = (int)((t / mr) % MZ);
        const long long bc = t / ((long long)mr * MZ);
        const int c = (int)(bc % C), b = (int)(bc / C);
        const long long s = ((long long)(kzi * mr + kr) * B + b) * 2 * C + 2 * c;
        const float gre = gXm[s], gim = gXm[s + 1];
        bf16 *q = gP2 + bc * Z2 * W2;
        q[(kzi * 2 + 0) * W2 + kr * 2 + 0] = __float2bfloat16(gre);
        q[(kzi * 2 + 1) * W2 + kr * 2 + 1] = __float2bfloat16(gre);
        q[(kzi * 2 + 0) * W2 + kr * 2 + 1] = __float2bfloat16(gim);
        q[(kzi * 2 + 1) * W2 + kr * 2 + 0] = __float2bfloat16(-gim);
    }
}

// Output head: u = Q2 h + q2b, T = T_init + S_Q q u0 + (T_D - T_init) u1.
// With Ttrue: loss sum += e^2 (e = (T - Ttrue)/(S_Q q)) and gu = dL/du (BF16).
__global__ void head_kernel(const bf16 *__restrict__ h, const double *__restrict__ params, int B, long long P, int H,
                            const float *__restrict__ Q2, const float *__restrict__ q2b, double T_init,
                            const signed char *__restrict__ reg, float *__restrict__ T,
                            const float *__restrict__ Ttrue, double inv_ntot, bf16 *__restrict__ gu,
                            double *__restrict__ loss)
{
    double lsum = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < B * P; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / P);
        const long long p = t - b * P;
        const bf16 *hp = h + (long long)b * H * P + p;
        float u0 = q2b[0], u1 = q2b[1];
        for (int k = 0; k < H; ++k) {
            const float hv = __bfloat162float(hp[(long long)k * P]);
            u0 = fmaf(Q2[k], hv, u0);
            u1 = fmaf(Q2[H + k], hv, u1);
        }
        const double q = params[7 * b + 5], Td = params[7 * b + 6];
        const double sc = kSQ * q;
        const double act = reg[p] >= 0 ? 1.0 : 0.0;  // void cells hold T_init
        const double Tv = T_init + act * (sc * u0 + (Td - T_init) * u1);
        T[t] = (float)Tv;
        if (Ttrue) {
            const double e = (Tv - (double)Ttrue[t]) / sc;
            lsum += e * e;
            const double gT = 2.0 * e / sc * inv_ntot * act;
            gu[(long long)b * 2 * P + p] = __float2bfloat16((float)(gT * sc));
            gu[(long long)b * 2 * P + P + p] = __float2bfloat16((float)(gT * (Td - T_init)));
        }
    }
    if (Ttrue) {
        __shared__ double red[256];
        red[threadIdx.x] = lsum;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(loss, red[0]);
    }
}

// dst[b][:] = src[idx[b]][:]   (a minibatch of training fields)
__global__ void gather_rows_kernel(const float *__restrict__ src, const int *__restrict__ idx, int B, long long P,
                                   float *__restrict__ dst)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < B * P; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / P);
        const long long p = t - b * P;
        dst[t] = src[(long long)idx[b] * P + p];
    }
}

// Per sample b (block b): max |T - Tt| and max |Tt - T_init| -> out[2b], out[2b+1].
__global__ void err_kernel(const float *__restrict__ T, const float *__restrict__ Tt, long long P, double T_init,
                           double *__restrict__ out)
{
    const int b = blockIdx.x;
    double e = 0.0, r = 0.0;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) {
        const double tt = (double)Tt[(long long)b * P + p];
        e = fmax(e, fabs((double)T[(long long)b * P + p] - tt));
        r = fmax(r, fabs(tt - T_init));
    }
    __shared__ double se[256], sr[256];
    se[threadIdx.x] = e;
    sr[threadIdx.x] = r;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + s]);
            sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * b] = se[0];
        out[2 * b + 1] = sr[0];
    }
}

// out[r] += sum over b, p of src[b][r][p]   (block per (r, chunk))
__global__ void rowsum_kernel(const bf16 *__restrict__ src, int B, int R, long long P, float *__restrict__ out)
{
    const int r = blockIdx.y;
    float s = 0.f;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < B * P; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / P);
        const long long p = t - b * P;
        s += __bfloat162float(src[((long long)b * R + r) * P + p]);
    }
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[r], red[0]);
}

// out[e] += sum_{q < nparts} parts[q n + e]
__global__ void reduce_parts_kernel(const float *__restrict__ parts, int nparts, int n, float *__restrict__ out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < nparts; ++q) s += parts[(long long)q * n + e];
        out[e] += s;
    }
}

// dWblk [MZ*mr][2C][2C] -> dRre, dRim [MZ][mr][C][C] (+=)
__global__ void wblk_grad_kernel(const float *__restrict__ dW, int NM, int C, float *__restrict__ gRre,
                                 float *__restrict__ gRim)
{
    const long long n = (long long)NM * C * C;
    const int C2 = 2 * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t % C), c = (int)((t / C) % C);
        const long long m = t / ((long long)C * C);
        const float *w = dW + m * C2 * C2;
        gRre[t] += w[(2 * c) * C2 + 2 * o] + w[(2 * c + 1) * C2 + 2 * o + 1];
        gRim[t] += w[(2 * c) * C2 + 2 * o + 1] - w[(2 * c + 1) * C2 + 2 * o];
    }
}

__global__ void adam_kernel(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.f - b1) * ge;
        const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        w[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
    }
}

__global__ void cast_kernel(const float *__restrict__ src, long long n, bf16 *__restrict__ dst)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16(src[e]);
}

// Wblk [MZ*mr][(c,p)][(o,q)] from Rre, Rim [MZ][mr][C][C]
__global__ void wblk_kernel(const float *__restrict__ Rre, const float *__restrict__ Rim, int NM, int C,
                            bf16 *__restrict__ Wb)
{
    const long long n = (long long)NM * C * C;
    const int C2 = 2 * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t % C), c = (int)((t / C) % C);
        const long long m = t / ((long long)C * C);
        bf16 *w = Wb + m * C2 * C2;
        const float re = Rre[t], im = Rim[t];
        w[(2 * c) * C2 + 2 * o] = __float2bfloat16(re);
        w[(2 * c + 1) * C2 + 2 * o] = __float2bfloat16(-im);
        w[(2 * c) * C2 + 2 * o + 1] = __float2bfloat16(im);
        w[(2 * c + 1) * C2 + 2 * o + 1] = __float2bfloat16(re);
    }
}

int grid_for(long long n, int block = 256)
{
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

// ------------------------------------------------------------------ context
struct surr_ctx {
    surr_dims d{};
    int MZ = 0, NM = 0, W2 = 0, Z2 = 0, H = 0;
    long long P = 0;
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    double T_init = 0.0, dt = 0.0;
    int steps = 0, heater = 0;
    // geometry copy for the solver
    std::vector<double> r_faces, z_faces, T_bc;
    std::vector<int> r_cells, z_cells, bc, box_region;
    std::vector<heat_box> boxes;
    std::vector<double> C_reg;
    int n_regions = 0;
    // parameter offsets
    size_t n_params = 0;
    size_t oP, opb, oQ1, oq1b, oQ2, oq2b;
    std::vector<size_t> oW, owb, oRre, oRim;
    // device state
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int adam_t = 0;
    bf16 *Wb = nullptr, *Q1b = nullptr, *Q2b = nullptr, *Wblk = nullptr;  // BF16 working copies
    bf16 *Fr = nullptr, *Gr = nullptr, *Fz = nullptr;                      // DFT tables
    float *rn = nullptr, *zn = nullptr;
    signed char *d_reg = nullptr;  // [Nz][Nr] region of each cell, -1 on void
    double *d_params = nullptr, *d_loss = nullptr;
    // workspace (max_batch samples)
    bf16 *act = nullptr;       // (L+1) x [B][C][P]
    float *pre = nullptr;      // L x [B][C][P]
    float *S = nullptr;        // [B][C][P] (also the spectral adjoint in backward)
    bf16 *A1 = nullptr, *A3 = nullptr;   // [B C Nz][2mr]
    float *P2 = nullptr;       // [B C][2MZ][2mr]
    bf16 *Yh = nullptr;        // [B C][2MZ][2mr]
    bf16 *Xm = nullptr;        // L x [NM][B][2C]
    float *Ym = nullptr;       // [NM][B][2C]
    bf16 *Ymb = nullptr;       // [NM][B][2C]
    float *hpre = nullptr;     // [B][H][P]
    bf16 *h = nullptr;         // [B][H][P]
    float *Tout = nullptr;     // [B][P]
    float *Ttrue = nullptr;    // [B][P]
    bf16 *gu = nullptr;        // [B][2][P]
    bf16 *dp0 = nullptr, *dp1 = nullptr;  // [B][max(H,C)][P]
    float *dv0 = nullptr;      // [B][C][P]
    float *part = nullptr;     // split-K partials
    float *dWblk = nullptr;    // [NM][2C][2C]
    int *d_idx = nullptr;      // [max_batch] minibatch sample indices (surr_train)
    double *d_err = nullptr;   // [2 max_batch] per-sample error maxima (surr_errors)
    size_t part_n = 0;
};

namespace {

void free_surr(surr_ctx *s)
{
    if (!s) return;
    void *bufs[] = {s->w,  s->g,  s->m,    s->v,    s->Wb,   s->Q1b,  s->Q2b, s->Wblk, s->Fr,   s->Gr,
                    s->Fz, s->rn, s->zn,   s->d_params, s->d_loss, s->act, s->pre, s->S,  s->A1,  s->A3,
                    s->P2, s->Yh, s->Xm,   s->Ym,   s->Ymb,  s->hpre, s->h,   s->Tout, s->Ttrue, s->gu,
                    s->dp0, s->dp1, s->dv0, s->part, s->dWblk, s->d_idx, s->d_err, s->d_reg};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete s;
}

template <typename T>
cudaError_t dalloc(T *&p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T));
}

cudaError_t refresh(surr_ctx *s)
{
    const int C = s->d.C;
    for (int l = 0; l < s->d.L; ++l) {
        cast_kernel<<<grid_for(C * C), 256, 0, s->stream>>>(s->w + s->oW[l], (long long)C * C, s->Wb + (size_t)l * C * C);
        wblk_kernel<<<grid_for((long long)s->NM * C * C), 256, 0, s->stream>>>(
            s->w + s->oRre[l], s->w + s->oRim[l], s->NM, C, s->Wblk + (size_t)l * s->NM * 4 * C * C);
    }
    cast_kernel<<<grid_for(s->H * C), 256, 0, s->stream>>>(s->w + s->oQ1, (long long)s->H * C, s->Q1b);
    cast_kernel<<<grid_for(2 * s->H), 256, 0, s->stream>>>(s->w + s->oQ2, 2LL * s->H, s->Q2b);
    return cudaGetLastError();
}

// Forward of B <= max_batch samples whose params are in d_params.
// train: keep pre-activations and the hidden head input for backward.
cudaError_t forward_chunk(surr_ctx *s, int B, bool train, const float *Ttrue, float *T)
{
    const surr_dims &d = s->d;
    const int C = d.C, Nz = d.Nz, Nr = d.Nr, W2 = s->W2, Z2 = s->Z2, NM = s->NM, H = s->H;
    const long long P = s->P, CP = (long long)C * P;
    const long long actsz = (long long)s->max_batch * CP;
    cudaStream_t st = s->stream;
    cudaError_t e;
    lift_kernel<<<dim3((unsigned)((P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024), B), 256, 0, st>>>(
        s->d_params, s->rn, s->zn, s->d_reg, s->heater, B, Nz, Nr, C, s->w + s->oP, s->w + s->opb, s->act);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = 0; l < d.L; ++l) {
        const bf16 *vl = s->act + (train ? l : (l & 1)) * actsz;
        bf16 *vn = s->act + (train ? l + 1 : ((l + 1) & 1)) * actsz;
        bf16 *Xm = s->Xm + (train ? (size_t)l * NM * s->max_batch * 2 * C : 0);
        GemmArgs g;
        // A1 = v Fr^T
        g = GemmArgs();
        g.M = B * C * Nz; g.N = W2; g.K = Nr;
        g.A = vl; g.lda = Nr;
        g.B = s->Fr; g.ldb = Nr; g.transB = 1;
        g.Cb = s->A1; g.ldc = W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // P2 = Fz A1
        g = GemmArgs();
        g.M = Z2; g.N = W2; g.K = Nz;
        g.A = s->Fz; g.lda = Nz;
        g.B = s->A1; g.ldb = W2; g.sB1 = (long long)Nz * W2;
        g.batch = B * C;
        g.Cf = s->P2; g.ldc = W2; g.sC1 = (long long)Z2 * W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        mix_in_kernel<<<grid_for((long long)B * C * NM), 256, 0, st>>>(s->P2, B, C, s->MZ, d.mr, Xm);
        // Y = X Wblk per mode
        g = GemmArgs();
        g.M = B; g.N = 2 * C; g.K = 2 * C;
        g.A = Xm; g.lda = 2 * C; g.sA1 = (long long)B * 2 * C;
        g.B = s->Wblk + (size_t)l * NM * 4 * C * C; g.ldb = 2 * C; g.sB1 = 4LL * C * C;
        g.batch = NM;
        g.Cf = s->Ym; g.ldc = 2 * C; g.sC1 = (long long)B * 2 * C;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        mix_out_kernel<<<grid_for((long long)B * C * NM), 256, 0, st>>>(s->Ym, B, C, s->MZ, d.mr, s->Yh);
        // A3 = Fz^T Yh
        g = GemmArgs();
        g.M = Nz; g.N = W2; g.K = Z2;
        g.A = s->Fz; g.lda = Nz; g.transA = 1;
        g.B = s->Yh; g.ldb = W2; g.sB1 = (long long)Z2 * W2;
        g.batch = B * C;
        g.Cb = s->A3; g.ldc = W2; g.sC1 = (long long)Nz * W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // S = A3 Gr
        g = GemmArgs();
        g.M = B * C * Nz; g.N = Nr; g.K = W2;
        g.A = s->A3; g.lda = W2;
        g.B = s->Gr; g.ldb = Nr;
        g.Cf = s->S; g.ldc = Nr;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // pre = W v + wb + S; v_{l+1} = gelu(pre) (not on the last layer)
        g = GemmArgs();
        g.M = C; g.N = (int)P; g.K = C;
        g.A = s->Wb + (size_t)l * C * C; g.lda = C;
        g.B = vl; g.ldb = P; g.sB1 = CP;
        g.batch = B;
        g.bias_m = s->w + s->owb[l];
        g.add = s->S;
        g.pre = train ? s->pre + (size_t)l * actsz : nullptr;
        g.act = l < d.L - 1 ? fno::ACT_GELU : fno::ACT_NONE;
        g.Cb = vn; g.ldc = P; g.sC1 = CP;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
    }
    const bf16 *vL = s->act + (train ? d.L : (d.L & 1)) * actsz;
    GemmArgs g;
    g.M = H; g.N = (int)P; g.K = C;
    g.A = s->Q1b; g.lda = C;
    g.B = vL; g.ldb = P; g.sB1 = CP;
    g.batch = B;
    g.bias_m = s->w + s->oq1b;
    g.pre = train ? s->hpre : nullptr;
    g.act = fno::ACT_GELU;
    g.Cb = s->h; g.ldc = P; g.sC1 = (long long)H * P;
    if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
    head_kernel<<<grid_for(B * P), 256, 0, st>>>(s->h, s->d_params, B, P, H, s->w + s->oQ2, s->w + s->oq2b, s->T_init,
                                                 s->d_reg, T, Ttrue, 1.0 / ((double)B * P), s->gu, s->d_loss);
    return cudaGetLastError();
}

// Split-K weight gradient: out (+)= sum_b A[b] [M x P] B[b]^T, A and B both
// [.][rows][P] BF16 with per-sample strides.
cudaError_t wgrad(surr_ctx *s, int B, int M, int N, const bf16 *A, long long sA, const bf16 *Bm, long long sB,
                  float *out)
{
    const long long P = s->P;
    const int chunk = (int)(P / kSplit);
    GemmArgs g;
    g.M = M; g.N = N; g.K = chunk;
    g.A = A; g.lda = P; g.sA1 = sA; g.sA2 = chunk;
    g.B = Bm; g.ldb = P; g.transB = 1; g.sB1 = sB; g.sB2 = chunk;
    g.batch = B * kSplit; g.nb2 = kSplit;
    g.Cf = s->part; g.ldc = N; g.sC1 = (long long)kSplit * M * N; g.sC2 = (long long)M * N;
    cudaError_t e = fno::gemm(g, s->stream);
    if (e != cudaSuccess) return e;
    reduce_parts_kernel<<<grid_for(M * N), 256, 0, s->stream>>>(s->part, B * kSplit, M * N, out);
    return cudaGetLastError();
}

cudaError_t backward_chunk(surr_ctx *s, int B)
{
    const surr_dims &d = s->d;
    const int C = d.C, Nz = d.Nz, Nr = d.Nr, W2 = s->W2, Z2 = s->Z2, NM = s->NM, H = s->H;
    const long long P = s->P, CP = (long long)C * P, HP = (long long)H * P;
    const long long actsz = (long long)s->max_batch * CP;
    cudaStream_t st = s->stream;
    float *gw = s->g;
    cudaError_t e;
    const int rs_chunks = 64;
    // head
    if ((e = wgrad(s, B, 2, H, s->gu, 2 * P, s->h, HP, gw + s->oQ2)) != cudaSuccess) return e;
    rowsum_kernel<<<dim3(rs_chunks, 2), 256, 0, st>>>(s->gu, B, 2, P, gw + s->oq2b);
    GemmArgs g;
    g.M = H; g.N = (int)P; g.K = 2;
    g.A = s->Q2b; g.lda = H; g.transA = 1;
    g.B = s->gu; g.ldb = P; g.sB1 = 2 * P;
    g.batch = B;
    g.act = fno::ACT_GELU_GRAD; g.aux = s->hpre;
    g.Cb = s->dp0; g.ldc = P; g.sC1 = HP;
    if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
    const bf16 *vL = s->act + (size_t)d.L * actsz;
    if ((e = wgrad(s, B, H, C, s->dp0, HP, vL, CP, gw + s->oQ1)) != cudaSuccess) return e;
    rowsum_kernel<<<dim3(rs_chunks, H), 256, 0, st>>>(s->dp0, B, H, P, gw + s->oq1b);
    // dv_L = Q1^T ghpre (the last layer has no activation: this is dpre_{L-1})
    g = GemmArgs();
    g.M = C; g.N = (int)P; g.K = H;
    g.A = s->Q1b; g.lda = C; g.transA = 1;
    g.B = s->dp0; g.ldb = P; g.sB1 = HP;
    g.batch = B;
    g.Cb = s->dp1; g.ldc = P; g.sC1 = CP;
    if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
    bf16 *dpre = s->dp1, *dnext = s->dp0;
    for (int l = d.L - 1; l >= 0; --l) {
        const bf16 *vl = s->act + (size_t)l * actsz;
        const bf16 *Xm = s->Xm + (size_t)l * NM * s->max_batch * 2 * C;
        const bf16 *Wbl = s->Wblk + (size_t)l * NM * 4 * C * C;
        if ((e = wgrad(s, B, C, C, dpre, CP, vl, CP, gw + s->oW[l])) != cudaSuccess) return e;
        rowsum_kernel<<<dim3(rs_chunks, C), 256, 0, st>>>(dpre, B, C, P, gw + s->owb[l]);
        // gA3 = dpre Gr^T
        g = GemmArgs();
        g.M = B * C * Nz; g.N = W2; g.K = Nr;
        g.A = dpre; g.lda = Nr;
        g.B = s->Gr; g.ldb = Nr; g.transB = 1;
        g.Cb = s->A3; g.ldc = W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // gYh = Fz gA3
        g = GemmArgs();
        g.M = Z2; g.N = W2; g.K = Nz;
        g.A = s->Fz; g.lda = Nz;
        g.B = s->A3; g.ldb = W2; g.sB1 = (long long)Nz * W2;
        g.batch = B * C;
        g.Cf = s->P2; g.ldc = W2; g.sC1 = (long long)Z2 * W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        mix_out_bwd_kernel<<<grid_for((long long)B * C * NM), 256, 0, st>>>(s->P2, B, C, s->MZ, d.mr, s->Ymb);
        // dWblk = X^T gY per mode
        g = GemmArgs();
        g.M = 2 * C; g.N = 2 * C; g.K = B;
        g.A = Xm; g.lda = 2 * C; g.transA = 1; g.sA1 = (long long)B * 2 * C;
        g.B = s->Ymb; g.ldb = 2 * C; g.sB1 = (long long)B * 2 * C;
        g.batch = NM;
        g.Cf = s->dWblk; g.ldc = 2 * C; g.sC1 = 4LL * C * C;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        wblk_grad_kernel<<<grid_for((long long)NM * C * C), 256, 0, st>>>(s->dWblk, NM, C, gw + s->oRre[l],
                                                                          gw + s->oRim[l]);
        // gX = gY Wblk^T
        g = GemmArgs();
        g.M = B; g.N = 2 * C; g.K = 2 * C;
        g.A = s->Ymb; g.lda = 2 * C; g.sA1 = (long long)B * 2 * C;
        g.B = Wbl; g.ldb = 2 * C; g.transB = 1; g.sB1 = 4LL * C * C;
        g.batch = NM;
        g.Cf = s->Ym; g.ldc = 2 * C; g.sC1 = (long long)B * 2 * C;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        mix_in_bwd_kernel<<<grid_for((long long)B * C * NM), 256, 0, st>>>(s->Ym, B, C, s->MZ, d.mr, s->Yh);
        // gA1 = Fz^T gP2
        g = GemmArgs();
        g.M = Nz; g.N = W2; g.K = Z2;
        g.A = s->Fz; g.lda = Nz; g.transA = 1;
        g.B = s->Yh; g.ldb = W2; g.sB1 = (long long)Z2 * W2;
        g.batch = B * C;
        g.Cb = s->A1; g.ldc = W2; g.sC1 = (long long)Nz * W2;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // spectral part of dv_l: gA1 Fr
        g = GemmArgs();
        g.M = B * C * Nz; g.N = Nr; g.K = W2;
        g.A = s->A1; g.lda = W2;
        g.B = s->Fr; g.ldb = Nr;
        g.Cf = s->S; g.ldc = Nr;
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        // dv_l = W^T dpre + spectral part; times gelu'(pre_{l-1}) below layer 0
        g = GemmArgs();
        g.M = C; g.N = (int)P; g.K = C;
        g.A = s->Wb + (size_t)l * C * C; g.lda = C; g.transA = 1;
        g.B = dpre; g.ldb = P; g.sB1 = CP;
        g.batch = B;
        g.add = s->S;
        g.ldc = P; g.sC1 = CP;
        if (l > 0) {
            g.act = fno::ACT_GELU_GRAD;
            g.aux = s->pre + (size_t)(l - 1) * actsz;
            g.Cb = dnext;
        } else {
            g.Cf = s->dv0;
        }
        if ((e = fno::gemm(g, st)) != cudaSuccess) return e;
        bf16 *t = dpre;
        dpre = dnext;
        dnext = t;
    }
    lift_bwd_kernel<<<dim3(C, B), 256, 0, st>>>(s->d_params, s->rn, s->zn, s->d_reg, s->heater, B, Nz, Nr, C,
                                               s->dv0, gw + s->oP, gw + s->opb);
    return cudaGetLastError();
}

int upload_params(surr_ctx *s, const double *params, int B)
{
    SURR_TRY(cudaMemcpyAsync(s->d_params, params, (size_t)B * 7 * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    return HEAT_OK;
}

bool params_ok(const double *p, int B)
{
    for (int b = 0; b < B; ++b) {
        for (int m = 0; m < 5; ++m)
            if (!(p[7 * b + m] > 0.0) || !std::isfinite(p[7 * b + m])) return false;
        if (!(p[7 * b + 5] > 0.0) || !std::isfinite(p[7 * b + 5]) || !std::isfinite(p[7 * b + 6])) return false;
    }
    return true;
}

// Solver runs of B instances (FP32 batched path) -> T floats [B][Nz][Nr] (host or device).
int solve_batch(surr_ctx *s, const double *params, int B, float *T, int on_device)
{
    const int Nr = s->d.Nr, Nz = s->d.Nz;
    const size_t ncell = (size_t)Nr * Nz;
    const int chunk = 512;
    std::vector<double> kbuf, qbuf, Tbc;
    std::vector<heat_geometry> geoms;
    std::vector<heat_materials> mats;
    std::vector<double> field(ncell);
    std::vector<float> ffield(ncell);
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int n = B - b0 < chunk ? B - b0 : chunk;
        kbuf.assign((size_t)n * s->n_regions, 0.0);
        qbuf.assign((size_t)n * s->n_regions, 0.0);
        Tbc.assign((size_t)n * 4, 0.0);
        geoms.assign(n, heat_geometry());
        mats.assign(n, heat_materials());
        for (int i = 0; i < n; ++i) {
            const double *p = params + 7 * (size_t)(b0 + i);
            heat_geometry &g = geoms[i];
            g.n_r_layers = (int)s->r_cells.size();
            g.r_faces = s->r_faces.data();
            g.r_cells = s->r_cells.data();
            g.n_z_layers = (int)s->z_cells.size();
            g.z_faces = s->z_faces.data();
            g.z_cells = s->z_cells.data();
            g.n_boxes = (int)s->boxes.size();
            g.boxes = s->boxes.data();
            for (int f = 0; f < 4; ++f) {
                g.bc[f] = s->bc[f];
                g.T_bc[f] = s->bc[f] == HEAT_BC_DIRICHLET ? p[6] : s->T_bc[f];
            }
            double *k = &kbuf[(size_t)i * s->n_regions];
            double *q = &qbuf[(size_t)i * s->n_regions];
            for (int r = 0; r < s->n_regions; ++r) k[r] = p[r < 5 ? r : 4];
            q[s->heater] = p[5];
            heat_materials &m = mats[i];
            m.n_regions = s->n_regions;
            m.k = k;
            m.C = s->C_reg.data();
            m.q = q;
            m.T_init = s->T_init;
        }
        std::vector<double> dts(n, s->dt);
        heat_options opt{HEAT_FP32, HEAT_HARMONIC};
        heat_batch *hb = nullptr;
        int st = heat_batch_create(n, geoms.data(), mats.data(), &opt, dts.data(), s->stream, &hb);
        if (st != HEAT_OK) return st;
        st = heat_batch_step(hb, s->steps);
        if (st == HEAT_OK) st = heat_batch_sync(hb);
        for (int i = 0; i < n && st == HEAT_OK; ++i) {
            heat_ctx *c = nullptr;
            st = heat_batch_member(hb, i, &c);
            if (st != HEAT_OK) break;
            st = heat_field(c, field.data(), ncell, 0);
            if (st != HEAT_OK) break;
            for (size_t x = 0; x < ncell; ++x) ffield[x] = (float)field[x];
            float *dst = T + (size_t)(b0 + i) * ncell;
            if (on_device) {
                cudaError_t e = cudaMemcpyAsync(dst, ffield.data(), ncell * sizeof(float), cudaMemcpyHostToDevice,
                                                s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
                st = cuda_status(e);
            } else {
                std::memcpy(dst, ffield.data(), ncell * sizeof(float));
            }
        }
        heat_batch_destroy(hb);
        if (st != HEAT_OK) return st;
    }
    return HEAT_OK;
}

}  // namespace

extern "C" {

int surr_create(const surr_dims *dims, const heat_geometry *geom, const heat_materials *base, int heater_region,
                double dt, int steps, int max_batch, void *stream, surr_ctx **out)
{
    if (!out) return HEAT_ERR_ARG;
    *out = nullptr;
    if (!dims || !geom || !base || !(dt > 0.0) || steps < 0 || max_batch < 1 || max_batch > 65535) return HEAT_ERR_ARG;
    const surr_dims d = *dims;
    if (d.Nz < 2 || d.Nr < 2 || d.C < 1 || d.L < 1 || d.mz < 1 || d.mr < 1 || 2 * d.mz > d.Nz || 2 * d.mr >= d.Nr)
        return HEAT_ERR_ARG;
    if (((long long)d.Nz * d.Nr) % kSplit != 0) return HEAT_ERR_ARG;
    if (base->n_regions < 5 || heater_region < 0 || heater_region >= base->n_regions) return HEAT_ERR_ARG;
    // the grid's cell centres come from the solver's own grid builder
    heat_options opt{HEAT_FP64, HEAT_HARMONIC};
    heat_ctx *probe = nullptr;
    int st = heat_create(geom, base, &opt, dt, stream, &probe);
    if (st != HEAT_OK) return st;
    int Nr = 0, Nz = 0;
    std::vector<double> rc(d.Nr), zc(d.Nz);
    st = heat_info(probe, &Nr, &Nz, nullptr, nullptr, nullptr);
    if (st == HEAT_OK && (Nr != d.Nr || Nz != d.Nz)) st = HEAT_ERR_ARG;
    if (st == HEAT_OK) st = heat_info(probe, nullptr, nullptr, rc.data(), zc.data(), nullptr);
    heat_destroy(probe);
    if (st != HEAT_OK) return st;

    surr_ctx *s = new (std::nothrow) surr_ctx();
    if (!s) return HEAT_ERR_OOM;
    s->d = d;
    s->MZ = 2 * d.mz;
    s->NM = s->MZ * d.mr;
    s->W2 = 2 * d.mr;
    s->Z2 = 2 * s->MZ;
    s->H = 2 * d.C;
    s->P = (long long)d.Nz * d.Nr;
    s->max_batch = max_batch;
    s->stream = static_cast<cudaStream_t>(stream);
    s->T_init = base->T_init;
    s->dt = dt;
    s->steps = steps;
    s->heater = heater_region;
    s->r_faces.assign(geom->r_faces, geom->r_faces + geom->n_r_layers + 1);
    s->r_cells.assign(geom->r_cells, geom->r_cells + geom->n_r_layers);
    s->z_faces.assign(geom->z_faces, geom->z_faces + geom->n_z_layers + 1);
    s->z_cells.assign(geom->z_cells, geom->z_cells + geom->n_z_layers);
    s->boxes.assign(geom->boxes, geom->boxes + geom->n_boxes);
    s->bc.assign(geom->bc, geom->bc + 4);
    s->T_bc.assign(geom->T_bc, geom->T_bc + 4);
    s->n_regions = base->n_regions;
    s->C_reg.assign(base->C, base->C + base->n_regions);

    // parameter offsets (the order of include/surrogate.h)
    const int C = d.C, H = s->H;
    size_t o = 0;
    s->oP = o; o += (size_t)C * kF;
    s->opb = o; o += C;
    for (int l = 0; l < d.L; ++l) {
        s->oW.push_back(o); o += (size_t)C * C;
        s->owb.push_back(o); o += C;
        s->oRre.push_back(o); o += (size_t)s->NM * C * C;
        s->oRim.push_back(o); o += (size_t)s->NM * C * C;
    }
    s->oQ1 = o; o += (size_t)H * C;
    s->oq1b = o; o += H;
    s->oQ2 = o; o += 2 * (size_t)H;
    s->oq2b = o; o += 2;
    s->n_params = o;

    const size_t B = max_batch;
    const long long P = s->P;
    const size_t CP = (size_t)C * P;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(dalloc(s->w, o)); A(dalloc(s->g, o)); A(dalloc(s->m, o)); A(dalloc(s->v, o));
    A(dalloc(s->Wb, (size_t)d.L * C * C));
    A(dalloc(s->Wblk, (size_t)d.L * s->NM * 4 * C * C));
    A(dalloc(s->Q1b, (size_t)H * C));
    A(dalloc(s->Q2b, 2 * (size_t)H));
    A(dalloc(s->Fr, (size_t)s->W2 * d.Nr));
    A(dalloc(s->Gr, (size_t)s->W2 * d.Nr));
    A(dalloc(s->Fz, (size_t)s->Z2 * d.Nz));
    A(dalloc(s->rn, d.Nr));
    A(dalloc(s->d_reg, (size_t)d.Nz * d.Nr));
    A(dalloc(s->zn, d.Nz));
    A(dalloc(s->d_params, B * 7));
    A(dalloc(s->d_loss, 1));
    A(dalloc(s->act, (size_t)(d.L + 1) * B * CP));
    A(dalloc(s->pre, (size_t)d.L * B * CP));
    A(dalloc(s->S, B * CP));
    A(dalloc(s->A1, B * C * d.Nz * s->W2));
    A(dalloc(s->A3, B * C * d.Nz * s->W2));
    A(dalloc(s->P2, B * C * s->Z2 * s->W2));
    A(dalloc(s->Yh, B * C * s->Z2 * s->W2));
    A(dalloc(s->Xm, (size_t)d.L * s->NM * B * 2 * C));
    A(dalloc(s->Ym, (size_t)s->NM * B * 2 * C));
    A(dalloc(s->Ymb, (size_t)s->NM * B * 2 * C));
    A(dalloc(s->hpre, B * H * P));
    A(dalloc(s->h, B * H * P));
    A(dalloc(s->Tout, B * P));
    A(dalloc(s->Ttrue, B * P));
    A(dalloc(s->gu, B * 2 * P));
    A(dalloc(s->dp0, B * H * P));
    A(dalloc(s->dp1, B * H * P));
    A(dalloc(s->dv0, B * CP));
    s->part_n = B * kSplit * (size_t)H * (H > C ? H : C);
    A(dalloc(s->part, s->part_n));
    A(dalloc(s->dWblk, (size_t)s->NM * 4 * C * C));
    A(dalloc(s->d_idx, B));
    A(dalloc(s->d_err, 2 * B));
    if (e != cudaSuccess) {
        free_surr(s);
        return cuda_status(e);
    }
    // DFT tables and scaled coordinates (double precision angles)
    {
        const int Nr_ = d.Nr, Nz_ = d.Nz, mr = d.mr, W2 = s->W2, Z2 = s->Z2;
        std::vector<bf16> fr((size_t)W2 * Nr_), gr((size_t)W2 * Nr_), fz((size_t)Z2 * Nz_);
        const double N = (double)Nr_ * Nz_;
        for (int kr = 0; kr < mr; ++kr) {
            const double a = kr == 0 ? 1.0 : 2.0;
            for (int i = 0; i < Nr_; ++i) {
                const double th = 2.0 * kPiD * (double)((long long)kr * i % Nr_) / Nr_;
                fr[(size_t)(2 * kr) * Nr_ + i] = __float2bfloat16((float)std::cos(th));
                fr[(size_t)(2 * kr + 1) * Nr_ + i] = __float2bfloat16((float)(-std::sin(th)));
                gr[(size_t)(2 * kr) * Nr_ + i] = __float2bfloat16((float)(a * std::cos(th) / N));
                gr[(size_t)(2 * kr + 1) * Nr_ + i] = __float2bfloat16((float)(-a * std::sin(th) / N));
            }
        }
        for (int kzi = 0; kzi < s->MZ; ++kzi) {
            const int kz = kzi < d.mz ? kzi : Nz_ - s->MZ + kzi;
            for (int j = 0; j < Nz_; ++j) {
                const double th = 2.0 * kPiD * (double)((long long)kz * j % Nz_) / Nz_;
                fz[(size_t)(2 * kzi) * Nz_ + j] = __float2bfloat16((float)std::cos(th));
                fz[(size_t)(2 * kzi + 1) * Nz_ + j] = __float2bfloat16((float)std::sin(th));
            }
        }
        const double R = s->r_faces.back(), Z = s->z_faces.back();
        std::vector<float> rn(Nr_), zn(Nz_);
        for (int i = 0; i < Nr_; ++i) rn[i] = (float)(2.0 * rc[i] / R - 1.0);
        for (int j = 0; j < Nz_; ++j) zn[j] = (float)(2.0 * zc[j] / Z - 1.0);
        A(cudaMemcpyAsync(s->Fr, fr.data(), fr.size() * sizeof(bf16), cudaMemcpyHostToDevice, s->stream));
        A(cudaMemcpyAsync(s->Gr, gr.data(), gr.size() * sizeof(bf16), cudaMemcpyHostToDevice, s->stream));
        A(cudaMemcpyAsync(s->Fz, fz.data(), fz.size() * sizeof(bf16), cudaMemcpyHostToDevice, s->stream));
        A(cudaMemcpyAsync(s->rn, rn.data(), rn.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        // region of each cell: the first box that contains its centre (the
        // solver's rule), -1 on void
        std::vector<signed char> reg((size_t)Nz_ * Nr_, (signed char)-1);
        for (int j = 0; j < Nz_; ++j)
            for (int i = 0; i < Nr_; ++i)
                for (size_t b = 0; b < s->boxes.size(); ++b) {
                    const heat_box &bx = s->boxes[b];
                    if (rc[i] >= bx.r0 && rc[i] <= bx.r1 && zc[j] >= bx.z0 && zc[j] <= bx.z1) {
                        const int r = bx.region;
                        reg[(size_t)j * Nr_ + i] = (signed char)(r >= 0 && r < s->n_regions ? r : -1);
                        break;
                    }
                }
        A(cudaMemcpyAsync(s->d_reg, reg.data(), reg.size(), cudaMemcpyHostToDevice, s->stream));
        A(cudaMemcpyAsync(s->zn, zn.data(), zn.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        A(cudaMemsetAsync(s->w, 0, o * sizeof(float), s->stream));
        A(cudaMemsetAsync(s->m, 0, o * sizeof(float), s->stream));
        A(cudaMemsetAsync(s->v, 0, o * sizeof(float), s->stream));
        A(cudaStreamSynchronize(s->stream));
    }
    if (e == cudaSuccess) e = refresh(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        free_surr(s);
        return cuda_status(e);
    }
    *out = s;
    return HEAT_OK;
}

size_t surr_n_params(const surr_ctx *s) { return s ? s->n_params : 0; }

int surr_set_params(surr_ctx *s, const float *flat, size_t n, int on_device)
{
    if (!s || !flat || n != s->n_params) return HEAT_ERR_ARG;
    SURR_TRY(cudaMemcpyAsync(s->w, flat, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s->stream));
    SURR_TRY(cudaMemsetAsync(s->m, 0, n * sizeof(float), s->stream));
    SURR_TRY(cudaMemsetAsync(s->v, 0, n * sizeof(float), s->stream));
    s->adam_t = 0;
    SURR_TRY(refresh(s));
    SURR_TRY(cudaStreamSynchronize(s->stream));
    return HEAT_OK;
}

int surr_get_params(surr_ctx *s, float *flat, size_t n, int on_device)
{
    if (!s || !flat || n != s->n_params) return HEAT_ERR_ARG;
    SURR_TRY(cudaMemcpyAsync(flat, s->w, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             s->stream));
    SURR_TRY(cudaStreamSynchronize(s->stream));
    return HEAT_OK;
}

int surr_forward(surr_ctx *s, const double *params, int B, float *T, int on_device)
{
    if (!s || !params || !T || B < 0) return HEAT_ERR_ARG;
    if (!params_ok(params, B)) return HEAT_ERR_ARG;
    const size_t ncell = (size_t)s->P;
    for (int b0 = 0; b0 < B; b0 += s->max_batch) {
        const int n = B - b0 < s->max_batch ? B - b0 : s->max_batch;
        int st = upload_params(s, params + 7 * (size_t)b0, n);
        if (st != HEAT_OK) return st;
        float *dst = on_device ? T + (size_t)b0 * ncell : s->Tout;
        SURR_TRY(forward_chunk(s, n, false, nullptr, dst));
        if (!on_device) {
            SURR_TRY(cudaMemcpyAsync(T + (size_t)b0 * ncell, s->Tout, (size_t)n * ncell * sizeof(float),
                                     cudaMemcpyDeviceToHost, s->stream));
        }
    }
    SURR_TRY(cudaStreamSynchronize(s->stream));
    return HEAT_OK;
}

int surr_loss_grad(surr_ctx *s, const double *params, int B, const float *T_true, int true_on_device, double *loss,
                   float *grad, int grad_on_device)
{
    if (!s || !params || !T_true || B < 1 || B > s->max_batch) return HEAT_ERR_ARG;
    if (!params_ok(params, B)) return HEAT_ERR_ARG;
    int st = upload_params(s, params, B);
    if (st != HEAT_OK) return st;
    const float *Tt = T_true;
    if (!true_on_device) {
        SURR_TRY(cudaMemcpyAsync(s->Ttrue, T_true, (size_t)B * s->P * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        Tt = s->Ttrue;
    }
    SURR_TRY(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    SURR_TRY(cudaMemsetAsync(s->g, 0, s->n_params * sizeof(float), s->stream));
    SURR_TRY(forward_chunk(s, B, true, Tt, s->Tout));
    SURR_TRY(backward_chunk(s, B));
    double l = 0.0;
    SURR_TRY(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (grad)
        SURR_TRY(cudaMemcpyAsync(grad, s->g, s->n_params * sizeof(float),
                                 grad_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    SURR_TRY(cudaStreamSynchronize(s->stream));
    if (loss) *loss = l / ((double)B * s->P);
    return std::isfinite(l) ? HEAT_OK : HEAT_ERR_NONFINITE;
}

int surr_adam(surr_ctx *s, double lr, double beta1, double beta2, double eps)
{
    if (!s || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0))
        return HEAT_ERR_ARG;
    s->adam_t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(beta1, s->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(beta2, s->adam_t)));
    adam_kernel<<<grid_for((long long)s->n_params), 256, 0, s->stream>>>((long long)s->n_params, s->w, s->g, s->m, s->v,
                                                                         (float)lr, (float)beta1, (float)beta2,
                                                                         (float)eps, c1, c2);
    SURR_TRY(cudaGetLastError());
    SURR_TRY(refresh(s));
    return HEAT_OK;
}

int surr_solve(surr_ctx *s, const double *params, int B, float *T, int on_device)
{
    if (!s || !params || !T || B < 0) return HEAT_ERR_ARG;
    if (!params_ok(params, B)) return HEAT_ERR_ARG;
    return solve_batch(s, params, B, T, on_device);
}

int surr_infer_checked(surr_ctx *s, const double *params, int B, int n_check, double tol, unsigned seed, float *T,
                       int on_device, int *used_fallback, double *max_err)
{
    if (!s || !params || !T || B < 1 || n_check < 0 || n_check > B || !(tol > 0.0)) return HEAT_ERR_ARG;
    int st = surr_forward(s, params, B, T, on_device);
    if (st != HEAT_OK) return st;
    const size_t ncell = (size_t)s->P;
    std::vector<double> cp((size_t)n_check * 7);
    std::vector<size_t> idx(n_check);
    for (int i = 0; i < n_check; ++i) {
        idx[i] = (size_t)(((unsigned long long)seed + (unsigned long long)i * B / n_check) % B);
        std::memcpy(&cp[(size_t)i * 7], params + 7 * idx[i], 7 * sizeof(double));
    }
    std::vector<float> ref((size_t)n_check * ncell), net(ncell);
    if (n_check > 0 && (st = solve_batch(s, cp.data(), n_check, ref.data(), 0)) != HEAT_OK) return st;
    double worst = 0.0;
    for (int i = 0; i < n_check; ++i) {
        if (on_device) {
            SURR_TRY(cudaMemcpyAsync(net.data(), T + idx[i] * ncell, ncell * sizeof(float), cudaMemcpyDeviceToHost,
                                     s->stream));
            SURR_TRY(cudaStreamSynchronize(s->stream));
        } else {
            std::memcpy(net.data(), T + idx[i] * ncell, ncell * sizeof(float));
        }
        double emax = 0.0, rise = 0.0;
        const float *r = &ref[(size_t)i * ncell];
        for (size_t x = 0; x < ncell; ++x) {
            emax = std::fmax(emax, std::fabs((double)net[x] - (double)r[x]));
            rise = std::fmax(rise, std::fabs((double)r[x] - s->T_init));
        }
        const double err = rise > 0.0 ? emax / rise : (emax > 0.0 ? INFINITY : 0.0);
        worst = std::fmax(worst, err);
    }
    if (max_err) *max_err = worst;
    const int fb = worst > tol ? 1 : 0;
    if (used_fallback) *used_fallback = fb;
    if (fb) return solve_batch(s, params, B, T, on_device);
    return HEAT_OK;
}

int surr_train(surr_ctx *s, const double *params, int n, const float *T_true, int epochs, int batch, double lr0,
               double lr_min_frac, unsigned seed, double *last_epoch_loss)
{
    if (!s || !params || !T_true || n < 1 || epochs < 1 || batch < 1 || batch > s->max_batch || !(lr0 > 0.0) ||
        !(lr_min_frac >= 0.0 && lr_min_frac <= 1.0))
        return HEAT_ERR_ARG;
    if (!params_ok(params, n)) return HEAT_ERR_ARG;
    const long long P = s->P;
    const int per_epoch = (n + batch - 1) / batch;
    const double total = (double)epochs * per_epoch;
    std::vector<int> perm(n), idx(batch);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::vector<double> hp((size_t)batch * 7);
    // splitmix64 stream for the per-epoch shuffles
    unsigned long long state = 0x9e3779b97f4a7c15ULL * ((unsigned long long)seed + 1ULL);
    auto next = [&]() {
        unsigned long long z = (state += 0x9e3779b97f4a7c15ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        return z ^ (z >> 31);
    };
    double epoch_loss = 0.0;
    long long step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n - 1; i > 0; --i) {
            const int k = (int)(next() % (unsigned long long)(i + 1));
            const int t = perm[i];
            perm[i] = perm[k];
            perm[k] = t;
        }
        SURR_TRY(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int B = n - b0 < batch ? n - b0 : batch;
            for (int b = 0; b < B; ++b) {
                idx[b] = perm[b0 + b];
                std::memcpy(&hp[(size_t)b * 7], params + 7 * (size_t)idx[b], 7 * sizeof(double));
            }
            SURR_TRY(cudaMemcpyAsync(s->d_params, hp.data(), (size_t)B * 7 * sizeof(double), cudaMemcpyHostToDevice,
                                     s->stream));
            SURR_TRY(cudaMemcpyAsync(s->d_idx, idx.data(), (size_t)B * sizeof(int), cudaMemcpyHostToDevice, s->stream));
            gather_rows_kernel<<<grid_for((long long)B * P), 256, 0, s->stream>>>(T_true, s->d_idx, B, P, s->Ttrue);
            SURR_TRY(cudaGetLastError());
            SURR_TRY(cudaMemsetAsync(s->g, 0, s->n_params * sizeof(float), s->stream));
            SURR_TRY(forward_chunk(s, B, true, s->Ttrue, s->Tout));
            SURR_TRY(backward_chunk(s, B));
            const double lr = lr0 * (lr_min_frac + (1.0 - lr_min_frac) * 0.5 * (1.0 + std::cos(kPiD * step / total)));
            s->adam_t += 1;
            const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, s->adam_t)));
            const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, s->adam_t)));
            adam_kernel<<<grid_for((long long)s->n_params), 256, 0, s->stream>>>(
                (long long)s->n_params, s->w, s->g, s->m, s->v, (float)lr, 0.9f, 0.999f, 1e-8f, c1, c2);
            SURR_TRY(cudaGetLastError());
            SURR_TRY(refresh(s));
            ++step;
        }
        double l = 0.0;
        SURR_TRY(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        SURR_TRY(cudaStreamSynchronize(s->stream));
        // each minibatch adds its squared-error sum scaled by 1 (head_kernel), so the mean is over all cells
        epoch_loss = l / ((double)n * P);
        if (!std::isfinite(epoch_loss)) return HEAT_ERR_NONFINITE;
    }
    if (last_epoch_loss) *last_epoch_loss = epoch_loss;
    return HEAT_OK;
}

int surr_errors(surr_ctx *s, const double *params, int B, const float *T_true, int true_on_device, double *errs)
{
    if (!s || !params || !T_true || !errs || B < 1) return HEAT_ERR_ARG;
    if (!params_ok(params, B)) return HEAT_ERR_ARG;
    const long long P = s->P;
    std::vector<double> e2((size_t)2 * s->max_batch);
    for (int b0 = 0; b0 < B; b0 += s->max_batch) {
        const int n = B - b0 < s->max_batch ? B - b0 : s->max_batch;
        int st = upload_params(s, params + 7 * (size_t)b0, n);
        if (st != HEAT_OK) return st;
        const float *Tt = T_true + (size_t)b0 * P;
        if (!true_on_device) {
            SURR_TRY(cudaMemcpyAsync(s->Ttrue, Tt, (size_t)n * P * sizeof(float), cudaMemcpyHostToDevice, s->stream));
            Tt = s->Ttrue;
        }
        SURR_TRY(forward_chunk(s, n, false, nullptr, s->Tout));
        err_kernel<<<n, 256, 0, s->stream>>>(s->Tout, Tt, P, s->T_init, s->d_err);
        SURR_TRY(cudaGetLastError());
        SURR_TRY(cudaMemcpyAsync(e2.data(), s->d_err, (size_t)2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                                 s->stream));
        SURR_TRY(cudaStreamSynchronize(s->stream));
        for (int b = 0; b < n; ++b)
            errs[b0 + b] = e2[2 * b + 1] > 0.0 ? e2[2 * b] / e2[2 * b + 1] : (e2[2 * b] > 0.0 ? INFINITY : 0.0);
    }
    return HEAT_OK;
}

void surr_destroy(surr_ctx *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_surr(s);
}

}  // extern "C"
