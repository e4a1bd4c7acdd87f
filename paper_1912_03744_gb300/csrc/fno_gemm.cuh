// fno_gemm.cuh -- BF16 tensor-core GEMM with FP32 accumulation for the
// surrogate (mma.sync m16n8k16, sm_103a), with the epilogues the network's
// forward and backward passes need.
//
//   C[z] = alpha op(A)[z] op(B)[z] (+ beta C[z]) (+ bias) (+ D[z]), then an
//   optional activation, stored as FP32 and/or BF16.
//   op(A) is M x K: transA = 0 reads A[m lda + k], transA = 1 reads A[k lda + m].
//   op(B) is K x N: transB = 0 reads B[k ldb + n], transB = 1 reads B[n ldb + k].
//   C, D, pre, aux are row-major M x N with leading dimension ldc.
// Batch index z = z1 nb2 + z2 (two-level strides, so a batch can also split
// the K range: split-K partial products land in separate C slices).
// Block tile 64 x 64 x 32, 4 warps of 32 x 32; operands staged in padded
// shared memory (row stride 40 bf16, conflict-free fragment loads); 16-byte
// global loads along the contiguous dimension where aligned and in range.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace fno {

using bf16 = __nv_bfloat16;

enum { ACT_NONE = 0, ACT_GELU = 1, ACT_GELU_GRAD = 2 };

struct GemmArgs {
    int M = 0, N = 0, K = 0;
    const bf16 *A = nullptr;
    long long lda = 0, sA1 = 0, sA2 = 0;
    int transA = 0;
    const bf16 *B = nullptr;
    long long ldb = 0, sB1 = 0, sB2 = 0;
    int transB = 0;
    int batch = 1, nb2 = 1;
    float alpha = 1.f, beta = 0.f;
    float *Cf = nullptr;           // FP32 output (also read when beta != 0)
    bf16 *Cb = nullptr;            // BF16 output
    long long ldc = 0, sC1 = 0, sC2 = 0;
    const float *bias_m = nullptr; // + bias_m[row]
    const float *bias_n = nullptr; // + bias_n[col]
    const float *add = nullptr;    // + add[off] (C's layout)
    float *pre = nullptr;          // pre-activation store (C's layout)
    const float *aux = nullptr;    // ACT_GELU_GRAD: multiply by gelu'(aux[off])
    int act = ACT_NONE;
};

__device__ __forceinline__ float gelu_f(float x)
{
    const float c = 0.7978845608028654f;  // sqrt(2/pi)
    return 0.5f * x * (1.f + tanhf(c * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad_f(float x)
{
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (x + 0.044715f * x * x * x));
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * x * x);
}

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8, GLD = GBK + GPAD;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage rows [r0, r0+64) x k [k0, k0+32) of a row-major-in-k operand (element
// (r, k) at P[r ld + k]) into S[r][k].
__device__ __forceinline__ void stage_kmajor(bf16 (*S)[GLD], const bf16 *__restrict__ P, long long ld, int R,
                                             int K, int r0, int k0)
{
    const bf16 zero = __float2bfloat16(0.f);
    for (int c = threadIdx.x; c < 64 * 4; c += blockDim.x) {
        const int r = c >> 2, kk = (c & 3) * 8;
        const int gr = r0 + r, gk = k0 + kk;
        const bf16 *src = P + (long long)gr * ld + gk;
        if (gr < R && gk + 8 <= K && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            *reinterpret_cast<uint4 *>(&S[r][kk]) = *reinterpret_cast<const uint4 *>(src);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) S[r][kk + e] = (gr < R && gk + e < K) ? src[e] : zero;
        }
    }
}

// Stage rows [r0, r0+64) x k [k0, k0+32) of an operand stored k-major-outer
// (element (r, k) at P[k ld + r]) into S[r][k].
__device__ __forceinline__ void stage_rmajor(bf16 (*S)[GLD], const bf16 *__restrict__ P, long long ld, int R,
                                             int K, int r0, int k0)
{
    const bf16 zero = __float2bfloat16(0.f);
    for (int c = threadIdx.x; c < 32 * 8; c += blockDim.x) {
        const int k = c >> 3, rr = (c & 7) * 8;
        const int gk = k0 + k, gr = r0 + rr;
        const bf16 *src = P + (long long)gk * ld + gr;
        if (gk < K && gr + 8 <= R && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            uint4 v = *reinterpret_cast<const uint4 *>(src);
            const bf16 *e8 = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int e = 0; e < 8; ++e) S[rr + e][k] = e8[e];
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) S[rr + e][k] = (gk < K && gr + e < R) ? src[e] : zero;
        }
    }
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(16) bf16 As[GBM][GLD];
    __shared__ __align__(16) bf16 Bs[GBN][GLD];
    const int z = blockIdx.z;
    const int z1 = z / g.nb2, z2 = z - z1 * g.nb2;
    const bf16 *A = g.A + z1 * g.sA1 + z2 * g.sA2;
    const bf16 *B = g.B + z1 * g.sB1 + z2 * g.sB2;
    const long long cofs = z1 * g.sC1 + z2 * g.sC2;
    const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    for (int k0 = 0; k0 < g.K; k0 += GBK) {
        if (g.transA) stage_rmajor(As, A, g.lda, g.M, g.K, m0, k0);
        else stage_kmajor(As, A, g.lda, g.M, g.K, m0, k0);
        if (g.transB) stage_kmajor(Bs, B, g.ldb, g.N, g.K, n0, k0);
        else stage_rmajor(Bs, B, g.ldb, g.N, g.K, n0, k0);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + gq;
                a[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tq * 2]);
                a[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tq * 2]);
                a[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tq * 2 + 8]);
                a[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tq * 2 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cidx = wn * 32 + j * 8 + gq;
                b[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][ks + tq * 2]);
                b[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][ks + tq * 2 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + wm * 32 + i * 16 + gq + (e >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + j * 8 + tq * 2 + (e & 1);
                if (row >= g.M || col >= g.N) continue;
                const long long off = cofs + (long long)row * g.ldc + col;
                float v = g.alpha * acc[i][j][e];
                if (g.beta != 0.f) v += g.beta * g.Cf[off];
                if (g.bias_m) v += g.bias_m[row];
                if (g.bias_n) v += g.bias_n[col];
                if (g.add) v += g.add[off];
                if (g.pre) g.pre[off] = v;
                if (g.act == ACT_GELU) v = gelu_f(v);
                else if (g.act == ACT_GELU_GRAD) v *= gelu_grad_f(g.aux[off]);
                if (g.Cf) g.Cf[off] = v;
                if (g.Cb) g.Cb[off] = __float2bfloat16(v);
            }
}

// The network's pointwise products: M and K at most 64 (the channel counts),
// N the pixels of a sample (long, contiguous in B and C: transB = 0).  As a
// tiled GEMM the M x K operand half-fills a 64 x 64 tile and the epilogue's
// streams dominate; here a thread owns two adjacent pixels, reads their K
// values as BF16 pairs (coalesced across the block), and forms the M outputs
// four at a time from op(A) in shared memory (FP32, exact copies of the BF16
// weights: every product is exact, as on the tensor cores), the four rows'
// epilogue inputs fetched together before their sums, so that their load
// latencies overlap; stores are pairs.  Requires even N, leading dimensions
// and batch strides, and 8-byte aligned FP32 / 4-byte aligned BF16 arrays.
constexpr int PW_THREADS = 128;

template <int MM, int KK>
__global__ void __launch_bounds__(PW_THREADS) pointwise_kernel(const GemmArgs g)
{
    static_assert(MM % 4 == 0 && KK % 4 == 0, "rows in groups of 4, k in float4 reads");
    __shared__ __align__(16) float As[MM][KK];
    const int z = blockIdx.y;
    const int z1 = z / g.nb2, z2 = z - z1 * g.nb2;
    const bf16 *A = g.A + z1 * g.sA1 + z2 * g.sA2;
    const bf16 *B = g.B + z1 * g.sB1 + z2 * g.sB2;
    const long long cofs = z1 * g.sC1 + z2 * g.sC2;
    for (int e = threadIdx.x; e < MM * KK; e += PW_THREADS) {
        const int m = e / KK, k = e - m * KK;
        As[m][k] = __bfloat162float(g.transA ? A[(long long)k * g.lda + m] : A[(long long)m * g.lda + k]);
    }
    __syncthreads();
    const long long n = ((long long)blockIdx.x * PW_THREADS + threadIdx.x) * 2;
    if (n >= g.N) return;
    float b0[KK], b1[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(B + (long long)k * g.ldb + n);
        b0[k] = __low2float(v);
        b1[k] = __high2float(v);
    }
#pragma unroll 1
    for (int m0 = 0; m0 < MM; m0 += 4) {
        float2 ad[4], ax[4], cf[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long off = cofs + (long long)(m0 + u) * g.ldc + n;
            ad[u] = g.add ? *reinterpret_cast<const float2 *>(g.add + off) : make_float2(0.f, 0.f);
            ax[u] = g.act == ACT_GELU_GRAD ? *reinterpret_cast<const float2 *>(g.aux + off) : make_float2(0.f, 0.f);
            cf[u] = g.beta != 0.f ? *reinterpret_cast<const float2 *>(g.Cf + off) : make_float2(0.f, 0.f);
        }
        const float2 bn = g.bias_n ? *reinterpret_cast<const float2 *>(g.bias_n + n) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = m0 + u;
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int k = 0; k < KK; k += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(&As[m][k]);
                a0 = fmaf(a.x, b0[k], a0);
                a1 = fmaf(a.x, b1[k], a1);
                a0 = fmaf(a.y, b0[k + 1], a0);
                a1 = fmaf(a.y, b1[k + 1], a1);
                a0 = fmaf(a.z, b0[k + 2], a0);
                a1 = fmaf(a.z, b1[k + 2], a1);
                a0 = fmaf(a.w, b0[k + 3], a0);
                a1 = fmaf(a.w, b1[k + 3], a1);
            }
            const long long off = cofs + (long long)m * g.ldc + n;
            float v0 = g.alpha * a0, v1 = g.alpha * a1;
            if (g.beta != 0.f) v0 += g.beta * cf[u].x, v1 += g.beta * cf[u].y;
            if (g.bias_m) v0 += g.bias_m[m], v1 += g.bias_m[m];
            if (g.bias_n) v0 += bn.x, v1 += bn.y;
            if (g.add) v0 += ad[u].x, v1 += ad[u].y;
            if (g.pre) *reinterpret_cast<float2 *>(g.pre + off) = make_float2(v0, v1);
            if (g.act == ACT_GELU) {
                v0 = gelu_f(v0);
                v1 = gelu_f(v1);
            } else if (g.act == ACT_GELU_GRAD) {
                v0 *= gelu_grad_f(ax[u].x);
                v1 *= gelu_grad_f(ax[u].y);
            }
            if (g.Cf) *reinterpret_cast<float2 *>(g.Cf + off) = make_float2(v0, v1);
            if (g.Cb) *reinterpret_cast<__nv_bfloat162 *>(g.Cb + off) = __floats2bfloat162_rn(v0, v1);
        }
    }
}

template <int MM, int KK>
inline bool pointwise_try(const GemmArgs &g, cudaStream_t s, cudaError_t &e)
{
    if (g.M != MM || g.K != KK) return false;
    const dim3 grid((unsigned)((g.N / 2 + PW_THREADS - 1) / PW_THREADS), g.batch, 1);
    pointwise_kernel<MM, KK><<<grid, PW_THREADS, 0, s>>>(g);
    e = cudaGetLastError();
    return true;
}

// The pointwise kernel's layout conditions (see above).
inline bool pointwise_fits(const GemmArgs &g)
{
    auto al = [](const void *p, unsigned a) { return ((uintptr_t)p % a) == 0; };
    const bool even = g.N % 2 == 0 && g.ldb % 2 == 0 && g.ldc % 2 == 0 && g.sB1 % 2 == 0 && g.sB2 % 2 == 0 &&
                      g.sC1 % 2 == 0 && g.sC2 % 2 == 0;
    return g.transB == 0 && g.N >= 1024 && g.batch <= 65535 && even && al(g.B, 4) && al(g.Cb, 4) && al(g.Cf, 8) &&
           al(g.add, 8) && al(g.pre, 8) && al(g.aux, 8) && al(g.bias_n, 8);
}

inline cudaError_t gemm(const GemmArgs &g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if (pointwise_fits(g)) {
        cudaError_t e = cudaSuccess;
        if (pointwise_try<32, 32>(g, s, e) || pointwise_try<64, 32>(g, s, e) || pointwise_try<32, 64>(g, s, e))
            return e;
    }
    const dim3 grid((g.M + GBM - 1) / GBM, (g.N + GBN - 1) / GBN, g.batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace fno
