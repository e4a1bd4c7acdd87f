// heat_rwalk.cuh -- the r-sweep of the increment form (half-step 1 of the
// Peaceman-Rachford step, Sec. 3, eq. "scheme_eq_1") for FP32 lines of up to
// 32 RW_K cells, with the rows staged in shared memory by bulk copies and each
// line walked by one warp.
//
// A block of 4 warps walks a band of rows in groups of 4, warp w taking row
// j0 + w of each group.  The rows reach shared memory through a ring of
// kRwSlots rows: one cp.async.bulk copy per row (Nr * 4 bytes, one thread
// issues it), completed on a per-slot mbarrier, issued one group ahead, so a
// group's rows j0-1 .. j0+4 are resident while the next group's arrive.  The
// new row leaves by one cp.async.bulk store from a per-warp staging row.
//
// Line solve.  The line matrix is fixed per row class; its factorised
// coefficients {f, cp, q inv, inv} (f = xm inv, cp = xp inv, as in the other
// r-sweeps) sit in shared memory for the class the block is walking, laid out
// [k][lane] so that a warp's access at step k is 32 consecutive entries.  Lane
// l owns the K consecutive cells [l K, l K + K) of the row (K odd: lanes' cells
// fall in distinct banks of the unpadded row).  Four walks over the chunk:
//   1  right-hand side times inv, d_i (from rows j-1, j, j+1), kept in
//      registers; the chunk's forward summary B (the recurrence y = f y + d
//      from a zero carry);
//   -  scan of the maps y -> B + F y over the lanes (F = prod f, multipliers
//      per class) gives each chunk's incoming y;
//   2  forward recurrence from that carry, y over d in registers;
//   3  backward summary (x = y + cp x from a zero carry);
//   -  suffix scan of the maps (H = prod cp) gives each chunk's incoming x;
//   4  backward recurrence from it, theta + x to the staging row.
// The walks are unrolled (K is a template constant), about 25 instructions per
// cell, and a line needs no cross-warp join.
//
// Every wait on an mbarrier is bounded (a timer limit): on expiry the block
// records HEAT_ERR_TIMEOUT in the instance's status word, waits (bounded) for
// its copies still in flight and returns; the host reads the status.
#pragma once

#include "heat_internal.h"

namespace heat {

constexpr int kRwWarps = 4;         // warps (rows) per block
constexpr int kRwSlots = 10;        // ring rows: a group's j0-1 .. j0+4 and the next group's 4
constexpr unsigned long long kRwWaitNs = 1000000000ull;  // a wait gives up after 1 s

__device__ __forceinline__ unsigned long long rw_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned rw_smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void rw_mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rw_smem_addr(b)), "r"(count) : "memory");
}
// One row, global -> shared, completing `bytes` of transaction on barrier b.
__device__ __forceinline__ void rw_load_row(void *dst, const void *src, unsigned bytes, unsigned long long *b)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rw_smem_addr(b)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            rw_smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(rw_smem_addr(b))
        : "memory");
}
// Wait until barrier b completes the phase with the given parity, for at most
// limit_ns; false if the time ran out.
__device__ __forceinline__ bool rw_wait(unsigned long long *b, unsigned parity, unsigned long long limit_ns)
{
    const unsigned a = rw_smem_addr(b);
    const unsigned long long t0 = rw_now();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (rw_now() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void rw_store_row(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(rw_smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void rw_store_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void rw_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void rw_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory layout of one block (floats unless noted), K = RW_K:
//   ring   kRwSlots rows of SLOT = 32 K + 4 floats (row, then 4 ghost/pad floats)
//   dbuf   kRwWarps rows of SLOT (each warp's staging row for the bulk store)
//   tab    32 K float4 {f, cp, q inv, inv} of the current row class, [k][lane]
//   tcc    32 K column classes (bytes), [k][lane]
//   zrow   kRwWarps x 32 float2 (zm, zp) of the warp's row for each column class
//   bars   kRwSlots mbarriers (8 bytes each)
template <int K>
struct RwLayout {
    static constexpr int SLOT = 32 * K + 4;
    static constexpr size_t ring = 0;
    static constexpr size_t dbuf = ring + (size_t)kRwSlots * SLOT * 4;
    static constexpr size_t tab = dbuf + (size_t)kRwWarps * SLOT * 4;
    static constexpr size_t tcc = tab + (size_t)32 * K * 16;
    static constexpr size_t zrow = (tcc + (size_t)32 * K + 15) / 16 * 16;
    static constexpr size_t bars = zrow + (size_t)kRwWarps * 32 * 8;
    static constexpr size_t bytes = bars + (size_t)kRwSlots * 8;
};

template <int K>
__global__ void __launch_bounds__(32 * kRwWarps, 1) rwalk_kernel(const SweepArgs<float> *__restrict__ args, int flip)
{
    using L = RwLayout<K>;
    constexpr int SLOT = L::SLOT;
    pdl_launch_dependents();
    const SweepArgs<float> &A = args[blockIdx.y];
    const float *__restrict__ th = flip ? A.f1 : A.f0;
    float *__restrict__ out = flip ? A.f0 : A.f1;
    const int Nr = A.Nr, Nz = A.Nz;
    const int rows_per_block = A.band;  // a multiple of kRwWarps
    const int jstart = blockIdx.x * rows_per_block;
    if (jstart >= Nz) return;  // (block-uniform)
    const int jend = min(Nz, jstart + rows_per_block);
    extern __shared__ __align__(128) unsigned char rw_smem[];
    float *ring = reinterpret_cast<float *>(rw_smem + L::ring);
    float4 *tab = reinterpret_cast<float4 *>(rw_smem + L::tab);
    signed char *tcc = reinterpret_cast<signed char *>(rw_smem + L::tcc);
    float2 *zrow = reinterpret_cast<float2 *>(rw_smem + L::zrow);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(rw_smem + L::bars);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const float bc0 = (float)A.bc.th[0], bc1 = (float)A.bc.th[1];
    const float bc2 = (float)A.bc.th[2], bc3 = (float)A.bc.th[3];
    const unsigned row_bytes = (unsigned)Nr * 4u;
    const unsigned long long limit = A.rw_stall ? 2000000ull : kRwWaitNs;
    int *status = A.status;

    if (tid == 0) {
        for (int s = 0; s < kRwSlots; ++s) rw_mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the pad after each ring row: a ghost theta_bc(r_hi) at Nr (the r_hi
    // neighbour of the last cell), zeros beyond (cells past Nr have all-zero
    // coefficients)
    for (int s = 0; s < kRwSlots; ++s)
        for (int x = Nr + tid; x < SLOT; x += blockDim.x) ring[(size_t)s * SLOT + x] = x == Nr ? bc1 : 0.0f;
    for (int b = 0; b < kRwWarps; ++b) {
        float *d = reinterpret_cast<float *>(rw_smem + L::dbuf) + (size_t)b * SLOT;
        for (int x = Nr + tid; x < SLOT; x += blockDim.x) d[x] = 0.0f;
    }
    __syncthreads();
    if (A.rw_stall) {
        // failure-detection test: wait on a barrier nothing will complete,
        // with no copy issued, so the wait runs out and the status is set
        if (!rw_wait(&bars[0], 0, limit) && tid == 0) atomicOr(status, 1);
        return;
    }
    pdl_wait();

    // ring slot of row x and the parity of its load (loads of a slot alternate phases)
    auto slot_of = [&](int x) { return (x - jstart + 1) % kRwSlots; };
    auto parity_of = [&](int x) { return (unsigned)(((x - jstart + 1) / kRwSlots) & 1); };
    auto slot_ptr = [&](int x) { return ring + (size_t)slot_of(x) * SLOT; };
    // issue the load of row x (thread 0), or fill a ghost row (rows outside the field)
    auto issue = [&](int x) {
        float *dst = slot_ptr(x);
        if (x < 0 || x >= Nz) {
            const float g = x < 0 ? bc2 : bc3;
            for (int c = tid; c < Nr; c += blockDim.x) dst[c] = g;
            // complete the slot's phase all the same, so that its later loads
            // keep the parity slot_of / parity_of expect
            if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rw_smem_addr(&bars[slot_of(x)]))
                                       : "memory");
            return;
        }
        if (tid == 0) {
            rw_fence_async();
            rw_load_row(dst, th + (size_t)x * Nr, row_bytes, &bars[slot_of(x)]);
        }
    };
    auto ready = [&](int x) {  // wait for row x (all threads); false on time-out
        if (x < 0 || x >= Nz) return true;
        return rw_wait(&bars[slot_of(x)], parity_of(x), limit);
    };
    bool ok = true;
    auto give_up = [&](int issued_to) {
        // record the time-out; let every load still in flight land (bounded) first
        if (tid == 0) atomicOr(status, 1);
        for (int x = max(max(0, jstart - 1), issued_to - kRwSlots + 1); x <= min(Nz - 1, issued_to); ++x)
            rw_wait(&bars[slot_of(x)], parity_of(x), limit);  // the latest load of each slot
        if (lane == 0) rw_store_wait_all();
    };

    // prologue: rows jstart-1 .. jstart+4 (the first group) and the next group's 4
    const int last_needed = min(Nz, jend);  // rows up to jend (the r+1 neighbour of the last row)
    int issued = jstart - 2;
    auto issue_upto = [&](int x_to) {
        for (int x = issued + 1; x <= min(x_to, last_needed); ++x) issue(x);
        issued = max(issued, min(x_to, last_needed));
    };
    issue_upto(jstart + 8);
    __syncthreads();  // ghost rows filled

    int acls = -1;     // class whose coefficients are in tab
    float m[5], n[5];  // scan multipliers of that class (this lane)
    const int nc = A.rw_ncc;
    __shared__ int s_cls[kRwWarps];
    for (int j0 = jstart; j0 < jend; j0 += kRwWarps) {
        // this group's rows j0-1 .. j0+4 resident
        for (int x = j0 - 1; x <= min(j0 + kRwWarps, last_needed); ++x) ok = ok && ready(x);
        if (!__syncthreads_and(ok)) {
            give_up(issued);
            return;
        }
        const int j = j0 + w;
        // the rows of a group may span row classes: walk them one class at a time
        int my_cls = j < jend ? A.rowcls[j] : -1;  // -1: nothing (left) to walk
        for (;;) {
            if (lane == 0) s_cls[w] = my_cls;
            __syncthreads();  // (also: every walk of the previous round is over)
            int cls = -1;
#pragma unroll
            for (int v = 0; v < kRwWarps; ++v) cls = cls < 0 ? s_cls[v] : cls;
            if (cls < 0) break;
            if (cls != acls) {
                // the class's coefficients (all threads), then its scan multipliers
                const float4 *src = A.rw_tab + (size_t)cls * 32 * K;
                for (int e = tid; e < 32 * K; e += blockDim.x) tab[e] = src[e];
                if (acls < 0)
                    for (int e = tid; e < 32 * K; e += blockDim.x) tcc[e] = A.rw_cc[e];
                __syncthreads();
                float pf = 1.0f, ph = 1.0f;
#pragma unroll 1
                for (int k = 0; k < K; ++k) {
                    const float4 c = tab[k * 32 + lane];
                    pf *= c.x;
                    ph *= c.y;
                }
                // m_l = prod F over lanes lane-2^l+1 .. lane (0 below 2^l),
                // n_l = prod H over lanes lane .. lane+2^l-1 (0 past lane 31)
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const int off = 1 << l;
                    m[l] = lane >= off ? pf : 0.0f;
                    n[l] = lane + off < 32 ? ph : 0.0f;
                    const float pf2 = __shfl_up_sync(FULL, pf, off);
                    const float ph2 = __shfl_down_sync(FULL, ph, off);
                    pf = lane >= off ? pf * pf2 : pf;
                    ph = lane + off < 32 ? ph * ph2 : ph;
                }
                acls = cls;
            }
            __syncthreads();  // s_cls is rewritten next round
            if (my_cls != cls) continue;
            my_cls = -1;
            // this warp walks row j; the chunk's right-hand side and forward
            // results stay in registers (K is a compile-time constant)
            const float *__restrict__ rm = slot_ptr(j - 1);
            const float *__restrict__ rc = slot_ptr(j);
            const float *__restrict__ rp = slot_ptr(j + 1);
            float *__restrict__ D = reinterpret_cast<float *>(rw_smem + L::dbuf) + (size_t)w * SLOT;
            if (lane < nc) {
                const size_t zo = (size_t)lane * Nz + j;
                zrow[w * 32 + lane] = make_float2(A.Z.xm[zo], A.Z.xp[zo]);
            }
            __syncwarp();
            const float2 *__restrict__ zr = zrow + w * 32;
            const float4 *__restrict__ tb = tab + lane;
            const signed char *__restrict__ tc8 = tcc + lane;
            const int i0 = lane * K;
            float d[K];
            // walk 1: right-hand side times inv; forward summary from a zero carry
            float tl = i0 == 0 ? bc0 : rc[i0 - 1];
            float tc = rc[i0];
            float y = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = i0 + k;
                const float tr = rc[i + 1];
                const float4 c = tb[k * 32];
                const float2 z = zr[tc8[k * 32]];
                float v = fmaf(c.x, tl - tc, c.z);
                v = fmaf(c.y, tr - tc, v);
                const float zz = fmaf(z.y, rp[i] - tc, z.x * (rm[i] - tc));
                d[k] = fmaf(c.w, zz, v);
                y = fmaf(c.x, y, d[k]);
                tl = tc;
                tc = tr;
            }
#pragma unroll
            for (int l = 0; l < 5; ++l) y = fmaf(m[l], __shfl_up_sync(FULL, y, 1 << l), y);
            float yin = __shfl_up_sync(FULL, y, 1);
            if (lane == 0) yin = 0.0f;
            // walk 2: forward recurrence from the carry
#pragma unroll
            for (int k = 0; k < K; ++k) {
                yin = fmaf(tb[k * 32].x, yin, d[k]);
                d[k] = yin;
            }
            // walk 3: backward summary from a zero carry
            float g = 0.0f;
#pragma unroll
            for (int k = K - 1; k >= 0; --k) g = fmaf(tb[k * 32].y, g, d[k]);
#pragma unroll
            for (int l = 0; l < 5; ++l) g = fmaf(n[l], __shfl_down_sync(FULL, g, 1 << l), g);
            float xin = __shfl_down_sync(FULL, g, 1);
            if (lane == 31) xin = 0.0f;
            // the staging buffer's previous store has read it
            if (lane == 0) rw_store_wait_read<0>();
            __syncwarp();
            // walk 4: backward recurrence from the carry; theta + x to the staging row
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                xin = fmaf(tb[k * 32].y, xin, d[k]);
                D[i0 + k] = rc[i0 + k] + xin;
            }
            rw_fence_async();  // the generic writes of D before the async store reads them
            __syncwarp();
            if (lane == 0) rw_store_row(out + (size_t)j * Nr, D, row_bytes);
        }
        // every warp is past the group's rows: the slots of rows j0-1 .. j0+2
        // take the group after next's rows j0+9 .. j0+12
        __syncthreads();
        issue_upto(j0 + 3 * kRwWarps);
        __syncthreads();  // ghost rows written before anyone reads them
    }
    if (lane == 0) rw_store_wait_all();
}

}  // namespace heat
