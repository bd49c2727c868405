// Tensor-core (tcgen05) gradient update of the float32 iterations (Alg. 2):
//   G = H X + B X C,   R = H X - B X Lambda0  (kkt^2 += |R|^2 over the columns < p)
// for 128-row tiles of the n x ld blocks.  One GEMM per tile, D = (B X)[128 x K] [C | Lambda0]
// with K = ld (padded to 16) and N = 2 ld16.  Since G tends to zero by cancellation near the
// fixed point, the operands are split three ways in bf16 (v = h + m + l) and six products
// hh + hm + mh + hl + mm + lh are accumulated in float32 (the dropped terms are ~2^-24 of each
// product, float32 rounding).  Each persistent CTA walks row tiles: the tile's contiguous rows of
// B X and H X arrive by the TMA bulk-copy engine (double-buffered, mbarrier transaction counts);
// the threads split B X into the K-major core-matrix layout; one thread issues the MMAs; warps 0-3
// read their 32 rows back, form G in place of H X in shared memory and accumulate |R|^2; one thread
// stores the G tile with a TMA bulk store.  [C | Lambda0] is split once per CTA.  Every wait is
// bounded: on timeout the CTA records an error flag, waits (bounded) for its own loads in flight,
// drains its stores, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int RTM = 128;                         // rows per tile (MMA M)
constexpr long long RWAIT = 1LL << 22;

__device__ __forceinline__ uint32_t r32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t rdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// element (r, k) of a K-major tile with KP columns
__device__ __forceinline__ int roff(int r, int k, int KP) { return ((r >> 3) * (KP >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ bool rwait(uint64_t *bar, uint32_t parity) {
    uint32_t done = 0;
    for (long long w = 0; w < RWAIT && !done; ++w)
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(r32(bar)), "r"(parity)
            : "memory");
    return done != 0;
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16(r1);
    l = __float2bfloat16(r1 - __bfloat162float(m));
}

// thread 0: rows [r0, r0 + rows) of B X and H X into raw buffer dst (2 x RTM x ld floats)
__device__ __forceinline__ void grad_loads(uint64_t *bar, float *dst, const float *BX, const float *HX, int64_t r0,
                                           int rows, int ld) {
    const uint32_t bytes = (uint32_t)rows * (uint32_t)ld * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(r32(bar)), "r"(2u * bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     r32(dst)), "l"(BX + r0 * ld), "r"(bytes), "r"(r32(bar)) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     r32(dst + (size_t)RTM * ld)), "l"(HX + r0 * ld), "r"(bytes), "r"(r32(bar)) : "memory");
}

__global__ void __launch_bounds__(256, 1) k_grad_tc(int64_t n, int p, int ld, int KP, int nh, int tcols,
                                                    const float *__restrict__ HX, const float *__restrict__ BX,
                                                    const double *__restrict__ C, const double *__restrict__ L0,
                                                    float *G, double *kkt2, int *err, double *gpart,
                                                    unsigned *gcount) {
    extern __shared__ __align__(128) unsigned char rsm[];
    const int NP = 2 * nh;
    float *raw = reinterpret_cast<float *>(rsm);                              // 2 x (B X, H X) tiles
    __nv_bfloat16 *A3 = reinterpret_cast<__nv_bfloat16 *>(raw + (size_t)4 * RTM * ld);   // 3 x RTM x KP
    __nv_bfloat16 *B3 = A3 + (size_t)3 * RTM * KP;                                      // 3 x NP x KP
    __shared__ __align__(8) uint64_t bar_ld[2], bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntile = (n + RTM - 1) / RTM;
    const int T = (int)((ntile - blockIdx.x + gridDim.x - 1) / gridDim.x);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(r32(&tmem_base)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // operand tiles start at zero (padding columns k >= ld, rows n >= ld of each half)
    for (int e = tid; e < (3 * RTM + 3 * NP) * KP / 8; e += blockDim.x)
        reinterpret_cast<uint4 *>(A3)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(r32(&bar_ld[b])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(r32(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    __syncthreads();
    // [C | Lambda0]^T split three ways: element (col, k) = C[k][col] or Lambda0[k][col]
    for (int e = tid; e < 2 * ld * ld; e += blockDim.x) {
        const int half = e / (ld * ld), q = e - half * ld * ld, k = q / ld, col = q - k * ld;
        const float v = (float)(half ? L0 : C)[(int64_t)k * ld + col];
        __nv_bfloat16 h, m, l;
        split3(v, h, m, l);
        const int o = roff(half * nh + col, k, KP);
        B3[o] = h;
        B3[(size_t)NP * KP + o] = m;
        B3[(size_t)2 * NP * KP + o] = l;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    int pending[2] = {0, 0};
    if (tid == 0 && T > 0) {
        const int64_t r0 = (int64_t)blockIdx.x * RTM;
        grad_loads(&bar_ld[0], raw, BX, HX, r0, (int)(n - r0 < RTM ? n - r0 : RTM), ld);
        pending[0] = 1;
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(RTM >> 4) << 24);
    const uint32_t sbo = (uint32_t)(KP >> 3) * 128u;
    double part = 0.0;
    int mma_out = 0;                             // this thread saw tile t's MMAs time out (still in flight)
    int t = 0;
    for (; t < T; ++t) {
        const int buf = t & 1;
        const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * RTM;
        const int rows = (int)(n - r0 < RTM ? n - r0 : RTM);
        float *bx = raw + (size_t)buf * 2 * RTM * ld, *hx = bx + (size_t)RTM * ld;
        if (tid == 0 && t + 1 < T) {
            // the other buffer's G tile (tile t - 1) must have left shared memory first
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            const int64_t r1 = r0 + (int64_t)gridDim.x * RTM;
            grad_loads(&bar_ld[buf ^ 1], raw + (size_t)(buf ^ 1) * 2 * RTM * ld, BX, HX, r1,
                       (int)(n - r1 < RTM ? n - r1 : RTM), ld);
            pending[buf ^ 1] = 1;
        }
        const bool ok = rwait(&bar_ld[buf], (uint32_t)((t >> 1) & 1));
        if (tid == 0 && ok) pending[buf] = 0;
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        // B X split three ways into the K-major A tiles (rows past the end are zero)
        for (int e = tid; e < RTM * ld; e += blockDim.x) {
            const int r = e / ld, k = e - r * ld;
            const float v = r < rows ? bx[e] : 0.f;
            __nv_bfloat16 h, m, l;
            split3(v, h, m, l);
            const int o = roff(r, k, KP);
            A3[o] = h;
            A3[(size_t)RTM * KP + o] = m;
            A3[(size_t)2 * RTM * KP + o] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            // hh + hm + mh + hl + mm + lh
            const int ta[6] = {0, 0, 1, 0, 1, 2}, tb[6] = {0, 1, 0, 2, 1, 0};
            for (int term = 0; term < 6; ++term)
                for (int kk = 0; kk < KP / 16; ++kk) {
                    const uint64_t ad = rdesc(r32(A3 + (size_t)ta[term] * RTM * KP) + kk * 256, 128, sbo);
                    const uint64_t bd = rdesc(r32(B3 + (size_t)tb[term] * NP * KP) + kk * 256, 128, sbo);
                    const uint32_t accum = (term > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                r32(&bar_mma)));
        }
        if (!rwait(&bar_mma, (uint32_t)(t & 1))) { abort_flag = 1; mma_out = 1; }
        __syncthreads();
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (warp < 4) {                          // G = H X + D1 in place of H X, |H X - D2|^2
            const int r = warp * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            float rp = 0.f;                      // this row's |R|^2 (at most 64 terms) in float
            for (int cb = 0; cb < nh; cb += 16) {
                uint32_t v1[16], v2[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v1[0]), "=r"(v1[1]), "=r"(v1[2]), "=r"(v1[3]), "=r"(v1[4]), "=r"(v1[5]), "=r"(v1[6]),
                      "=r"(v1[7]), "=r"(v1[8]), "=r"(v1[9]), "=r"(v1[10]), "=r"(v1[11]), "=r"(v1[12]), "=r"(v1[13]),
                      "=r"(v1[14]), "=r"(v1[15])
                    : "r"(taddr + cb));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]),
                      "=r"(v2[7]), "=r"(v2[8]), "=r"(v2[9]), "=r"(v2[10]), "=r"(v2[11]), "=r"(v2[12]), "=r"(v2[13]),
                      "=r"(v2[14]), "=r"(v2[15])
                    : "r"(taddr + nh + cb));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (r >= rows) continue;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = cb + q;
                    if (col >= ld) break;
                    float *hp = hx + (size_t)r * ld + col;
                    const float h = *hp;
                    *hp = h + __uint_as_float(v1[q]);                 // G
                    if (col < p) {
                        const float res = h - __uint_as_float(v2[q]);   // R
                        rp = fmaf(res, res, rp);
                    }
                }
            }
            part += (double)rp;
        }
        // the G tile leaves by a bulk store from shared memory
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(G + r0 * ld), "r"(r32(hx)),
                         "r"((uint32_t)rows * (uint32_t)ld * 4u) : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    double cta_kkt2 = 0.0;                       // this CTA's |R|^2, added over the grid at the end
    for (int w = 0; w < 8; ++w) cta_kkt2 += red[w];
    if (tid == 0) {
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // our G stores have landed
        if (abort_flag) {
            atomicExch(err, 1);
            for (int b = 0; b < 2; ++b)
                if (pending[b]) rwait(&bar_ld[b], (uint32_t)(((t + (b != (t & 1))) >> 1) & 1));
            // MMAs whose commit timed out may still read shared memory and write tensor memory:
            // wait once more (bounded) before the tensor memory is released
            if (mma_out) rwait(&bar_mma, (uint32_t)(t & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
    const double tot[1] = {cta_kkt2};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { *kkt2 += v; });
}

}  // namespace

// Tensor-core gradient for float32 blocks; false when the shapes do not suit it (the caller then
// runs the CUDA-core kernel).  kkt2 must be zero on entry.
bool launch_grad_tc(ofks_ctx *c, const float *HX, const float *BX, float *G, double *kkt2) {
    const int ld = c->ld;
    if (!c->prm.gram_tc || ld < 4 || ld % 4 || ld > 64 || c->n < RTM) return false;
    const int KP = (ld + 15) / 16 * 16, nh = KP, NP = 2 * nh;
    const int tcols = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
    const size_t smem = sizeof(float) * 4 * RTM * ld + sizeof(__nv_bfloat16) * (size_t)(3 * RTM + 3 * NP) * KP;
    if (smem > 220 * 1024) return false;
    const int64_t ntile = (c->n + RTM - 1) / RTM;
    const unsigned grid = (unsigned)(ntile < 152 ? ntile : 152);
    cudaFuncSetAttribute(k_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_grad_tc<<<grid, 256, smem, c->stream>>>(c->n, c->p, ld, KP, nh, tcols, HX, BX, c->d_C, c->d_L0, G, kkt2,
                                              c->d_flag + 2, c->d_gpart, c->d_gcount);
    c->kernels += 1;
    return true;
}
