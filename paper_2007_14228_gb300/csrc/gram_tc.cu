// Tensor-core (tcgen05) Grams of the float32 iterations: XA = X^T A and XB = X^T B in one pass
// (A = H X and B = B X give Lambda0 = X^T H X and S = X^T B X of Alg. 2).
//
// D[m][n] = sum_k X[k][m] Y[k][n] with Y = [A | B] side by side: M = 128 (the columns of X,
// zero-padded), N = 2 * ld16 (ld16 = ld rounded up to 16), K = the rows of the blocks.  Each
// persistent CTA walks 64-row slabs of the rows: the slab's contiguous rows of X, A and B
// (64 * ld floats each) arrive in shared memory by the TMA bulk-copy engine (cp.async.bulk with
// an mbarrier transaction count, double-buffered so the next slab streams in while this one is
// converted and multiplied); the threads split every float v three ways in bf16 (v = h + m + l:
// h = bf16(v), m = bf16(v - h), l = bf16(v - h - m)) and write the parts transposed into the
// no-swizzle K-major core-matrix layout; one elected thread issues the six products
// hh + hm + mh + hl + lh + mm (the dropped terms are ~2^-24 of each product, float32's own
// rounding) as M = 128, N = 2 ld16, K = 16 MMAs into a float32 accumulator in tensor memory.  (A
// two-way split, hh + hl + lh, leaves ~2^-16 of each product; in the multipliers, which sum
// products of both signs, that held the float32 iterations' energy 3.7e-3 Ha from the float64
// fixed point on the chain.)  Eight warps convert; after its last slab a CTA's warps 0-3 read
// their 32 rows each back and write the upper triangle (i <= j < p) as the CTA's float64
// partial; k_gram_fin adds the CTAs' partials in order and mirrors.  Four CTAs' worth of slabs
// per SM (in waves) keep the float32 accumulation short.
// Every wait is bounded: on timeout the CTA records an error flag, waits (bounded) for its own
// copies in flight, frees its tensor memory and returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int GKS = 64;                          // rows per slab
constexpr int GTM = 128;                         // MMA M (columns of X, padded)
constexpr long long GWAIT = 1LL << 22;           // mbarrier polls before giving up

__device__ __forceinline__ uint32_t s32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t gdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// element (r, k) of a K-major tile with GKS columns: core matrix (r / 8, k / 8) of 8 x 8
__device__ __forceinline__ int goff(int r, int k) { return ((r >> 3) * (GKS >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16(r1);
    l = __float2bfloat16(r1 - __bfloat162float(m));
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done = 0;
    for (long long w = 0; w < GWAIT && !done; ++w)
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(s32(bar)), "r"(parity)
            : "memory");
    return done != 0;
}

// thread 0: the three slabs of rows [r0, r0 + rows) into raw buffer `buf`
__device__ __forceinline__ void issue_loads(uint64_t *bar, float *dst, const float *X, const float *A,
                                            const float *B, int64_t r0, int rows, int ld) {
    const uint32_t bytes = (uint32_t)rows * (uint32_t)ld * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(bar)), "r"(3u * bytes) : "memory");
    const float *src[3] = {X + r0 * ld, A + r0 * ld, B + r0 * ld};
    for (int q = 0; q < 3; ++q)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                s32(dst + (size_t)q * GKS * ld)),
            "l"(src[q]), "r"(bytes), "r"(s32(bar))
            : "memory");
}

__global__ void __launch_bounds__(256, 1) k_gram_tc(int64_t n, int p, int ld, int nh, int tcols, const float *__restrict__ X,
                                                    const float *__restrict__ A, const float *__restrict__ B, double *part,
                                                    int *err) {
    extern __shared__ __align__(128) unsigned char gsm[];
    const int NP = 2 * nh;
    float *raw = reinterpret_cast<float *>(gsm);                           // 2 buffers x 3 x GKS x ld
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(raw + (size_t)2 * 3 * GKS * ld);   // 3 x GTM x GKS
    __nv_bfloat16 *ys = xs + (size_t)3 * GTM * GKS;                                          // 3 x NP x GKS
    __shared__ __align__(8) uint64_t bar_ld[2], bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nslab = (n + GKS - 1) / GKS;
    const int T = (int)((nslab - blockIdx.x + gridDim.x - 1) / gridDim.x);   // slabs of this CTA

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&tmem_base)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // operand tiles start at zero: the padding rows (m >= ld) and columns stay zero
    for (int e = tid; e < 3 * (GTM + NP) * GKS / 8; e += blockDim.x)
        reinterpret_cast<uint4 *>(xs)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(&bar_ld[b])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    int pending[2] = {0, 0};                     // loads issued and not yet waited for, per buffer (thread 0's view)
    if (tid == 0 && T > 0) {
        const int64_t r0 = (int64_t)blockIdx.x * GKS;
        issue_loads(&bar_ld[0], raw, X, A, B, r0, (int)(n - r0 < GKS ? n - r0 : GKS), ld);
        pending[0] = 1;
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(GTM >> 4) << 24);
    int t = 0;
    for (; t < T; ++t) {
        const int buf = t & 1;
        const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * GKS;
        const int rows = (int)(n - r0 < GKS ? n - r0 : GKS);
        if (tid == 0 && t + 1 < T) {             // the next slab streams in meanwhile
            const int64_t r1 = r0 + (int64_t)gridDim.x * GKS;
            issue_loads(&bar_ld[buf ^ 1], raw + (size_t)(buf ^ 1) * 3 * GKS * ld, X, A, B, r1,
                        (int)(n - r1 < GKS ? n - r1 : GKS), ld);
            pending[buf ^ 1] = 1;
        }
        bool ok = bar_wait(&bar_ld[buf], (uint32_t)((t >> 1) & 1));
        if (tid == 0 && ok) pending[buf] = 0;       // a timed-out copy stays pending
        if (ok && t > 0) ok = bar_wait(&bar_mma, (uint32_t)((t - 1) & 1));   // the MMAs still read the tiles
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        // three-way split, transposed into the K-major tiles: X^T (m = column of X) and [A | B]^T
        const float *rx = raw + (size_t)buf * 3 * GKS * ld, *ra = rx + (size_t)GKS * ld, *rb = ra + (size_t)GKS * ld;
        const size_t xq = (size_t)GTM * GKS, yq = (size_t)NP * GKS;
        for (int e = tid; e < GKS * ld; e += blockDim.x) {
            const int k = e / ld, m = e - k * ld;
            const bool in = k < rows;
            __nv_bfloat16 h, md, l;
            split3(in ? rx[e] : 0.f, h, md, l);
            xs[goff(m, k)] = h; xs[xq + goff(m, k)] = md; xs[2 * xq + goff(m, k)] = l;
            split3(in ? ra[e] : 0.f, h, md, l);
            ys[goff(m, k)] = h; ys[yq + goff(m, k)] = md; ys[2 * yq + goff(m, k)] = l;
            split3(in ? rb[e] : 0.f, h, md, l);
            ys[goff(nh + m, k)] = h; ys[yq + goff(nh + m, k)] = md; ys[2 * yq + goff(nh + m, k)] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t sbo = (GKS / 8) * 128u;
            // parts 0 = h, 1 = m, 2 = l: hh, hm, mh, hl, lh, mm
            const int ta[6] = {0, 0, 1, 0, 2, 1}, tb[6] = {0, 1, 0, 2, 0, 1};
            uint32_t opa[6], opb[6];
            for (int q = 0; q < 6; ++q) {
                opa[q] = s32(xs + (size_t)ta[q] * GTM * GKS);
                opb[q] = s32(ys + (size_t)tb[q] * NP * GKS);
            }
            for (int term = 0; term < 6; ++term)
                for (int kk = 0; kk < GKS / 16; ++kk) {
                    const uint64_t ad = gdesc(opa[term] + kk * 256, 128, sbo);
                    const uint64_t bd = gdesc(opb[term] + kk * 256, 128, sbo);
                    const uint32_t accum = (t > 0 || term > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                s32(&bar_mma)));
        }
    }
    // the last commit, then the accumulator
    if (!abort_flag && T > 0 && !bar_wait(&bar_mma, (uint32_t)((T - 1) & 1))) abort_flag = 1;
    __syncthreads();
    if (!abort_flag && T > 0 && warp < 4) {    // warps 0-3 own the accumulator's 128 lanes
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int i = warp * 32 + lane;                                 // row of D: column i of X
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < NP; cb += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr + cb));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (i >= p) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int col = cb + q;
                const int m = col < nh ? 0 : 1, j = col < nh ? col : col - nh;
                if (j < i || j >= p) continue;
                part[(((int64_t)m * ld + i) * ld + j) * gridDim.x + blockIdx.x] = (double)__uint_as_float(v[q]);
            }
        }
    }
    if (abort_flag || T == 0) {                // no accumulator: this CTA's partials are zero
        for (int e = tid; e < 2 * ld * ld; e += blockDim.x) {
            const int m = e / (ld * ld), i = (e / ld) % ld, j = e % ld;
            if (i <= j && j < p) part[(((int64_t)m * ld + i) * ld + j) * gridDim.x + blockIdx.x] = 0.0;
        }
    }
    if (abort_flag) {
        if (tid == 0) atomicExch(err, 1);
        // our own bulk copies may still be in flight: wait for them (bounded) before leaving
        if (tid == 0)
            for (int b = 0; b < 2; ++b)
                if (pending[b]) bar_wait(&bar_ld[b], (uint32_t)(((t + (b != (t & 1))) >> 1) & 1));
        // so may the MMAs of the last committed slab (slabs 0 .. t-1 were committed; the earlier
        // ones were waited for): wait for that commit once more (bounded) before the tensor
        // memory is released
        if (tid == 0 && t > 0) bar_wait(&bar_mma, (uint32_t)((t - 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

}  // namespace

// Tensor-core Grams for float32 blocks; false when the shapes do not suit it (the caller then
// runs the CUDA-core kernel).  Each CTA writes its partial upper triangles of X^T A and X^T B to
// part, entry (m, i, j) of CTA u at ((m ld + i) ld + j) units + u; k_gram_fin adds them in CTA
// order and mirrors.
bool launch_gram_tc(ofks_ctx *c, const float *X, const float *A, const float *B, double *part, int64_t *units) {
    const int ld = c->ld;
    if (!c->prm.gram_tc || ld < 4 || ld % 4 || ld > 64 || c->n < GKS) return false;
    const int nh = (ld + 15) / 16 * 16, NP = 2 * nh;
    const int tcols = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
    const size_t smem = sizeof(float) * 2 * 3 * GKS * ld + sizeof(__nv_bfloat16) * (size_t)3 * (GTM + NP) * GKS;
    const int64_t nslab = (c->n + GKS - 1) / GKS;
    // partials of 2 ld^2 doubles per CTA must fit the scratch (CPART_MIN >= 2 * 64^2 * 608)
    const unsigned grid = (unsigned)std::min<int64_t>(nslab, 152 * 4);
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_tc<<<grid, 256, smem, c->stream>>>(c->n, c->p, ld, nh, tcols, X, A, B, part, c->d_flag + 2);
    c->kernels += 1;
    *units = grid;
    return true;
}
