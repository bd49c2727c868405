// Tensor-core (tcgen05) kernel for the hidden layers of the learned preconditioner:
//   Z = [H | A H] [W ; U] + b,  out = relu(Z)
// rows x 128 (bf16) times 128 x 64 (bf16) with float32 accumulation in tensor memory.
//
// One CTA of 4 warps owns one 128-row tile at a time (grid-stride over tiles).  Operands are
// converted to bf16 and stored in shared memory in the no-swizzle K-major layout: 8 x 8
// "core matrices" (8 rows of 16 bytes), adjacent along K at LBO = 128 B, adjacent along M/N at
// SBO = 16 * 128 B.  One elected thread issues 8 MMAs (M = 128, N = 64, K = 16 each) into a 64-
// column TMEM accumulator and commits them to an mbarrier; every warp then reads its 32 lanes
// (rows) with tcgen05.ld, adds the bias, applies relu and stores.  Waits on the mbarrier are
// bounded: on timeout the kernel records an error flag, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int TM = 128, TN = 64, TK = 128;           // tile rows, outputs, reduction (64 + 64)
constexpr uint32_t TMEM_COLS = 64;
constexpr long long WAIT_LIMIT = 1LL << 20;          // mbarrier polls before giving up (~1 s)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, version 1,
// no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor kind::f16: D f32, A bf16, B bf16, both K-major, N = TN, M = TM
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// element (r, k) of a core-matrix tile with K = TK: core (r/8, k/8) of 64 elements
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (TK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// out != nullptr: out = relu(Z) (rows x 64).  out == nullptr: the next layer's two row products
// a = relu(Z) w2 and q = relu(Z) u2 (w2, u2 of length 64) go to a and q instead.
template <class In>
__global__ void __launch_bounds__(128, 4) k_dense_tc(int64_t rows, const In *__restrict__ H,
                                                     const In *__restrict__ AH, const float *__restrict__ W,
                                                     const float *__restrict__ U, const float *__restrict__ b,
                                                     float *out, const float *__restrict__ w2,
                                                     const float *__restrict__ u2, float *a, float *q, int *err) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(dsm);   // TM x TK, 32 KiB
    __nv_bfloat16 *sB = sA + TM * TK;                               // TN x TK, 16 KiB
    __shared__ float sbias[TN], sw2[TN], su2[TN];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    // B = [W ; U]^T as TN x TK (row n, column k), bf16, core-matrix layout
    for (int e = tid; e < TN * TK; e += blockDim.x) {
        const int n = e / TK, k = e - n * TK;
        const float v = k < 64 ? W[k * TN + n] : U[(k - 64) * TN + n];
        sB[core_off(n, k)] = __float2bfloat16(v);
    }
    if (tid < TN) {
        sbias[tid] = __bfloat162float(__float2bfloat16(b[tid]));
        sw2[tid] = out ? 0.f : __bfloat162float(__float2bfloat16(w2[tid]));
        su2[tid] = out ? 0.f : __bfloat162float(__float2bfloat16(u2[tid]));
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;

    for (int64_t r0 = (int64_t)blockIdx.x * TM; r0 < rows; r0 += (int64_t)TM * gridDim.x) {
        if constexpr (sizeof(In) == 4) {
            // A tile: rows r0 .. r0 + 127 of [H | AH], converted to bf16, four values per load and
            // one 8-byte store (four consecutive K of one core-matrix row)
            for (int e = tid; e < TM * TK / 4; e += blockDim.x) {
                const int r = e / (TK / 4), k = 4 * (e - r * (TK / 4));
                const int64_t row = r0 + r;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < rows)
                    v = k < 64 ? *reinterpret_cast<const float4 *>(H + row * 64 + k)
                               : *reinterpret_cast<const float4 *>(AH + row * 64 + (k - 64));
                __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t *>(&lo);
                pk.y = *reinterpret_cast<uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>(sA + core_off(r, k)) = pk;
            }
        } else {
            // bf16 activations: one 16-byte load is one core-matrix row (eight consecutive K)
            for (int e = tid; e < TM * TK / 8; e += blockDim.x) {
                const int r = e / (TK / 8), k = 8 * (e - r * (TK / 8));
                const int64_t row = r0 + r;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (row < rows)
                    v = k < 64 ? *reinterpret_cast<const uint4 *>(H + row * 64 + k)
                               : *reinterpret_cast<const uint4 *>(AH + row * 64 + (k - 64));
                *reinterpret_cast<uint4 *>(sA + core_off(r, k)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const uint64_t ad = make_desc(a0 + kk * 256, 128, (TK / 8) * 128);
                const uint64_t bd = make_desc(b0 + kk * 256, 128, (TK / 8) * 128);
                const uint32_t acc = kk > 0 ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // bounded wait for the MMAs
        uint32_t done = 0;
        for (long long it = 0; it < WAIT_LIMIT && !done; ++it) {
            asm volatile(
                "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"(phase));
        }
        if (!done) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // accumulator rows 32 warp .. 32 warp + 31, 64 columns, 16 at a time
        const int64_t row = r0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        float da = 0.f, dq = 0.f;
#pragma unroll
        for (int cb = 0; cb < TN; cb += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr + cb));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (!out) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float hv = fmaxf(__uint_as_float(v[i]) + sbias[cb + i], 0.f);
                    da = fmaf(hv, sw2[cb + i], da);
                    dq = fmaf(hv, su2[cb + i], dq);
                }
            } else if (row < rows) {
                float4 *o = reinterpret_cast<float4 *>(out + row * TN + cb);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 t;
                    t.x = fmaxf(__uint_as_float(v[4 * q + 0]) + sbias[cb + 4 * q + 0], 0.f);
                    t.y = fmaxf(__uint_as_float(v[4 * q + 1]) + sbias[cb + 4 * q + 1], 0.f);
                    t.z = fmaxf(__uint_as_float(v[4 * q + 2]) + sbias[cb + 4 * q + 2], 0.f);
                    t.w = fmaxf(__uint_as_float(v[4 * q + 3]) + sbias[cb + 4 * q + 3], 0.f);
                    o[q] = t;
                }
            }
        }
        if (!out && row < rows) { a[row] = da; q[row] = dq; }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (abort_flag && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

// relu([H | AH] [W ; U] + b) for width-64 hidden layers on the tensor cores, into out, or (out
// null) only its products with w2 and u2 into a and q; the caller checks c->d_flag for a timed-out
// wait.  Four CTAs per SM (48 KiB of shared memory and 64 TMEM columns each), so that one CTA's
// tile loads overlap another's MMAs and epilogue.
void launch_dense_tc(ofks_ctx *c, int64_t rows, const float *H, const float *AH, const float *W, const float *U,
                     const float *b, float *out, const float *w2, const float *u2, float *a, float *q) {
    const int64_t tiles = (rows + TM - 1) / TM;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 4));
    const int smem = (TM + TN) * TK * (int)sizeof(__nv_bfloat16);
    cudaFuncSetAttribute(k_dense_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_dense_tc<float><<<grid, 128, smem, c->stream>>>(rows, H, AH, W, U, b, out, w2, u2, a, q, c->d_flag);
    c->kernels += 1;
}

// the same layer from bf16 activations (rows x 64 each), only the products a and q
void launch_dense_tc_bf16(ofks_ctx *c, int64_t rows, const __nv_bfloat16 *H, const __nv_bfloat16 *AH, const float *W,
                          const float *U, const float *b, const float *w2, const float *u2, float *a, float *q) {
    const int64_t tiles = (rows + TM - 1) / TM;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 4));
    const int smem = (TM + TN) * TK * (int)sizeof(__nv_bfloat16);
    cudaFuncSetAttribute(k_dense_tc<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_dense_tc<__nv_bfloat16><<<grid, 128, smem, c->stream>>>(rows, H, AH, W, U, b, nullptr, w2, u2, a, q, c->d_flag);
    c->kernels += 1;
}
