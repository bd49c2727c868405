// Shared device helpers of libofks: error checking, warp/block reductions, P2 tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define OFKS_WARP 32

// Rows per SELL slice (one warp covers the rows of a slice).
#define SELL_C 32

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread gets the result.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    return t;
}

// P2 basis on the reference tetrahedron at the symmetric 4-point rule.
// Point q has barycentric coordinates QB everywhere except QA at vertex q, with
// QA = (5 + 3 sqrt 5)/20 and QB = (5 - sqrt 5)/20; every weight is |T|/4.
// Vertex function N_a = l_a (2 l_a - 1); edge function N_ab = 4 l_a l_b for the edges
// 01, 02, 03, 12, 13, 23 (local ids 4..9).  At these points a basis value is one of four
// numbers, depending only on whether the function's vertex/edge touches vertex q.
constexpr double P2_QA = 0.58541019662496845446137605030969143531609275394172;
constexpr double P2_QB = 0.13819660112501051517954131656343618822796908201943;

__host__ __device__ inline void p2_edge(int e, int &a, int &b) {
    a = (e < 3) ? 0 : (e < 5 ? 1 : 2);
    b = (e == 0) ? 1 : ((e == 1 || e == 3) ? 2 : 3);
}

__host__ __device__ inline double p2N(int q, int i) {
    if (i < 4) return (i == q) ? P2_QA * (2.0 * P2_QA - 1.0) : P2_QB * (2.0 * P2_QB - 1.0);
    int a, b;
    p2_edge(i - 4, a, b);
    return (a == q || b == q) ? 4.0 * P2_QA * P2_QB : 4.0 * P2_QB * P2_QB;
}

__host__ __device__ inline double p2_bary(int q, int k) { return (k == q) ? P2_QA : P2_QB; }
