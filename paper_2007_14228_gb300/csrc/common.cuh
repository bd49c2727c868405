// Shared device helpers of libofks: error checking, warp/block reductions, P2 tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define OFKS_WARP 32

// Rows per SELL slice (one warp covers the rows of a slice).
#define SELL_C 32

// a float64 value as the float32 pair (hi, lo) with hi + lo ~ v to ~48 significant bits
__device__ __forceinline__ float2 ff_split(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

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

// ---- deterministic reductions
// Float addition is not associative: sums whose terms arrive by atomics in a run-dependent order
// round differently from run to run, and the step-size rule amplifies such differences into
// different iterate sequences.  Every sum over more than one block therefore goes through
// partials written to scratch memory by their block (or warp) and added in a fixed order, so the
// same inputs give bit-identical results on every run.

// Fixed-order sum of a[0..n) over the block (thread t takes t, t + blockDim.x, ...; then the
// fixed tree of block_sum); every thread gets it.  L1 is bypassed: the partials may have been
// written by other blocks of the same grid.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double ordered_sum(const double *a, int64_t n, double *sh) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(a + i);
    return block_sum(s, sh);
}

// Grid-wide sums of K block totals v[k] (every thread of the block holds them).  Block b writes
// its totals to part[k * gridDim.x + b]; the last block to finish (counted with an integer
// atomic on *count, whose order does not matter) adds the partials in block order and calls
// out(k, sum) from thread 0.  Every block of the grid calls this exactly once, as its last
// action; *count is zero on entry and is left zero.  part holds K * gridDim.x doubles.
template <int K, class Out>
__device__ __forceinline__ void grid_accumulate(const double (&v)[K], double *part, unsigned *count, Out out) {
    __shared__ bool last;
    __shared__ double gsh[32];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[(int64_t)k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const double s = ordered_sum(part + (int64_t)k * gridDim.x, gridDim.x, gsh);
        if (threadIdx.x == 0) out(k, s);
    }
    if (threadIdx.x == 0) *count = 0u;
}

// Per-block column sums for the flattened n x ld element loops whose thread keeps column
// j = (global thread index) mod ld: the block's threads of column k are added in thread order
// into part[k * gridDim.x + blockIdx.x] (k < ncol <= ld <= blockDim.x).  Every thread calls it.
__device__ __forceinline__ void col_partial(double acc, bool active, int ld, int ncol, double *part) {
    __shared__ double cval[256];
    cval[threadIdx.x] = active ? acc : 0.0;
    __syncthreads();
    const int k = threadIdx.x;
    if (k < ncol) {
        // thread t holds column ((blockIdx.x * blockDim.x + t) mod ld)
        const int t0 = (int)((k - (int64_t)blockIdx.x * blockDim.x % ld + ld) % ld);
        double s = 0.0;
        for (int t = t0; t < (int)blockDim.x; t += ld) s += cval[t];
        part[(int64_t)k * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
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
