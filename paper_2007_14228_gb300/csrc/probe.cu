// Arithmetic peak probe: the float64 and float32 FMA rates of the device the context runs on,
// the denominators of the ALU roofline of the plain float64 form (the paper's method in
// float64 on GB300 is bound by the FP64 pipe, not by HBM).  Eight independent FMA chains per
// thread, 8 CTAs of 256 threads per SM, timed with CUDA events on the context's stream.
#include "internal.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(ofks_ctx *c, int iters, double *tflops) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int blocks = sms * 8, threads = 256, reps = 5;
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&out, sizeof(T) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma_chains<T><<<blocks, threads, 0, c->stream>>>(out, iters, (T)0.999999, (T)1e-7);   // warm-up
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, threads, 0, c->stream>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1, c->stream);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        c->kernels += reps + 1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "fma probe");
    *tflops = 2.0 * 8.0 * reps * (double)blocks * threads * iters / (ms * 1e-3) / 1e12;
    return OFKS_OK;
}

}  // namespace

int ofks_fma_peak(ofks_ctx *c, int32_t precision, double *tflops) {
    if (!c || !tflops || (precision != OFKS_FP64 && precision != 32)) return OFKS_EINVAL;
    return precision == OFKS_FP64 ? run<double>(c, 1 << 14, tflops) : run<float>(c, 1 << 16, tflops);
}
