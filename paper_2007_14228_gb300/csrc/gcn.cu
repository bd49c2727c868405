// Learned preconditioner: a 3-layer graph network on the free-DoF graph of the P2 mesh that maps a
// gradient column G_c to an approximation of T_c^{-1} G_c (T_c = L/2 - Lambda_cc B, paper
// Eq. precondition-T), with its forward, backward and Adam kernels.
//
// Per column c (shift lam_c <= 0):  diag = dL/2 - lam_c dB,  z = g / diag,  s_c = rms(z),
//   features f = [z / s_c, log diag - mean log diag, -lam_c dB / diag, 1]
//   Z_l = H_l W_l + (A H_l) U_l + b_l,  H_{l+1} = relu(Z_l) (hidden) / Z_l (last)
//   D = s_c (f0 + H_3)
// A is the mean over the closed neighbourhood (1/|N(i)| on the pattern of L).  Activations are
// rows (i, c) of an (n p) x F float32 matrix, so the aggregation over nodes is the SELL SpMM
// with leading dimension p F.  Weights are float32 masters rounded to bfloat16 where used;
// products accumulate in float32, reductions over rows in float64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int F0 = 4;

__device__ __forceinline__ float bf(float w) { return __bfloat162float(__float2bfloat16(w)); }

// column sums of z^2 and of log(diag) (float64): the block's partials of column c to
// stats[c grid + block] and stats[(p + c) grid + block]
__global__ void __launch_bounds__(256) k_feat_stats(int64_t n, int p, const float *__restrict__ G,
                                                    const double *__restrict__ dL, const double *__restrict__ dB,
                                                    const double *__restrict__ shift, double *stats) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t S = (int64_t)gridDim.x * blockDim.x / p * p;
    const int c = (int)(gid % p);
    double a = 0.0, b = 0.0;
    if (gid < S) {
        const float lam = (float)fmin(shift[c], 0.0);
        for (int64_t e = gid; e < n * p; e += S) {
            const int64_t i = e / p;
            const float d = 0.5f * (float)dL[i] - lam * (float)dB[i];
            const float z = G[e] / d;
            a += (double)(z * z);
            b += (double)logf(d);
        }
    }
    // per-block column partials, added in block order by launch_col_fin
    col_partial(a, gid < S, p, p, stats);
    col_partial(b, gid < S, p, p, stats + (int64_t)p * gridDim.x);
}

// per column: the scale s_c = rms(z), the mean log-diagonal and the shift lam_c = min(Lambda_cc, 0)
// (float32, colf[0..p) s, [p..2p) mean log, [2p..3p) lam; s also to scale)
__global__ void k_col_scales(int64_t n, int p, const double *__restrict__ stats, const double *__restrict__ shift,
                             float *colf, float *scale) {
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        const float s = (float)sqrt(stats[c] / (double)n);
        colf[c] = s;
        colf[p + c] = (float)(stats[p + c] / (double)n);
        colf[2 * p + c] = (float)fmin(shift[c], 0.0);
        scale[c] = s;
    }
}

// features (rows (i, c)): one float4 per row, from the per-column values of k_col_scales
__global__ void __launch_bounds__(256) k_features(int64_t n, int p, const float *__restrict__ G,
                                                  const double *__restrict__ dL, const double *__restrict__ dB,
                                                  const float *__restrict__ colf, float *F) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    const int64_t i = e / p;
    const int c = (int)(e - i * p);
    const float lam = colf[2 * p + c], s = colf[c];
    const float db = (float)dB[i];
    const float d = 0.5f * (float)dL[i] - lam * db;
    float4 f;
    f.x = s > 0.f ? G[e] / d / s : 0.f;
    f.y = logf(d) - colf[p + c];
    f.z = -lam * db / d;
    f.w = 1.f;
    reinterpret_cast<float4 *>(F)[e] = f;
}

// Z = H W + AH U + b (rows x FO), H/AH rows x FI; out = relu(Z) if relu else Z.  A block owns 64
// rows; thread t owns rows 4 (t / (FO/ 4)) ... and 4 consecutive outputs.
template <int FI, int FO, class OT = float>
__global__ void __launch_bounds__(256) k_dense(int64_t rows, const float *__restrict__ H, const float *__restrict__ AH,
                                               const float *__restrict__ W, const float *__restrict__ U,
                                               const float *__restrict__ b, int relu, float *Z, OT *out) {
    constexpr int RB = FI >= 64 ? 16 : 64;             // rows per tile (static shared memory <= 48 KiB)
    constexpr int OC = FO >= 4 ? 4 : 1;                 // outputs per thread
    constexpr int TPR = FO / OC;                        // threads per row group
    constexpr int RPT = RB * TPR / 256 > 0 ? RB * TPR / 256 : 1;   // rows per thread
    __shared__ float sW[FI * FO], sU[FI * FO], sb[FO];
    __shared__ float sH[RB * FI], sA[RB * FI];
    for (int k = threadIdx.x; k < FI * FO; k += 256) { sW[k] = bf(W[k]); sU[k] = bf(U[k]); }
    for (int k = threadIdx.x; k < FO; k += 256) sb[k] = bf(b[k]);
    for (int64_t r0 = blockIdx.x * (int64_t)RB; r0 < rows; r0 += (int64_t)RB * gridDim.x) {
        __syncthreads();
        for (int k = threadIdx.x; k < RB * FI; k += 256) {
            const int64_t r = r0 + k / FI;
            sH[k] = r < rows ? H[r0 * FI + k] : 0.f;
            sA[k] = r < rows ? AH[r0 * FI + k] : 0.f;
        }
        __syncthreads();
        const int og = threadIdx.x % TPR, rg = threadIdx.x / TPR;
        if (rg * RPT < RB) {
            float acc[RPT][OC];
#pragma unroll
            for (int a = 0; a < RPT; ++a)
#pragma unroll
                for (int o = 0; o < OC; ++o) acc[a][o] = sb[og * OC + o];
            for (int k = 0; k < FI; ++k) {
                float w[OC], u[OC];
#pragma unroll
                for (int o = 0; o < OC; ++o) { w[o] = sW[k * FO + og * OC + o]; u[o] = sU[k * FO + og * OC + o]; }
#pragma unroll
                for (int a = 0; a < RPT; ++a) {
                    const float h = sH[(rg * RPT + a) * FI + k], ah = sA[(rg * RPT + a) * FI + k];
#pragma unroll
                    for (int o = 0; o < OC; ++o) acc[a][o] = fmaf(h, w[o], fmaf(ah, u[o], acc[a][o]));
                }
            }
#pragma unroll
            for (int a = 0; a < RPT; ++a) {
                const int64_t r = r0 + rg * RPT + a;
                if (r >= rows) continue;
                if constexpr (sizeof(OT) == 2 && OC == 4) {      // bf16 out: one 8-byte store
                    const float v0 = relu ? fmaxf(acc[a][0], 0.f) : acc[a][0], v1 = relu ? fmaxf(acc[a][1], 0.f) : acc[a][1];
                    const float v2 = relu ? fmaxf(acc[a][2], 0.f) : acc[a][2], v3 = relu ? fmaxf(acc[a][3], 0.f) : acc[a][3];
                    __nv_bfloat162 lo = __floats2bfloat162_rn(v0, v1), hi = __floats2bfloat162_rn(v2, v3);
                    uint2 pk;
                    pk.x = *reinterpret_cast<uint32_t *>(&lo);
                    pk.y = *reinterpret_cast<uint32_t *>(&hi);
                    *reinterpret_cast<uint2 *>(out + r * FO + og * OC) = pk;
                    if (Z)
#pragma unroll
                        for (int o = 0; o < OC; ++o) Z[r * FO + og * OC + o] = acc[a][o];
                } else {
#pragma unroll
                    for (int o = 0; o < OC; ++o) {
                        const float z = acc[a][o];
                        if (Z) Z[r * FO + og * OC + o] = z;
                        out[r * FO + og * OC + o] = (OT)(relu ? fmaxf(z, 0.f) : z);
                    }
                }
            }
        }
    }
}

// last layer (FO = 1): y = H w + AH u + b, one warp per 32 rows, FI features per row
__global__ void __launch_bounds__(256) k_dense_out(int64_t rows, int FI, const float *__restrict__ H,
                                                   const float *__restrict__ AH, const float *__restrict__ W,
                                                   const float *__restrict__ U, const float *__restrict__ b,
                                                   float *y) {
    __shared__ float sw[256], su[256];
    for (int k = threadIdx.x; k < FI; k += blockDim.x) { sw[k] = bf(W[k]); su[k] = bf(U[k]); }
    __syncthreads();
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float acc = bf(b[0]);
    for (int k = 0; k < FI; ++k) acc = fmaf(H[r * FI + k], sw[k], fmaf(AH[r * FI + k], su[k], acc));
    y[r] = acc;
}

// D = s_c (f0 + y)
__global__ void k_output(int64_t n, int p, const float *__restrict__ F, const float *__restrict__ y,
                         const float *__restrict__ scale, float *D) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    D[e] = scale[e % p] * (F[e * F0] + y[e]);
}

// the last layer at inference from its row products: y = H w + A (H u) + b, since A H u = (A H) u
// (A is linear): D = s_c (f0 + a + Aq + b) with a = H w and Aq = A (H u)
__global__ void k_output_dots(int64_t n, int p, const float *__restrict__ F, const float *__restrict__ a,
                              const float *__restrict__ Aq, const float *__restrict__ b,
                              const float *__restrict__ scale, float *D) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    D[e] = scale[e % p] * (F[e * F0] + (a[e] + Aq[e] + bf(b[0])));
}

// row products a = H w and q = H u of a rows x FI activation (weights rounded to bfloat16)
template <int FI>
__global__ void __launch_bounds__(256) k_rowdots(int64_t rows, const float *__restrict__ H, const float *__restrict__ w,
                                                 const float *__restrict__ u, float *a, float *q) {
    __shared__ float sw[FI], su[FI];
    for (int k = threadIdx.x; k < FI; k += blockDim.x) { sw[k] = bf(w[k]); su[k] = bf(u[k]); }
    __syncthreads();
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float x = 0.f, y = 0.f;
#pragma unroll 8
    for (int k = 0; k < FI; ++k) {
        const float h = H[r * FI + k];
        x = fmaf(h, sw[k], x);
        y = fmaf(h, su[k], y);
    }
    a[r] = x;
    q[r] = y;
}

// loss pieces: num[c] = sum (D - D*)^2, den[c] = sum D*^2 (float64), as per-block column partials
__global__ void __launch_bounds__(256) k_loss(int64_t n, int p, const float *__restrict__ D, const float *__restrict__ Ds,
                                              double *acc) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t S = (int64_t)gridDim.x * blockDim.x / p * p;
    double a = 0.0, b = 0.0;
    for (int64_t e = gid; gid < S && e < n * p; e += S) {
        const double r = (double)D[e] - (double)Ds[e];
        a += r * r;
        b += (double)Ds[e] * (double)Ds[e];
    }
    // per-block column partials, added in block order by launch_col_fin
    col_partial(a, gid < S, p, p, acc);
    col_partial(b, gid < S, p, p, acc + (int64_t)p * gridDim.x);
}

// dL/dy = 2 s_c (D - D*) / den_c / p
__global__ void k_dy(int64_t n, int p, const float *__restrict__ D, const float *__restrict__ Ds,
                     const float *__restrict__ scale, const double *__restrict__ acc, float *dy) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    const int c = (int)(e % p);
    dy[e] = (float)(2.0 * (double)scale[c] * ((double)D[e] - (double)Ds[e]) / acc[p + c] / p);
}

// Energy-norm loss (learned_loss = 1): with E = D - D* and TE = L E / 2 - lam_c B E for the
// columns of negative shift lam_c, num[c] = sum E TE and den[c] = sum G D* (= ||D*||_T^2, since
// T D* = G) as per-block column partials; TE goes to TEo.  Columns of non-negative shift (T = I,
// never preconditioned by the network) contribute nothing.
__global__ void __launch_bounds__(256) k_energy_terms(int64_t n, int p, const float *__restrict__ D,
                                                      const float *__restrict__ Ds, const float *__restrict__ LE,
                                                      const float *__restrict__ BE, const float *__restrict__ G,
                                                      const double *__restrict__ shift, float *TEo, double *acc) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t S = (int64_t)gridDim.x * blockDim.x / p * p;
    const int c = (int)(gid % p);
    const bool act = gid < S && shift[c] < 0.0;
    const float lam = act ? (float)shift[c] : 0.f;
    double a = 0.0, b = 0.0;
    for (int64_t e = gid; gid < S && e < n * p; e += S) {
        const float te = act ? 0.5f * LE[e] - lam * BE[e] : 0.f;
        TEo[e] = te;
        if (act) {
            a += (double)(D[e] - Ds[e]) * (double)te;
            b += (double)G[e] * (double)Ds[e];
        }
    }
    col_partial(a, gid < S, p, p, acc);
    col_partial(b, gid < S, p, p, acc + (int64_t)p * gridDim.x);
}

// dL/dy = 2 s_c TE / den_c / n_act on the columns with den_c > 0 (the active ones), 0 elsewhere
__global__ void k_dy_energy(int64_t n, int p, const float *__restrict__ TE, const float *__restrict__ scale,
                            const double *__restrict__ acc, float *dy) {
    __shared__ int nact;
    if (threadIdx.x == 0) {
        int k = 0;
        for (int c = 0; c < p; ++c) k += acc[p + c] > 0.0;
        nact = k;
    }
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    const int c = (int)(e % p);
    const double den = acc[p + c];
    dy[e] = den > 0.0 ? (float)(2.0 * (double)scale[c] * (double)TE[e] / den / nact) : 0.f;
}

__global__ void k_sub(int64_t m, const float *__restrict__ a, const float *__restrict__ b, float *o) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) o[i] = a[i] - b[i];
}

// dZ = dH * (Z > 0) in place (hidden layers)
__global__ void k_relu_back(int64_t m, const float *__restrict__ Z, float *dH) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < m && !(Z[e] > 0.f)) dH[e] = 0.f;
}

// gW += H^T dZ (FI x FO), gU += AH^T dZ, gb += sum dZ: row chunks per block, float64 atomics
template <int FI, int FO>
__global__ void __launch_bounds__(256) k_wgrad(int64_t rows, const float *__restrict__ H, const float *__restrict__ AH,
                                               const float *__restrict__ dZ, double *gW, double *gU, double *gb) {
    constexpr int NW = (FI * FO + 255) / 256;
    constexpr int RB = 32;
    __shared__ float sH[RB * FI], sA[RB * FI], sZ[RB * FO];
    float aW[NW], aU[NW], aB = 0.f;
#pragma unroll
    for (int q = 0; q < NW; ++q) { aW[q] = 0.f; aU[q] = 0.f; }
    for (int64_t r0 = blockIdx.x * (int64_t)RB; r0 < rows; r0 += (int64_t)RB * gridDim.x) {
        __syncthreads();
        for (int k = threadIdx.x; k < RB * FI; k += 256) {
            const int64_t r = r0 + k / FI;
            sH[k] = r < rows ? H[r0 * FI + k] : 0.f;
            sA[k] = r < rows ? AH[r0 * FI + k] : 0.f;
        }
        for (int k = threadIdx.x; k < RB * FO; k += 256) {
            const int64_t r = r0 + k / FO;
            sZ[k] = r < rows ? dZ[r0 * FO + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int o = threadIdx.x + 256 * q;
            if (o >= FI * FO) continue;
            const int fi = o / FO, fo = o - fi * FO;
            float w = aW[q], u = aU[q];
            for (int r = 0; r < RB; ++r) {
                const float z = sZ[r * FO + fo];
                w = fmaf(sH[r * FI + fi], z, w);
                u = fmaf(sA[r * FI + fi], z, u);
            }
            aW[q] = w; aU[q] = u;
        }
        if (threadIdx.x < FO)
            for (int r = 0; r < RB; ++r) aB += sZ[r * FO + threadIdx.x];
    }
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int o = threadIdx.x + 256 * q;
        if (o >= FI * FO) continue;
        atomicAdd(gW + o, (double)aW[q]);
        atomicAdd(gU + o, (double)aU[q]);
    }
    if (threadIdx.x < FO) atomicAdd(gb + threadIdx.x, (double)aB);
}

// dH = dZ W^T (into out), dAH = dZ U^T (into out2): rows x FI from rows x FO
template <int FI, int FO>
__global__ void __launch_bounds__(256) k_dinput(int64_t rows, const float *__restrict__ dZ, const float *__restrict__ W,
                                                const float *__restrict__ U, float *dH, float *dAH) {
    __shared__ float sW[FI * FO], sU[FI * FO];
    for (int k = threadIdx.x; k < FI * FO; k += 256) { sW[k] = bf(W[k]); sU[k] = bf(U[k]); }
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * FI) return;
    const int64_t r = e / FI;
    const int fi = (int)(e - r * FI);
    float a = 0.f, b = 0.f;
    for (int o = 0; o < FO; ++o) {
        const float z = dZ[r * FO + o];
        a = fmaf(z, sW[fi * FO + o], a);
        b = fmaf(z, sU[fi * FO + o], b);
    }
    dH[e] = a;
    dAH[e] = b;
}

__global__ void k_add(int64_t m, const float *__restrict__ a, float *b) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < m) b[e] += a[e];
}

// Adam on the flat parameter vector
__global__ void k_adam(int64_t m, const double *__restrict__ g, float *w, float *mo, float *ve, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float gi = (float)g[i];
    const float mi = b1 * mo[i] + (1.f - b1) * gi;
    const float vi = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = mi; ve[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// n x ld block (element type E) <-> n x p compact float; column k of the compact block is column
// cmap[k] of the block (k without a map)
template <class E>
__global__ void k_pack(int64_t n, int p, int ld, const int *__restrict__ cmap, const E *__restrict__ src, float *dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    const int64_t i = e / p;
    const int k = (int)(e - i * p);
    dst[e] = (float)src[i * ld + (cmap ? cmap[k] : k)];
}
template <class E>
__global__ void k_unpack(int64_t n, int p, int ld, const int *__restrict__ cmap, const float *__restrict__ src, E *dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * p) return;
    const int64_t i = e / p;
    const int k = (int)(e - i * p);
    dst[i * ld + (cmap ? cmap[k] : k)] = (E)src[e];
}

inline unsigned gr(int64_t m) { return (unsigned)std::max<int64_t>(1, (m + 255) / 256); }
inline unsigned gr_stride(int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 152 * 8)); }

// out = A in for bfloat16 activations of rowlen values per node (rowlen a multiple of 8), float32
// accumulation: one warp per (SELL slot, 256-value piece of the row); each lane owns 8 values
// (one 16-byte load per neighbour).  The neighbours come from the slot's SELL entries; padding
// entries have A = 0 and are skipped.
__global__ void __launch_bounds__(256) k_agg_bf16(int64_t n_slices, int rowlen, const int *__restrict__ slice_ptr,
                                                  const int *__restrict__ slice_w, const int *__restrict__ cols,
                                                  const int *__restrict__ perm, const float *__restrict__ val,
                                                  const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *out) {
    const int nchunk = (rowlen + 255) / 256;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n_slices * SELL_C * nchunk) return;
    const int64_t slot = gw / nchunk;
    const int ch = (int)(gw - slot * nchunk);
    const int64_t sl = slot / SELL_C;
    const int l = (int)(slot - sl * SELL_C);
    const int r = perm[slot];
    if (r < 0) return;                                   // the whole warp shares the slot
    const int k0 = ch * 256 + lane * 8;
    const bool own = k0 < rowlen;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int base = slice_ptr[sl], width = slice_w[sl];
    // four neighbours per pass, their loads issued before the multiply-adds (padding entries have
    // A = 0 and a valid column, so they are read and add nothing)
    const int kk = own ? k0 : 0;
    int j = 0;
    for (; j + 4 <= width; j += 4) {
        float a[4];
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = base + (j + u) * SELL_C + l;
            a[u] = __ldg(val + e);
            v[u] = __ldg(reinterpret_cast<const uint4 *>(in + (int64_t)__ldg(cols + e) * rowlen + kk));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v[u]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                acc[2 * i] = fmaf(a[u], f.x, acc[2 * i]);
                acc[2 * i + 1] = fmaf(a[u], f.y, acc[2 * i + 1]);
            }
        }
    }
    for (; j < width; ++j) {
        const int e = base + j * SELL_C + l;
        const float a = __ldg(val + e);
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in + (int64_t)__ldg(cols + e) * rowlen + kk));
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(h[i]);
            acc[2 * i] = fmaf(a, f.x, acc[2 * i]);
            acc[2 * i + 1] = fmaf(a, f.y, acc[2 * i + 1]);
        }
    }
    if (own) {
        uint4 o;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(acc[2 * i], acc[2 * i + 1]);
        *reinterpret_cast<uint4 *>(out + (int64_t)r * rowlen + k0) = o;
    }
}

}  // namespace

// layer dimensions for width H
static void dims(int H, int d[4]) { d[0] = F0; d[1] = H; d[2] = H; d[3] = 1; }

int64_t gcn_param_count(int H) {
    int d[4];
    dims(H, d);
    int64_t m = 0;
    for (int l = 0; l < 3; ++l) m += 2LL * d[l] * d[l + 1] + d[l + 1];
    return m;
}

// offsets of W_l, U_l, b_l in the flat vector
static void offsets(int H, int64_t off[3][3]) {
    int d[4];
    dims(H, d);
    int64_t o = 0;
    for (int l = 0; l < 3; ++l) {
        off[l][0] = o; o += (int64_t)d[l] * d[l + 1];
        off[l][1] = o; o += (int64_t)d[l] * d[l + 1];
        off[l][2] = o; o += d[l + 1];
    }
}

void gcn_free(ofks_ctx *c) {
    GcnState &g = c->gcn;
    for (float *q : {g.w, g.m, g.v, g.valA, g.valAT, g.F, g.H1, g.H2, g.Z1, g.Z2, g.AH, g.y, g.scale, g.Dn,
                     g.Ds, g.dA, g.dB2, g.G32, g.valL32, g.valB32, g.colf})
        if (q) cudaFree(q);
    for (double *q : {g.grad, g.stats, g.lacc}) if (q) cudaFree(q);
    c->gcn = GcnState{};
}

// aggregation values on the SELL pattern: A_ij = 1/|N(i)|, (A^T)_ij = 1/|N(j)|
__global__ void k_agg_values(int n_slices, const int *__restrict__ slice_ptr, const int *__restrict__ slice_w,
                             const int *__restrict__ cols, const int *__restrict__ perm, const double *__restrict__ valL,
                             const int *__restrict__ deg, float *valA, float *valAT) {
    const int s = blockIdx.x, lane = threadIdx.x;
    if (s >= n_slices || lane >= SELL_C) return;
    const int r = perm[s * SELL_C + lane];
    for (int j = 0; j < slice_w[s]; ++j) {
        const int e = slice_ptr[s] + j * SELL_C + lane;
        const bool real = r >= 0 && j < deg[r];
        valA[e] = real ? 1.f / (float)deg[r] : 0.f;
        valAT[e] = real ? 1.f / (float)deg[cols[e]] : 0.f;
    }
}

int gcn_setup(ofks_ctx *c, int H, uint64_t seed, const std::vector<int> &deg) {
    gcn_free(c);
    GcnState &g = c->gcn;
    g.H = H;
    const int64_t m = gcn_param_count(H);
    std::vector<float> w(m, 0.f);
    int64_t off[3][3];
    offsets(H, off);
    int d[4];
    dims(H, d);
    uint64_t st = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto gauss = [&]() {   // Box-Muller on a 64-bit LCG (weights only need to be reproducible)
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        const double u1 = ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        const double u2 = ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int l = 0; l < 2; ++l) {
        const double sc = std::sqrt(2.0 / (2.0 * d[l]));
        for (int64_t k = 0; k < (int64_t)d[l] * d[l + 1]; ++k) {
            w[off[l][0] + k] = (float)(sc * gauss());
            w[off[l][1] + k] = (float)(sc * gauss());
        }
    }
    auto alloc = [&](float **q, int64_t cnt) { return cudaMalloc((void **)q, sizeof(float) * std::max<int64_t>(cnt, 1)); };
    if (alloc(&g.w, m) || alloc(&g.m, m) || alloc(&g.v, m) ||
        cudaMalloc((void **)&g.grad, sizeof(double) * m) != cudaSuccess ||
        alloc(&g.valA, c->sell_len) || alloc(&g.valAT, c->sell_len))
        return ofks_fail(c, OFKS_ENOMEM, "learned preconditioner: parameters");
    cudaMemcpy(g.w, w.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
    cudaMemset(g.m, 0, sizeof(float) * m);
    cudaMemset(g.v, 0, sizeof(float) * m);
    int *d_deg = nullptr;
    if (cudaMalloc((void **)&d_deg, sizeof(int) * deg.size()) != cudaSuccess)
        return ofks_fail(c, OFKS_ENOMEM, "learned preconditioner: degrees");
    cudaMemcpy(d_deg, deg.data(), sizeof(int) * deg.size(), cudaMemcpyHostToDevice);
    k_agg_values<<<c->n_slices, SELL_C, 0, c->stream>>>(c->n_slices, c->d_slice_ptr, c->d_slice_w, c->d_cols, c->d_perm,
                                                        c->d_valL, d_deg, g.valA, g.valAT);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(d_deg);
    g.t = 0;
    return ofks_cuda_check(c, e, "learned preconditioner setup");
}

// activations for the current p
static int gcn_buffers(ofks_ctx *c) {
    GcnState &g = c->gcn;
    const int64_t rows = c->n * (int64_t)c->p;
    if (g.rows == rows && g.F) return OFKS_OK;
    for (float **q : {&g.F, &g.H1, &g.H2, &g.Z1, &g.Z2, &g.AH, &g.y, &g.scale, &g.Dn, &g.Ds, &g.dA, &g.dB2, &g.G32,
                      &g.colf}) {
        if (*q) cudaFree(*q);
        *q = nullptr;
    }
    for (double **q : {&g.stats, &g.lacc}) { if (*q) cudaFree(*q); *q = nullptr; }
    const int H = g.H;
    auto alloc = [&](float **q, int64_t cnt) { return cudaMalloc((void **)q, sizeof(float) * std::max<int64_t>(cnt, 1)); };
    if (alloc(&g.F, rows * F0) || alloc(&g.H1, rows * H) || alloc(&g.H2, rows * H) || alloc(&g.Z1, rows * H) ||
        alloc(&g.Z2, rows * H) || alloc(&g.AH, rows * H) || alloc(&g.y, rows) || alloc(&g.scale, c->p) ||
        alloc(&g.Dn, rows) || alloc(&g.Ds, rows) || alloc(&g.dA, rows * H) ||
        alloc(&g.dB2, rows * H) || alloc(&g.G32, rows) ||
        alloc(&g.colf, 3 * 256) ||
        cudaMalloc((void **)&g.stats, sizeof(double) * 2 * c->p) != cudaSuccess ||
        cudaMalloc((void **)&g.lacc, sizeof(double) * 2 * c->p) != cudaSuccess)
    {
        cudaGetLastError();                    // the failed allocation's error is reported here, once
        for (float **q : {&g.F, &g.H1, &g.H2, &g.Z1, &g.Z2, &g.AH, &g.y, &g.scale, &g.Dn, &g.Ds, &g.dA, &g.dB2,
                          &g.G32, &g.colf}) {
            if (*q) cudaFree(*q);
            *q = nullptr;
        }
        for (double **q : {&g.stats, &g.lacc}) { if (*q) cudaFree(*q); *q = nullptr; }
        g.rows = 0;
        return ofks_fail(c, OFKS_ENOMEM, "learned preconditioner: activations for %lld rows", (long long)rows);
    }
    g.rows = rows;
    return OFKS_OK;
}

int gcn_forward_prepare(ofks_ctx *c) { return gcn_buffers(c); }

// aggregation over nodes of an (n p) x F activation: out = A in (or A^T in)
static void aggregate(ofks_ctx *c, const float *val, const float *in, float *out, int F) {
    launch_sell_spmm_ld<float>(c, val, in, out, gcn_cols(c) * F);
}

#define DISPATCH_DENSE(FI_, FO_, ...)                                                              \
    do {                                                                                         \
        if (FI_ == 4 && FO_ == 64) { constexpr int A_ = 4, B_ = 64; __VA_ARGS__; }               \
        else if (FI_ == 64 && FO_ == 64) { constexpr int A_ = 64, B_ = 64; __VA_ARGS__; }        \
        else if (FI_ == 4 && FO_ == 32) { constexpr int A_ = 4, B_ = 32; __VA_ARGS__; }          \
        else if (FI_ == 32 && FO_ == 32) { constexpr int A_ = 32, B_ = 32; __VA_ARGS__; }        \
        else if (FI_ == 4 && FO_ == 16) { constexpr int A_ = 4, B_ = 16; __VA_ARGS__; }          \
        else if (FI_ == 16 && FO_ == 16) { constexpr int A_ = 16, B_ = 16; __VA_ARGS__; }        \
        else if (FI_ == 4 && FO_ == 8) { constexpr int A_ = 4, B_ = 8; __VA_ARGS__; }            \
        else { constexpr int A_ = 8, B_ = 8; __VA_ARGS__; }                                      \
    } while (0)

// forward on G32 (n x p float32, column-major-by-row layout (i, c)) -> g.Dn
int gcn_forward(ofks_ctx *c, const double *shift, bool keep) {
    GcnState &g = c->gcn;
    int rc = gcn_buffers(c);
    if (rc) return rc;
    const int64_t n = c->n, p = gcn_cols(c), rows = n * p;
    const int H = g.H;
    int64_t off[3][3];
    offsets(H, off);
    ProfScope ps(c, PF_GCN);
    {
        const unsigned gs = gr_stride(rows);
        k_feat_stats<<<gs, 256, 0, c->stream>>>(n, (int)p, g.G32, c->d_dL, c->d_dB, shift, c->d_cpart);
        launch_col_fin(c, (int)(2 * p), (int)(2 * p), gs, c->d_cpart, g.stats);
    }
    k_col_scales<<<1, 256, 0, c->stream>>>(n, (int)p, g.stats, shift, g.colf, g.scale);
    k_features<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, g.G32, c->d_dL, c->d_dB, g.colf, g.F);
    // layer 0: F (4) -> H1
    aggregate(c, g.valA, g.F, g.AH, F0);
    const unsigned gd = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 15) / 16, 152LL * 8));
    if (!keep && H == 64 && c->prm.learned_tc) {
        // inference on the tensor cores, which take bf16 operands: H1 and A H1 are kept in bf16
        // (half the bytes of the width-64p aggregation, the network's largest data movement)
        __nv_bfloat16 *H1b = reinterpret_cast<__nv_bfloat16 *>(g.H1), *AH1b = reinterpret_cast<__nv_bfloat16 *>(g.AH);
        k_dense<F0, 64, __nv_bfloat16><<<gd, 256, 0, c->stream>>>(rows, g.F, g.AH, g.w + off[0][0], g.w + off[0][1],
                                                                   g.w + off[0][2], 1, nullptr, H1b);
        const int rowlen = (int)(64 * p);
        const int64_t warps = (int64_t)c->n_slices * SELL_C * ((rowlen + 255) / 256);
        k_agg_bf16<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(
            c->n_slices, rowlen, c->d_slice_ptr, c->d_slice_w, c->d_cols, c->d_perm, g.valA, H1b, AH1b);
        float *a = g.y, *q = g.Ds, *Aq = g.Z1;
        launch_dense_tc_bf16(c, rows, H1b, AH1b, g.w + off[1][0], g.w + off[1][1], g.w + off[1][2], g.w + off[2][0],
                             g.w + off[2][1], a, q);
        launch_sell_spmm_ld<float>(c, g.valA, q, Aq, (int)p);
        k_output_dots<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, g.F, a, Aq, g.w + off[2][2], g.scale, g.Dn);
        c->kernels += 6;               // the aggregations, column sums and the tensor-core layer count themselves
        return ofks_cuda_check(c, cudaGetLastError(), "learned preconditioner forward");
    }
    DISPATCH_DENSE(F0, H, k_dense<A_, B_><<<gd, 256, 0, c->stream>>>(rows, g.F, g.AH, g.w + off[0][0], g.w + off[0][1],
                                                                      g.w + off[0][2], 1, nullptr, g.H1));
    // layer 1: H1 -> H2 (tensor cores for width 64 at inference; training keeps float32 activations)
    aggregate(c, g.valA, g.H1, g.AH, H);
    if (!keep) {
        // inference on the CUDA cores: the last layer needs H2 only through the row products
        // a = H2 w and q = H2 u (y = a + A q + b), so H2 is never aggregated (a width-p
        // aggregation instead of 64 p); the tensor-core path above forms a and q in its epilogue
        float *a = g.y, *q = g.Ds, *Aq = g.Z1;
        DISPATCH_DENSE(H, H, k_dense<A_, B_><<<gd, 256, 0, c->stream>>>(rows, g.H1, g.AH, g.w + off[1][0],
                                                                         g.w + off[1][1], g.w + off[1][2], 1, nullptr, g.H2));
        if (H == 64) k_rowdots<64><<<gr(rows), 256, 0, c->stream>>>(rows, g.H2, g.w + off[2][0], g.w + off[2][1], a, q);
        else if (H == 32) k_rowdots<32><<<gr(rows), 256, 0, c->stream>>>(rows, g.H2, g.w + off[2][0], g.w + off[2][1], a, q);
        else if (H == 16) k_rowdots<16><<<gr(rows), 256, 0, c->stream>>>(rows, g.H2, g.w + off[2][0], g.w + off[2][1], a, q);
        else k_rowdots<8><<<gr(rows), 256, 0, c->stream>>>(rows, g.H2, g.w + off[2][0], g.w + off[2][1], a, q);
        launch_sell_spmm_ld<float>(c, g.valA, q, Aq, (int)p);
        k_output_dots<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, g.F, a, Aq, g.w + off[2][2], g.scale, g.Dn);
        c->kernels += 7;
        return ofks_cuda_check(c, cudaGetLastError(), "learned preconditioner forward");
    }
    DISPATCH_DENSE(H, H, k_dense<A_, B_><<<gd, 256, 0, c->stream>>>(rows, g.H1, g.AH, g.w + off[1][0],
                                                                     g.w + off[1][1], g.w + off[1][2], 1, nullptr, g.H2));
    // layer 2: H2 -> y (A H2 kept in dA for the backward pass)
    aggregate(c, g.valA, g.H2, g.dA, H);
    k_dense_out<<<gr(rows), 256, 0, c->stream>>>(rows, H, g.H2, g.dA, g.w + off[2][0], g.w + off[2][1], g.w + off[2][2], g.y);
    k_output<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, g.F, g.y, g.scale, g.Dn);
    c->kernels += 7;
    return ofks_cuda_check(c, cudaGetLastError(), "learned preconditioner forward");
}

// loss of g.Dn against g.Ds and the parameter gradients in g.grad (float64)
int gcn_backward(ofks_ctx *c, const double *shift, double *loss) {
    GcnState &g = c->gcn;
    const int64_t n = c->n, p = gcn_cols(c), rows = n * p;
    const int H = g.H;
    int64_t off[3][3];
    offsets(H, off);
    const int64_t m = gcn_param_count(H);
    cudaMemsetAsync(g.grad, 0, sizeof(double) * m, c->stream);
    const bool energy = c->prm.learned_loss == 1;
    if (energy) {
        // T (D - D*) per column with float32 copies of L and B; scratch in Z2 (rows x H, H >= 3),
        // which the backward only fills later (dH2)
        if (!g.valL32) {
            if (cudaMalloc((void **)&g.valL32, sizeof(float) * c->sell_len) != cudaSuccess ||
                cudaMalloc((void **)&g.valB32, sizeof(float) * c->sell_len) != cudaSuccess)
                return ofks_fail(c, OFKS_ENOMEM, "learned preconditioner: float32 L and B");
            launch_convert<double, float>(c, c->d_valL, g.valL32, c->sell_len);
            launch_convert<double, float>(c, c->d_valB, g.valB32, c->sell_len);
        }
        float *E = g.Z2, *LE = g.Z2 + rows, *BE = g.Z2 + 2 * rows;
        k_sub<<<gr(rows), 256, 0, c->stream>>>(rows, g.Dn, g.Ds, E);
        launch_sell_spmm_ld<float>(c, g.valL32, E, LE, (int)p);
        launch_sell_spmm_ld<float>(c, g.valB32, E, BE, (int)p);
        const unsigned gs = gr_stride(rows);
        k_energy_terms<<<gs, 256, 0, c->stream>>>(n, (int)p, g.Dn, g.Ds, LE, BE, g.G32, shift, E, c->d_cpart);
        launch_col_fin(c, (int)(2 * p), (int)(2 * p), gs, c->d_cpart, g.lacc);
        k_dy_energy<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, E, g.scale, g.lacc, g.y);  // g.y <- dL/dy
        c->kernels += 5;
    } else {
        const unsigned gs = gr_stride(rows);
        k_loss<<<gs, 256, 0, c->stream>>>(n, (int)p, g.Dn, g.Ds, c->d_cpart);
        launch_col_fin(c, (int)(2 * p), (int)(2 * p), gs, c->d_cpart, g.lacc);
        k_dy<<<gr(rows), 256, 0, c->stream>>>(n, (int)p, g.Dn, g.Ds, g.scale, g.lacc, g.y);   // g.y <- dL/dy
    }
    const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 31) / 32, 152LL * 4));
    // layer 2 (H -> 1): dZ = dy; grads; dH2 = dy w^T, dAH2 = dy u^T
    if (H == 64) k_wgrad<64, 1><<<gw, 256, 0, c->stream>>>(rows, g.H2, g.dA, g.y, g.grad + off[2][0], g.grad + off[2][1], g.grad + off[2][2]);
    else if (H == 32) k_wgrad<32, 1><<<gw, 256, 0, c->stream>>>(rows, g.H2, g.dA, g.y, g.grad + off[2][0], g.grad + off[2][1], g.grad + off[2][2]);
    else if (H == 16) k_wgrad<16, 1><<<gw, 256, 0, c->stream>>>(rows, g.H2, g.dA, g.y, g.grad + off[2][0], g.grad + off[2][1], g.grad + off[2][2]);
    else k_wgrad<8, 1><<<gw, 256, 0, c->stream>>>(rows, g.H2, g.dA, g.y, g.grad + off[2][0], g.grad + off[2][1], g.grad + off[2][2]);
    const unsigned gi = gr(rows * H);
    if (H == 64) k_dinput<64, 1><<<gi, 256, 0, c->stream>>>(rows, g.y, g.w + off[2][0], g.w + off[2][1], g.Z2 /*dH2*/, g.dB2);
    else if (H == 32) k_dinput<32, 1><<<gi, 256, 0, c->stream>>>(rows, g.y, g.w + off[2][0], g.w + off[2][1], g.Z2, g.dB2);
    else if (H == 16) k_dinput<16, 1><<<gi, 256, 0, c->stream>>>(rows, g.y, g.w + off[2][0], g.w + off[2][1], g.Z2, g.dB2);
    else k_dinput<8, 1><<<gi, 256, 0, c->stream>>>(rows, g.y, g.w + off[2][0], g.w + off[2][1], g.Z2, g.dB2);
    // dH2 += A^T dAH2
    aggregate(c, g.valAT, g.dB2, g.AH, H);
    k_add<<<gr(rows * H), 256, 0, c->stream>>>(rows * H, g.AH, g.Z2);
    // layer 1 (H -> H): dZ1' = dH2 * (Z of layer 1 > 0); Z of layer 1 is g.H2's pre-activation: recompute mask from H2
    k_relu_back<<<gr(rows * H), 256, 0, c->stream>>>(rows * H, g.H2, g.Z2);      // H2 = relu(Z): H2 > 0 <=> Z > 0
    aggregate(c, g.valA, g.H1, g.AH, H);                                         // A H1 again
    DISPATCH_DENSE(H, H, k_wgrad<A_, B_><<<gw, 256, 0, c->stream>>>(rows, g.H1, g.AH, g.Z2, g.grad + off[1][0],
                                                                     g.grad + off[1][1], g.grad + off[1][2]));
    DISPATCH_DENSE(H, H, k_dinput<A_, B_><<<gr(rows * H), 256, 0, c->stream>>>(rows, g.Z2, g.w + off[1][0], g.w + off[1][1],
                                                                                g.dA, g.dB2));
    aggregate(c, g.valAT, g.dB2, g.AH, H);
    k_add<<<gr(rows * H), 256, 0, c->stream>>>(rows * H, g.AH, g.dA);             // dH1
    // layer 0 (4 -> H)
    k_relu_back<<<gr(rows * H), 256, 0, c->stream>>>(rows * H, g.H1, g.dA);
    aggregate(c, g.valA, g.F, g.AH, F0);
    DISPATCH_DENSE(F0, H, k_wgrad<A_, B_><<<gw, 256, 0, c->stream>>>(rows, g.F, g.AH, g.dA, g.grad + off[0][0],
                                                                      g.grad + off[0][1], g.grad + off[0][2]));
    c->kernels += 18;
    double h[2 * 256];
    const int pp = (int)std::min<int64_t>(p, 256);
    cudaError_t e = cudaMemcpyAsync(h, g.lacc, sizeof(double) * 2 * pp, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "learned preconditioner backward");
    double L = 0.0;
    int na = 0;
    for (int k = 0; k < pp; ++k)
        if (!energy || h[pp + k] > 0.0) { L += h[k] / h[pp + k]; ++na; }
    *loss = na ? L / na : 0.0;
    return OFKS_OK;
}

int gcn_adam(ofks_ctx *c, double lr) {
    GcnState &g = c->gcn;
    const int64_t m = gcn_param_count(g.H);
    g.t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)g.t), c2 = 1.f - std::pow(b2, (float)g.t);
    k_adam<<<gr(m), 256, 0, c->stream>>>(m, g.grad, g.w, g.m, g.v, (float)lr, b1, b2, c1, c2, 1e-8f);
    c->kernels += 1;
    return ofks_cuda_check(c, cudaGetLastError(), "Adam");
}

template <class E>
void gcn_pack(ofks_ctx *c, const E *src, float *dst, const int *cmap) {
    const int cols = gcn_cols(c);
    k_pack<E><<<gr(c->n * (int64_t)cols), 256, 0, c->stream>>>(c->n, cols, c->ld, cmap, src, dst);
    c->kernels += 1;
}
template <class E>
void gcn_unpack(ofks_ctx *c, const float *src, E *dst, const int *cmap) {
    const int cols = gcn_cols(c);
    k_unpack<E><<<gr(c->n * (int64_t)cols), 256, 0, c->stream>>>(c->n, cols, c->ld, cmap, src, dst);
    c->kernels += 1;
}
template void gcn_pack<double>(ofks_ctx *, const double *, float *, const int *);
template void gcn_pack<float>(ofks_ctx *, const float *, float *, const int *);
template void gcn_unpack<double>(ofks_ctx *, const float *, double *, const int *);
template void gcn_unpack<float>(ofks_ctx *, const float *, float *, const int *);
