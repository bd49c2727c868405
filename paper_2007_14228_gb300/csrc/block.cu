// Tall-skinny block kernels of one PCAL iteration (paper Alg. 2):
//   Grams X^T H X (Eq. multi) and X^T B X, the gradient grad L_beta = H X + B X C with
//   C = beta (S - I) - Lambda (Eq. PLAM-main), the residual H X - B X Lambda0 for kkt
//   (Sec. 4.1), the Jacobi-PCG vector updates of the preconditioner (Eq. precondition-T),
//   the Barzilai-Borwein inner products (Sec. 4.4), and the step/normalization of
//   Eq. (PCAL-main).  Blocks are row-major n x ld float64 with zero padding columns.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

enum { CB_SHIFT = 0, CB_ACTIVE = 1, CB_RZ = 2, CB_RZN = 3, CB_PQ = 4, CB_BETA = 5, CB_NORM = 6,
       CB_ALPHA = 7, CB_COUNT = 8 };

namespace {

// ---------------------------------------------------------------- Grams (upper tiles)
// XA = X^T A and XB = X^T B over the rows of one split, for output tile (ti, tj), ti <= tj.
// 16 x 16 threads, each an RT x RT register tile; rows staged KR at a time in shared memory.
template <int RT>
__global__ void __launch_bounds__(256) k_gram2(int64_t n, int p, int ld, int ntile,
                                               const double *__restrict__ X,
                                               const double *__restrict__ A,
                                               const double *__restrict__ B, double *XA, double *XB,
                                               int64_t rows_per_split) {
    constexpr int TS = 16 * RT, KR = 16;
    __shared__ double xs[KR][TS], as[KR][TS], bs[KR][TS];
    // decode the upper-triangular tile pair
    int pair = blockIdx.x, ti = 0;
    while (pair >= ntile - ti) { pair -= ntile - ti; ++ti; }
    const int tj = ti + pair;
    const int i0 = ti * TS, j0 = tj * TS;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = blockIdx.y * rows_per_split;
    const int64_t r1 = (r0 + rows_per_split < n) ? r0 + rows_per_split : n;
    double ca[RT][RT], cb[RT][RT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < RT; ++b) { ca[a][b] = 0.0; cb[a][b] = 0.0; }
    for (int64_t rb = r0; rb < r1; rb += KR) {
        for (int idx = threadIdx.x; idx < KR * TS; idx += 256) {
            const int rr = idx / TS, cc = idx % TS;
            const int64_t r = rb + rr;
            const bool okr = r < r1;
            xs[rr][cc] = (okr && i0 + cc < ld) ? X[r * ld + i0 + cc] : 0.0;
            as[rr][cc] = (okr && j0 + cc < ld) ? A[r * ld + j0 + cc] : 0.0;
            bs[rr][cc] = (okr && j0 + cc < ld) ? B[r * ld + j0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KR; ++k) {
            double xv[RT], av[RT], bv[RT];
#pragma unroll
            for (int a = 0; a < RT; ++a) xv[a] = xs[k][ty * RT + a];
#pragma unroll
            for (int b = 0; b < RT; ++b) { av[b] = as[k][tx * RT + b]; bv[b] = bs[k][tx * RT + b]; }
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    ca[a][b] = fma(xv[a], av[b], ca[a][b]);
                    cb[a][b] = fma(xv[a], bv[b], cb[a][b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < RT; ++b) {
            const int i = i0 + ty * RT + a, j = j0 + tx * RT + b;
            if (i < p && j < p && i <= j) {
                atomicAdd(XA + (int64_t)i * ld + j, ca[a][b]);
                atomicAdd(XB + (int64_t)i * ld + j, cb[a][b]);
            }
        }
}

__global__ void k_mirror2(int p, int ld, double *A, double *B) {
    for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < p * p; idx += blockDim.x * gridDim.x) {
        const int i = idx / p, j = idx % p;
        if (i > j) {
            A[(int64_t)i * ld + j] = A[(int64_t)j * ld + i];
            B[(int64_t)i * ld + j] = B[(int64_t)j * ld + i];
        }
    }
}

// ---------------------------------------------------------------- gradient and residual
// G = HX + BX C ;  kkt2 += ||HX - BX L0||^2 (columns < p).  32 column lanes x 8 row groups;
// each thread owns 4 rows of a 32-row tile and MC columns; C, L0 staged in KC-row chunks.
template <int MC>
__global__ void __launch_bounds__(256) k_grad(int64_t n, int p, int ld, const double *__restrict__ HX,
                                              const double *__restrict__ BX,
                                              const double *__restrict__ C,
                                              const double *__restrict__ L0, double *G,
                                              double *kkt2, int KC) {
    extern __shared__ double smem[];
    double *bx = smem;                 // 32 x ld
    double *cs = bx + 32 * ld;         // KC x ld
    double *ls = cs + KC * ld;         // KC x ld
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
    double part = 0.0;
    for (int64_t rt = blockIdx.x * 32LL; rt < n; rt += 32LL * gridDim.x) {
        double g[4][MC], rr[4][MC];
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * ld; idx += 256) {
            const int64_t r = rt + idx / ld;
            bx[idx] = r < n ? BX[rt * ld + idx] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t r = rt + rg * 4 + a;
#pragma unroll
            for (int m = 0; m < MC; ++m) {
                const int j = lane + 32 * m;
                const double h = (r < n && j < ld) ? HX[r * ld + j] : 0.0;
                g[a][m] = h; rr[a][m] = h;
            }
        }
        for (int k0 = 0; k0 < ld; k0 += KC) {
            const int kl = min(KC, ld - k0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < kl * ld; idx += 256) {
                cs[idx] = C[(int64_t)k0 * ld + idx];
                ls[idx] = L0[(int64_t)k0 * ld + idx];
            }
            __syncthreads();
            for (int kk = 0; kk < kl; ++kk) {
                double b[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) b[a] = bx[(rg * 4 + a) * ld + k0 + kk];
#pragma unroll
                for (int m = 0; m < MC; ++m) {
                    const int j = lane + 32 * m;
                    const double cv = j < ld ? cs[kk * ld + j] : 0.0;
                    const double lv = j < ld ? ls[kk * ld + j] : 0.0;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        g[a][m] = fma(b[a], cv, g[a][m]);
                        rr[a][m] = fma(-b[a], lv, rr[a][m]);
                    }
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t r = rt + rg * 4 + a;
            if (r >= n) continue;
#pragma unroll
            for (int m = 0; m < MC; ++m) {
                const int j = lane + 32 * m;
                if (j < ld) G[r * ld + j] = g[a][m];
                if (j < p) part += rr[a][m] * rr[a][m];
            }
        }
    }
    part = block_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(kkt2, part);
}

// ---------------------------------------------------------------- row-parallel helpers
// Thread layout for n x ld elementwise work with per-column sums: 32 column lanes x 8 rows.
#define ROWLOOP_BEGIN                                                                          \
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;                                \
    for (int64_t r = blockIdx.x * 8LL + rg; r < n; r += 8LL * gridDim.x) {                    \
        _Pragma("unroll") for (int m = 0; m < MC; ++m) {                                     \
            const int j = lane + 32 * m;                                                     \
            if (j >= ld) continue;                                                           \
            const int64_t e = r * ld + j;
#define ROWLOOP_END } }

// add per-thread column partials (MC per thread) into colsum[j] over the block
template <int MC>
__device__ __forceinline__ void col_reduce(double (&acc)[MC], int ld, int p, double *colsum) {
    __shared__ double sh[8][32 * MC];
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < MC; ++m) sh[rg][lane + 32 * m] = acc[m];
    __syncthreads();
    for (int j = threadIdx.x; j < 32 * MC; j += blockDim.x) {
        if (j >= p) continue;
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += sh[g][j];
        atomicAdd(colsum + j, s);
    }
}

// PCG start: D = 0, R = G, Z = R / diag, rz[c] = sum R Z  (diag = dL/2 - shift_c dB)
template <int MC>
__global__ void __launch_bounds__(256) k_pcg_init(int64_t n, int p, int ld, const double *__restrict__ G,
                                                  const double *__restrict__ dL,
                                                  const double *__restrict__ dB, const double *cb,
                                                  double *D, double *R, double *Z, double *rz) {
    double acc[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) acc[m] = 0.0;
    ROWLOOP_BEGIN
        const double gv = G[e];
        const double dg = 0.5 * dL[r] - cb[CB_SHIFT * ld + j] * dB[r];
        const double z = gv / dg;
        D[e] = 0.0; R[e] = gv; Z[e] = z;
        acc[m] += gv * z;
    ROWLOOP_END
    col_reduce<MC>(acc, ld, p, rz);
}

// alpha = rz/pq; D += alpha P; R -= alpha Q; Z = R/diag; rzn += R Z
template <int MC>
__global__ void __launch_bounds__(256) k_pcg_update(int64_t n, int p, int ld, const double *__restrict__ dL,
                                                    const double *__restrict__ dB, const double *cb,
                                                    const double *__restrict__ P,
                                                    const double *__restrict__ Q, double *D, double *R,
                                                    double *Z, double *rzn) {
    double acc[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) acc[m] = 0.0;
    ROWLOOP_BEGIN
        const double al = cb[CB_ALPHA * ld + j];
        const double dg = 0.5 * dL[r] - cb[CB_SHIFT * ld + j] * dB[r];
        D[e] = fma(al, P[e], D[e]);
        const double rv = fma(-al, Q[e], R[e]);
        const double z = rv / dg;
        R[e] = rv; Z[e] = z;
        acc[m] += rv * z;
    ROWLOOP_END
    col_reduce<MC>(acc, ld, p, rzn);
}

// columns whose shift is not negative take D = G (T = I in Eq. precondition-T)
template <int MC>
__global__ void __launch_bounds__(256) k_select(int64_t n, int ld, const double *cb,
                                                const double *__restrict__ G, double *D) {
    ROWLOOP_BEGIN
        if (cb[CB_ACTIVE * ld + j] == 0.0) D[e] = G[e];
    ROWLOOP_END
}

// Barzilai-Borwein sums: <dX,dD>, <dD,dD>, <dX,dX>, and ||X||^2, ||D||^2
template <int MC>
__global__ void __launch_bounds__(256) k_bb(int64_t n, int ld, const double *__restrict__ X,
                                            const double *__restrict__ Xp, const double *__restrict__ D,
                                            const double *__restrict__ Dp, int have_prev, double *sc) {
    __shared__ double red[8];
    double sy = 0, yy = 0, ss = 0, xx = 0, dd = 0;
    {
        ROWLOOP_BEGIN
            const double x = X[e], d = D[e];
            xx += x * x; dd += d * d;
            if (have_prev) {
                const double sx = x - Xp[e], yd = d - Dp[e];
                sy += sx * yd; yy += yd * yd; ss += sx * sx;
            }
        ROWLOOP_END
    }
    sy = block_sum(sy, red); yy = block_sum(yy, red); ss = block_sum(ss, red);
    xx = block_sum(xx, red); dd = block_sum(dd, red);
    if (threadIdx.x == 0) {
        atomicAdd(sc + SC_BB + 0, sy); atomicAdd(sc + SC_BB + 1, yy); atomicAdd(sc + SC_BB + 2, ss);
        atomicAdd(sc + SC_XNRM2, xx); atomicAdd(sc + SC_DNRM2, dd);
    }
}

// Y = X - D / eta
template <int MC>
__global__ void __launch_bounds__(256) k_step(int64_t n, int ld, const double *__restrict__ X,
                                              const double *__restrict__ D, const double *sc,
                                              double *Y) {
    const double inv = 1.0 / sc[SC_ETA];
    ROWLOOP_BEGIN
        Y[e] = fma(-inv, D[e], X[e]);
    ROWLOOP_END
}

// X_i = Y_i / ||Y_i||_B and B X_i = B Y_i / ||Y_i||_B   (Eq. PCAL-main)
template <int MC>
__global__ void __launch_bounds__(256) k_scale(int64_t n, int p, int ld, const double *colsum,
                                               double *Y, double *BY) {
    ROWLOOP_BEGIN
        if (j < p) {
            const double s = 1.0 / sqrt(colsum[j]);
            Y[e] *= s; BY[e] *= s;
        }
    ROWLOOP_END
}

// Y = X M with M (ld x ld, zero padded) staged in KC-row chunks
template <int MC>
__global__ void __launch_bounds__(256) k_block_small(int64_t n, int ld, const double *__restrict__ X,
                                                     const double *__restrict__ M, double *Y, int KC) {
    extern __shared__ double smem[];
    double *xs = smem;                 // 32 x ld
    double *ms = xs + 32 * ld;         // KC x ld
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
    for (int64_t rt = blockIdx.x * 32LL; rt < n; rt += 32LL * gridDim.x) {
        double y[4][MC];
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * ld; idx += 256) {
            const int64_t r = rt + idx / ld;
            xs[idx] = r < n ? X[rt * ld + idx] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < MC; ++m) y[a][m] = 0.0;
        for (int k0 = 0; k0 < ld; k0 += KC) {
            const int kl = min(KC, ld - k0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < kl * ld; idx += 256) ms[idx] = M[(int64_t)k0 * ld + idx];
            __syncthreads();
            for (int kk = 0; kk < kl; ++kk) {
                double b[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) b[a] = xs[(rg * 4 + a) * ld + k0 + kk];
#pragma unroll
                for (int m = 0; m < MC; ++m) {
                    const int j = lane + 32 * m;
                    const double mv = j < ld ? ms[kk * ld + j] : 0.0;
#pragma unroll
                    for (int a = 0; a < 4; ++a) y[a][m] = fma(b[a], mv, y[a][m]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t r = rt + rg * 4 + a;
            if (r >= n) continue;
#pragma unroll
            for (int m = 0; m < MC; ++m) {
                const int j = lane + 32 * m;
                if (j < ld) Y[r * ld + j] = y[a][m];
            }
        }
    }
}

inline int mc_of(int ld) { return (ld + 31) / 32; }

inline unsigned row_grid(int64_t rows_per_block, int64_t n) {
    int64_t g = (n + rows_per_block - 1) / rows_per_block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152LL * 16));
}

inline int kc_of(int ld) { return ld <= 64 ? ld : 32; }

}  // namespace

#define MC_DISPATCH(MC_, ...)                                  \
    switch (MC_) {                                             \
        case 1: { constexpr int M_ = 1; __VA_ARGS__; } break;  \
        case 2: { constexpr int M_ = 2; __VA_ARGS__; } break;  \
        case 3: { constexpr int M_ = 3; __VA_ARGS__; } break;  \
        case 4: { constexpr int M_ = 4; __VA_ARGS__; } break;  \
        case 5: { constexpr int M_ = 5; __VA_ARGS__; } break;  \
        case 6: { constexpr int M_ = 6; __VA_ARGS__; } break;  \
        case 7: { constexpr int M_ = 7; __VA_ARGS__; } break;  \
        default: { constexpr int M_ = 8; __VA_ARGS__; } break; \
    }

void launch_gram2(ofks_ctx *c, const double *X, const double *A, const double *B, double *XA, double *XB) {
    ProfScope ps(c, PF_GRAM);
    const int ld = c->ld, p = c->p;
    cudaMemsetAsync(XA, 0, sizeof(double) * ld * ld, c->stream);
    cudaMemsetAsync(XB, 0, sizeof(double) * ld * ld, c->stream);
    int RT = p <= 16 ? 1 : (p <= 32 ? 2 : (p <= 48 ? 3 : 4));
    const int TS = 16 * RT, ntile = (p + TS - 1) / TS, npair = ntile * (ntile + 1) / 2;
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, (152LL * 4) / npair + 1));
    const int64_t rps = ((c->n + splits - 1) / splits + 15) / 16 * 16;
    splits = (c->n + rps - 1) / rps;
    dim3 grid((unsigned)npair, (unsigned)splits);
#define G_(rt) k_gram2<rt><<<grid, 256, 0, c->stream>>>(c->n, p, ld, ntile, X, A, B, XA, XB, rps)
    switch (RT) { case 1: G_(1); break; case 2: G_(2); break; case 3: G_(3); break; default: G_(4); }
#undef G_
    k_mirror2<<<4, 256, 0, c->stream>>>(p, ld, XA, XB);
    c->kernels += 2;
}

void launch_grad_update(ofks_ctx *c) {
    c->kernels += 1;
    ProfScope ps(c, PF_GRAD);
    const int ld = c->ld, KC = kc_of(ld);
    const size_t sm = sizeof(double) * (32 * ld + 2 * KC * ld);
    double *G = c->d_G[c->cur];
    cudaMemsetAsync(c->d_sc + SC_KKT2, 0, sizeof(double), c->stream);
    const unsigned grid = row_grid(32, c->n);
    MC_DISPATCH(mc_of(ld), {
        cudaFuncSetAttribute(k_grad<M_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_grad<M_><<<grid, 256, sm, c->stream>>>(c->n, c->p, ld, c->d_HX, c->d_BX, c->d_C, c->d_L0, G,
                                                 c->d_sc + SC_KKT2, KC);
    });
}

void launch_pcg_init(ofks_ctx *c) {
    c->kernels += 1;
    const int ld = c->ld;
    double *cb = c->d_colA;
    cudaMemsetAsync(cb + CB_RZ * ld, 0, sizeof(double) * ld, c->stream);
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_pcg_init<M_><<<grid, 256, 0, c->stream>>>(
        c->n, c->p, ld, c->d_G[c->cur], c->d_dL, c->d_dB, cb, c->d_D[c->cur], c->d_R, c->d_Z, cb + CB_RZ * ld));
}

void launch_pcg_update(ofks_ctx *c, int) {
    c->kernels += 1;
    const int ld = c->ld;
    double *cb = c->d_colA;
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_pcg_update<M_><<<grid, 256, 0, c->stream>>>(
        c->n, c->p, ld, c->d_dL, c->d_dB, cb, c->d_P, c->d_Q, c->d_D[c->cur], c->d_R, c->d_Z,
        cb + CB_RZN * ld));
}

void launch_direction_select(ofks_ctx *c) {
    c->kernels += 1;
    const int ld = c->ld;
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_select<M_><<<grid, 256, 0, c->stream>>>(c->n, ld, c->d_colA, c->d_G[c->cur],
                                                                      c->d_D[c->cur]));
}

void launch_bb_dots(ofks_ctx *c) {
    c->kernels += 1;
    ProfScope ps(c, PF_BB);
    const int ld = c->ld, cur = c->cur, prv = cur ^ 1;
    cudaMemsetAsync(c->d_sc + SC_BB, 0, sizeof(double) * 3, c->stream);
    cudaMemsetAsync(c->d_sc + SC_XNRM2, 0, sizeof(double) * 2, c->stream);
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_bb<M_><<<grid, 256, 0, c->stream>>>(
        c->n, ld, c->d_X[cur], c->d_X[prv], c->d_D[cur], c->d_D[prv], c->have_prev ? 1 : 0, c->d_sc));
}

void launch_step_y(ofks_ctx *c, double *Y) {
    c->kernels += 1;
    const int ld = c->ld;
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_step<M_><<<grid, 256, 0, c->stream>>>(c->n, ld, c->d_X[c->cur], c->d_D[c->cur],
                                                                    c->d_sc, Y));
}

void launch_scale_cols(ofks_ctx *c, double *Y, double *BY, const double *colsum) {
    c->kernels += 1;
    const int ld = c->ld;
    const unsigned grid = row_grid(8, c->n);
    MC_DISPATCH(mc_of(ld), k_scale<M_><<<grid, 256, 0, c->stream>>>(c->n, c->p, ld, colsum, Y, BY));
}

void launch_block_times_small(ofks_ctx *c, const double *X, const double *M, double *Y) {
    c->kernels += 1;
    const int ld = c->ld, KC = kc_of(ld);
    const size_t sm = sizeof(double) * (32 * ld + KC * ld);
    const unsigned grid = row_grid(32, c->n);
    MC_DISPATCH(mc_of(ld), {
        cudaFuncSetAttribute(k_block_small<M_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_block_small<M_><<<grid, 256, sm, c->stream>>>(c->n, ld, X, M, Y, KC);
    });
}

void launch_tri_solve_rows(ofks_ctx *c, const double *V, double *X, const double *Rinv) {
    launch_block_times_small(c, V, Rinv, X);
}
