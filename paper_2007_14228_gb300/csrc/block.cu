// Tall-skinny block kernels of one PCAL iteration (paper Alg. 2):
//   Grams X^T H X (Eq. multi) and X^T B X, the gradient grad L_beta = H X + B X C with
//   C = beta (S - I) - Lambda (Eq. PLAM-main), the residual H X - B X Lambda0 for kkt
//   (Sec. 4.1), the Jacobi-PCG vector updates of the preconditioner (Eq. precondition-T),
//   the Barzilai-Borwein inner products (Sec. 4.4), and the step/normalization of
//   Eq. (PCAL-main).  Blocks are row-major n x ld (float64 or float32, T) with zero padding
//   columns; p x p matrices and every reduction are float64.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

// ---------------------------------------------------------------- Grams (upper tiles)
// XA = X^T A and XB = X^T B over the rows of one split, for output tile (ti, tj), ti <= tj.
// The tile is cut into RT x RT micro-tiles; only micro-tiles that hold entries i <= j < p are
// computed, numbered consecutively so that whole warps stay idle when there are fewer of them
// than threads (a float64 warp instruction costs the same however many lanes are active).
// Rows are staged KR at a time in shared memory.
// The block's partial tile (its split of the rows) goes to part, entry-major: the value of
// tile entry (m, a, b) of tile pair q at part[((q 2 + m) TS + a) TS + b) splits + split], and
// k_gram_fin adds the splits in order.
template <class T, int RT>
__global__ void __launch_bounds__(256) k_gram2(int64_t n, int p, int ld, int ntile,
                                               const T *__restrict__ X,
                                               const T *__restrict__ A,
                                               const T *__restrict__ B, double *part,
                                               int64_t rows_per_split) {
    constexpr int TS = 16 * RT, KR = 16;
    __shared__ T xs[KR][TS], as[KR][TS], bs[KR][TS];
    // decode the upper-triangular tile pair
    const int q = blockIdx.x;
    int pair = blockIdx.x, ti = 0;
    while (pair >= ntile - ti) { pair -= ntile - ti; ++ti; }
    const int tj = ti + pair;
    const int i0 = ti * TS, j0 = tj * TS;
    const int nbi = (min(TS, p - i0) + RT - 1) / RT, nbj = (min(TS, p - j0) + RT - 1) / RT;
    // this thread's micro-tile (bi, bj)
    int bi = 0, bj = 0;
    bool act;
    if (ti == tj) {                                     // upper triangle of micro-tiles
        int idx = threadIdx.x;
        act = idx < nbi * (nbi + 1) / 2;
        while (act && idx >= nbi - bi) { idx -= nbi - bi; ++bi; }
        bj = bi + idx;
    } else {
        act = (int)threadIdx.x < nbi * nbj;
        bi = threadIdx.x / nbj;
        bj = threadIdx.x - bi * nbj;
    }
    const int64_t r0 = blockIdx.y * rows_per_split;
    const int64_t r1 = (r0 + rows_per_split < n) ? r0 + rows_per_split : n;
    T ca[RT][RT], cb[RT][RT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < RT; ++b) { ca[a][b] = T(0); cb[a][b] = T(0); }
    for (int64_t rb = r0; rb < r1; rb += KR) {
        for (int idx = threadIdx.x; idx < KR * TS; idx += 256) {
            const int rr = idx / TS, cc = idx - rr * TS;
            const int64_t r = rb + rr;
            const bool okr = r < r1;
            xs[rr][cc] = (okr && i0 + cc < ld) ? X[r * ld + i0 + cc] : T(0);
            as[rr][cc] = (okr && j0 + cc < ld) ? A[r * ld + j0 + cc] : T(0);
            bs[rr][cc] = (okr && j0 + cc < ld) ? B[r * ld + j0 + cc] : T(0);
        }
        __syncthreads();
        if (act)
#pragma unroll 4
        for (int k = 0; k < KR; ++k) {
            T xv[RT], av[RT], bv[RT];
#pragma unroll
            for (int a = 0; a < RT; ++a) xv[a] = xs[k][bi * RT + a];
#pragma unroll
            for (int b = 0; b < RT; ++b) { av[b] = as[k][bj * RT + b]; bv[b] = bs[k][bj * RT + b]; }
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
    if (!act) return;
    const int64_t S = gridDim.y;
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < RT; ++b) {
            const int la = bi * RT + a, lb = bj * RT + b, i = i0 + la, j = j0 + lb;
            if (i < p && j < p && i <= j) {
                part[(((int64_t)q * 2 * TS + la) * TS + lb) * S + blockIdx.y] = (double)ca[a][b];
                part[((((int64_t)q * 2 + 1) * TS + la) * TS + lb) * S + blockIdx.y] = (double)cb[a][b];
            }
        }
}

// Float32 Grams for 64 < ld <= 256 (where the tensor-core form's operands no longer fit): one CTA
// per (upper 64 x 64 tile pair (i, j), range of rows).  Rows arrive 32 at a time as float4 loads
// into registers while the previous 32 are multiplied from shared memory; a thread keeps a 4 x 4
// tile of X^T A and of X^T B: per row one float4 of X, A and B feed 32 FMAs.  Partial tiles are
// added to the float64 outputs (upper triangle i <= j < p) at the end.
constexpr int GM_T = 64, GM_KR = 32;

__global__ void __launch_bounds__(256) k_gram_f32w(int64_t n, int p, int ld, int ntile, const float *__restrict__ X,
                                                   const float *__restrict__ A, const float *__restrict__ B,
                                                   double *part, int64_t rows_per_split) {
    __shared__ __align__(16) float xs[GM_KR][GM_T], as[GM_KR][GM_T], bs[GM_KR][GM_T];
    const int qp = blockIdx.x;
    int pair = blockIdx.x, ti = 0;
    while (pair >= ntile - ti) { pair -= ntile - ti; ++ti; }
    const int tj = ti + pair;
    const int i0 = ti * GM_T, j0 = tj * GM_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = blockIdx.y * rows_per_split;
    const int64_t r1 = r0 + rows_per_split < n ? r0 + rows_per_split : n;
    // loader: thread -> (row lr, float4 column q) of the 32 x 64 chunk, two items per array
    float4 vx[2], va[2], vb[2];
    auto fetch = [&](int64_t rb) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + 256 * h, lr = e >> 4, q = (e & 15) * 4;
            const int64_t r = rb + lr;
            const bool okr = r < r1;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            vx[h] = (okr && i0 + q < ld) ? *reinterpret_cast<const float4 *>(X + r * ld + i0 + q) : z;
            va[h] = (okr && j0 + q < ld) ? *reinterpret_cast<const float4 *>(A + r * ld + j0 + q) : z;
            vb[h] = (okr && j0 + q < ld) ? *reinterpret_cast<const float4 *>(B + r * ld + j0 + q) : z;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + 256 * h, lr = e >> 4, q = (e & 15) * 4;
            *reinterpret_cast<float4 *>(&xs[lr][q]) = vx[h];
            *reinterpret_cast<float4 *>(&as[lr][q]) = va[h];
            *reinterpret_cast<float4 *>(&bs[lr][q]) = vb[h];
        }
    };
    float ca[4][4], cb[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { ca[a][b] = 0.f; cb[a][b] = 0.f; }
    if (r0 < r1) fetch(r0);
    for (int64_t rb = r0; rb < r1; rb += GM_KR) {
        __syncthreads();
        stash();
        __syncthreads();
        if (rb + GM_KR < r1) fetch(rb + GM_KR);       // the next chunk is in flight meanwhile
#pragma unroll 4
        for (int k = 0; k < GM_KR; ++k) {
            const float4 x4 = *reinterpret_cast<const float4 *>(&xs[k][4 * ty]);
            const float4 a4 = *reinterpret_cast<const float4 *>(&as[k][4 * tx]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&bs[k][4 * tx]);
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w}, av[4] = {a4.x, a4.y, a4.z, a4.w},
                        bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    ca[a][b] = fmaf(xv[a], av[b], ca[a][b]);
                    cb[a][b] = fmaf(xv[a], bv[b], cb[a][b]);
                }
        }
    }
    const int64_t S = gridDim.y;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int la = 4 * ty + a, lb = 4 * tx + b, i = i0 + la, j = j0 + lb;
            if (i < p && j < p && i <= j) {
                part[(((int64_t)qp * 2 * GM_T + la) * GM_T + lb) * S + blockIdx.y] = (double)ca[a][b];
                part[((((int64_t)qp * 2 + 1) * GM_T + la) * GM_T + lb) * S + blockIdx.y] = (double)cb[a][b];
            }
        }
}

// The Grams from the split partials: one warp per upper entry (m, i <= j < p) adds its units
// (splits) in order (lanes stride, then a fixed butterfly) and writes the entry and its mirror.
// Tiles of TS x TS, ntile per side, pairs numbered row by row over the upper triangle.
__global__ void __launch_bounds__(256) k_gram_fin(int p, int ld, int TS, int ntile, int64_t units,
                                                  const double *__restrict__ part, double *XA, double *XB) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nup = (int64_t)p * (p + 1) / 2;
    if (w >= 2 * nup) return;
    const int m = (int)(w / nup);
    int64_t r = w - m * nup;
    int i = 0;
    while (r >= p - i) { r -= p - i; ++i; }
    const int j = i + (int)r;
    const int ti = i / TS, tj = j / TS;
    const int64_t q = (int64_t)ti * ntile - (int64_t)ti * (ti - 1) / 2 + (tj - ti);
    const int64_t e = ((q * 2 + m) * TS + (i - ti * TS)) * TS + (j - tj * TS);
    const double *a = part + e * units;
    double s = 0.0;
    for (int64_t u = lane; u < units; u += 32) s += __ldcg(a + u);
    s = warp_sum(s);
    if (lane == 0) {
        double *M = m == 0 ? XA : XB;
        M[(int64_t)i * ld + j] = s;
        M[(int64_t)j * ld + i] = s;
    }
}

// ---------------------------------------------------------------- gradient and residual
// G = HX + BX C ;  kkt2 += ||HX - BX L0||^2 (columns < p).  A 32-row tile is staged in shared
// memory; its 32 x ld outputs are spread over the 256 threads (output o = tid + 256 i), so
// every lane issues useful float64 FMAs whatever ld is.  C and L0 are staged in KC-row chunks.
template <class T, int NO>
__global__ void __launch_bounds__(256) k_grad(int64_t n, int p, int ld, const T *__restrict__ HX,
                                              const T *__restrict__ BX,
                                              const double *__restrict__ C,
                                              const double *__restrict__ L0, T *G,
                                              double *kkt2, int KC, double *gpart, unsigned *gcount) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bx = reinterpret_cast<T *>(smem_raw);   // 32 x ld
    T *cs = bx + 32 * ld;                       // KC x ld
    T *ls = cs + KC * ld;                       // KC x ld
    __shared__ double red[8];
    const int nout = 32 * ld;
    double part = 0.0;
    for (int64_t rt = blockIdx.x * 32LL; rt < n; rt += 32LL * gridDim.x) {
        T g[NO], rr[NO];
        int orow[NO], ocol[NO];
        __syncthreads();
        for (int idx = threadIdx.x; idx < nout; idx += 256) {
            const int64_t r = rt + idx / ld;
            bx[idx] = r < n ? BX[rt * ld + idx] : T(0);
        }
#pragma unroll
        for (int i = 0; i < NO; ++i) {
            const int o = threadIdx.x + 256 * i;
            orow[i] = o / ld;
            ocol[i] = o - orow[i] * ld;
            const int64_t r = rt + orow[i];
            const T h = (o < nout && r < n) ? HX[rt * ld + o] : T(0);
            g[i] = h; rr[i] = h;
        }
        for (int k0 = 0; k0 < ld; k0 += KC) {
            const int kl = min(KC, ld - k0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < kl * ld; idx += 256) {
                cs[idx] = (T)C[(int64_t)k0 * ld + idx];
                ls[idx] = (T)L0[(int64_t)k0 * ld + idx];
            }
            __syncthreads();
            for (int kk = 0; kk < kl; ++kk) {
#pragma unroll
                for (int i = 0; i < NO; ++i) {
                    if (threadIdx.x + 256 * i < nout) {
                        const T b = bx[orow[i] * ld + k0 + kk];
                        g[i] = fma(b, cs[kk * ld + ocol[i]], g[i]);
                        rr[i] = fma(-b, ls[kk * ld + ocol[i]], rr[i]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NO; ++i) {
            const int o = threadIdx.x + 256 * i;
            const int64_t r = rt + orow[i];
            if (o >= nout || r >= n) continue;
            G[rt * ld + o] = g[i];
            if (ocol[i] < p) part += (double)(rr[i] * rr[i]);
        }
    }
    const double tot[1] = {block_sum(part, red)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { *kkt2 += v; });
}

// float32 blocks: the same product with 64-row tiles and a 4-row x CPT-column register tile per
// thread (columns tx + 16 k), C and L0 held whole in shared memory: 2 (4 + CPT) shared loads per
// 8 CPT FMAs, where the float64 form above spends 3 per 2 (its limit is the FP64 pipe, not
// shared memory).
template <int CPT>
__global__ void __launch_bounds__(256) k_grad_f32(int64_t n, int p, int ld, const float *__restrict__ HX,
                                                  const float *__restrict__ BX, const double *__restrict__ C,
                                                  const double *__restrict__ L0, float *G, double *kkt2,
                                                  double *gpart, unsigned *gcount) {
    extern __shared__ __align__(16) float gsm[];
    float *cs = gsm;                 // ld x ld
    float *ls = cs + ld * ld;        // ld x ld
    float *bx = ls + ld * ld;        // 64 x ld
    __shared__ double red[8];
    for (int i = threadIdx.x; i < ld * ld; i += blockDim.x) { cs[i] = (float)C[i]; ls[i] = (float)L0[i]; }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double part = 0.0;
    for (int64_t r0 = blockIdx.x * 64LL; r0 < n; r0 += 64LL * gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < 64 * ld; i += blockDim.x) {
            const int64_t r = r0 + i / ld;
            bx[i] = r < n ? BX[r0 * ld + i] : 0.f;
        }
        __syncthreads();
        float g[4][CPT], rr[4][CPT];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t r = r0 + 4 * ty + i;
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int col = tx + 16 * k;
                const float h = (r < n && col < ld) ? HX[r * ld + col] : 0.f;
                g[i][k] = h; rr[i][k] = h;
            }
        }
        for (int kk = 0; kk < ld; ++kk) {
            float b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = bx[(4 * ty + i) * ld + kk];
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int col = tx + 16 * k;
                const float cv = col < ld ? cs[kk * ld + col] : 0.f, lv = col < ld ? ls[kk * ld + col] : 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    g[i][k] = fmaf(b[i], cv, g[i][k]);
                    rr[i][k] = fmaf(-b[i], lv, rr[i][k]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t r = r0 + 4 * ty + i;
            if (r >= n) continue;
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int col = tx + 16 * k;
                if (col >= ld) continue;
                G[r * ld + col] = g[i][k];
                if (col < p) part += (double)(rr[i][k] * rr[i][k]);
            }
        }
    }
    const double tot[1] = {block_sum(part, red)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { *kkt2 += v; });
}

// float32 blocks with 64 < ld <= 256: C and L0 no longer fit in shared memory whole, so each CTA
// owns a 64-column slice of the outputs (C[:, c0:c0+64] and L0[:, c0:c0+64] stay in shared
// memory) and walks 64-row tiles of B X, staged transposed so that one float4 load gives four
// rows of a column k.  A thread keeps a 4-row x 4-column tile of G and of R: per k one float4 of
// B X, one of C and one of L0 feed 32 FMAs.  The CTAs of one row tile run side by side (slice =
// block index mod the slice count), so their B X reads after the first come from L2.
constexpr int GW_ROWS = 64, GW_COLS = 64, GW_PAD = GW_ROWS + 4;

__global__ void __launch_bounds__(256) k_grad_f32w(int64_t n, int p, int ld, int nslices,
                                                   const float *__restrict__ HX, const float *__restrict__ BX,
                                                   const double *__restrict__ C, const double *__restrict__ L0,
                                                   float *G, double *kkt2, double *gpart, unsigned *gcount) {
    extern __shared__ __align__(16) float gwm[];
    float *cs = gwm;                          // ld x GW_COLS
    float *ls = cs + ld * GW_COLS;            // ld x GW_COLS
    float *bt = ls + ld * GW_COLS;            // ld x GW_PAD: bt[k GW_PAD + row] = B X[r0 + row][k]
    __shared__ double red[8];
    const int slice = blockIdx.x % nslices, c0 = slice * GW_COLS;
    const int cps = gridDim.x / nslices, ci = blockIdx.x / nslices;   // CTAs per slice, this CTA's index
    for (int i = threadIdx.x; i < ld * GW_COLS; i += blockDim.x) {
        const int k = i / GW_COLS, col = c0 + (i - k * GW_COLS);
        cs[i] = col < ld ? (float)C[(int64_t)k * ld + col] : 0.f;
        ls[i] = col < ld ? (float)L0[(int64_t)k * ld + col] : 0.f;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int col0 = c0 + 4 * tx;             // this thread's 4 columns (ld % 4 == 0: all in or all out)
    const bool cin = col0 < ld;
    double part = 0.0;
    for (int64_t r0 = (int64_t)ci * GW_ROWS; r0 < n; r0 += (int64_t)GW_ROWS * cps) {
        const int rows = (int)(n - r0 < GW_ROWS ? n - r0 : GW_ROWS);
        // the tile's float4 pieces: all loads issued before the transposed stores (one round trip)
        constexpr int MAXV = GW_ROWS * 256 / 4 / 256;
        const int nv = GW_ROWS * ld / 4;
        float4 v[MAXV];
#pragma unroll
        for (int q = 0; q < MAXV; ++q) {
            const int e4 = threadIdx.x + q * 256;
            v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e4 < nv && (e4 * 4) / ld < rows) v[q] = *reinterpret_cast<const float4 *>(BX + r0 * ld + e4 * 4);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXV; ++q) {
            const int e4 = threadIdx.x + q * 256;
            if (e4 >= nv) break;
            const int row = (e4 * 4) / ld, k = e4 * 4 - row * ld;      // k..k+3 lie in the same row
            bt[k * GW_PAD + row] = v[q].x;
            bt[(k + 1) * GW_PAD + row] = v[q].y;
            bt[(k + 2) * GW_PAD + row] = v[q].z;
            bt[(k + 3) * GW_PAD + row] = v[q].w;
        }
        __syncthreads();
        float g[4][4], rr[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = 4 * ty + i;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
            if (cin && row < rows) h = *reinterpret_cast<const float4 *>(HX + (r0 + row) * ld + col0);
            g[i][0] = rr[i][0] = h.x; g[i][1] = rr[i][1] = h.y; g[i][2] = rr[i][2] = h.z; g[i][3] = rr[i][3] = h.w;
        }
#pragma unroll 2
        for (int kk = 0; kk < ld; ++kk) {
            const float4 b = *reinterpret_cast<const float4 *>(bt + kk * GW_PAD + 4 * ty);
            const float4 cv = *reinterpret_cast<const float4 *>(cs + kk * GW_COLS + 4 * tx);
            const float4 lv = *reinterpret_cast<const float4 *>(ls + kk * GW_COLS + 4 * tx);
            const float bb[4] = {b.x, b.y, b.z, b.w}, cc[4] = {cv.x, cv.y, cv.z, cv.w}, ll[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    g[i][j] = fmaf(bb[i], cc[j], g[i][j]);
                    rr[i][j] = fmaf(-bb[i], ll[j], rr[i][j]);
                }
        }
        if (!cin) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = 4 * ty + i;
            if (row >= rows) continue;
            *reinterpret_cast<float4 *>(G + (r0 + row) * ld + col0) = make_float4(g[i][0], g[i][1], g[i][2], g[i][3]);
            float rp = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (col0 + j < p) rp = fmaf(rr[i][j], rr[i][j], rp);
            part += (double)rp;
        }
    }
    const double tot[1] = {block_sum(part, red)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { *kkt2 += v; });
}

// ---------------------------------------------------------------- elementwise block kernels
// Flattened over the n x ld elements with a stride that is a multiple of ld, so each thread
// keeps one column: per-column scalars are read once and per-column sums stay in a register.
#define ELEM_BEGIN                                                                  \
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;            \
    const int64_t S = stride;                                                       \
    const int j = (int)(gid % ld);                                                  \
    (void)j;                                                                        \
    const int64_t total = n * ld;                                                   \
    if (gid < S) {                                                                  \
        int64_t r = gid / ld;                                                       \
        const int64_t dr = S / ld;                                                  \
        for (int64_t e = gid; e < total; e += S, r += dr) {
#define ELEM_END } }

constexpr int MAXLD = 256;

// element (r, k) of a chunk-major float32 PCG block with row stride ns (n rounded up to 32):
// ((k / 4) ns + r) 4 + k % 4, so the four columns of a chunk of one row are one 16-byte piece and
// consecutive rows are consecutive pieces
__device__ __forceinline__ int64_t sidx(int64_t r, int k, int64_t ns) { return (((int64_t)(k >> 2) * ns + r) << 2) + (k & 3); }

// PCG start: W = 1/diag with diag = dL/2 - shift_c dB, D = 0, R = G, Z = G W, rz[c] = sum R Z.
// The PCG block has width ld; with cmap its column c < p is column cmap[c] of G (row pitch ldg),
// its other columns are zero.  With Qn (natural layout, pitch ldg) the columns whose CB_WARM entry
// is set start from the natural-layout Dn with T Dn in Qn: R = G - Qn, D = Dn.
template <class T>
__global__ void __launch_bounds__(256) k_pcg_init(int64_t n, int p, int ld, int64_t stride,
                                                  const T *__restrict__ G, int ldg, const int *__restrict__ cmap,
                                                  const T *Qn, const T *Dn,
                                                  const double *__restrict__ dL,
                                                  const double *__restrict__ dB, const double *cb,
                                                  T *W, T *D, T *R, T *Z, double *part) {
    T acc = T(0);
    ELEM_BEGIN
        const T sh = (T)cb[CB_SHIFT * ld + j];
        const T w = T(1) / (T(0.5) * (T)dL[r] - sh * (T)dB[r]);
        const int64_t src = cmap ? (j < p ? r * ldg + cmap[j] : -1) : e;
        T gv = src >= 0 ? G[src] : T(0), dv = T(0);
        if (Qn && src >= 0 && cb[CB_WARM * ld + j] != 0.0) { gv -= Qn[src]; dv = Dn[src]; }
        const T z = gv * w;
        W[e] = w; D[e] = dv; R[e] = gv; Z[e] = z;
        acc = fma(gv, z, acc);
    ELEM_END
    col_partial((double)acc, gid < stride, ld, ld, part);      // rz
}

// learned preconditioner judge sums per column, in the norm of the Jacobi diagonal M of T (the
// norm in which the PCG measures its residuals, r^T M^{-1} r): |G - T D|^2, |G|^2 (T D in Q), and
// G.D
template <class T>
__global__ void __launch_bounds__(256) k_judge(int64_t n, int p, int ld, int64_t stride, const T *__restrict__ G,
                                               const T *__restrict__ Q, const T *__restrict__ D,
                                               const double *__restrict__ dL, const double *__restrict__ dB,
                                               const double *__restrict__ cb, double *part) {
    T a = T(0), b = T(0), d = T(0);
    ELEM_BEGIN
        const T sh = (T)cb[CB_SHIFT * ld + j];
        const T w = cb[CB_ACTIVE * ld + j] != 0.0 ? T(1) / (T(0.5) * (T)dL[r] - sh * (T)dB[r]) : T(1);
        const T g = G[e], rv = g - Q[e];
        a = fma(rv * w, rv, a); b = fma(g * w, g, b); d = fma(g, D[e], d);
    ELEM_END
    const int64_t set = (int64_t)ld * gridDim.x;            // |G - T D|^2, |G|^2, G.D
    col_partial((double)a, gid < stride, ld, ld, part);
    col_partial((double)b, gid < stride, ld, ld, part + set);
    col_partial((double)d, gid < stride, ld, ld, part + 2 * set);
}

// PCG restarted from the current D (the network's output): R = G - Q with Q = T D, Z = R W
template <class T>
__global__ void __launch_bounds__(256) k_pcg_init_warm(int64_t n, int p, int ld, int64_t stride,
                                                       const T *__restrict__ G, const T *__restrict__ Q,
                                                       const double *__restrict__ dL,
                                                       const double *__restrict__ dB, const double *cb,
                                                       T *W, T *R, T *Z, double *part) {
    T acc = T(0);
    ELEM_BEGIN
        const T sh = (T)cb[CB_SHIFT * ld + j];
        const T w = T(1) / (T(0.5) * (T)dL[r] - sh * (T)dB[r]);
        const T rv = G[e] - Q[e];
        const T z = rv * w;
        W[e] = w; R[e] = rv; Z[e] = z;
        acc = fma(rv, z, acc);
    ELEM_END
    col_partial((double)acc, gid < stride, ld, ld, part);      // rz
}

// alpha = rz/pq; D += alpha P; R -= alpha Q; Z = R W; rzn += R Z
template <class T>
__global__ void __launch_bounds__(256) k_pcg_update(int64_t n, int p, int ld, int64_t stride, const double *cb,
                                                    const T *__restrict__ W,
                                                    const T *__restrict__ P,
                                                    const T *__restrict__ Q, T *D, T *R,
                                                    T *Z, double *part) {
    T acc = T(0);
    const T al = (T)cb[CB_ALPHA * ld + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % ld];
    ELEM_BEGIN
        D[e] = fma(al, P[e], D[e]);
        const T rv = fma(-al, Q[e], R[e]);
        const T z = rv * W[e];
        R[e] = rv; Z[e] = z;
        acc = fma(rv, z, acc);
    ELEM_END
    col_partial((double)acc, gid < stride, ld, ld, part);      // rzn
}

// ---- float32 PCG blocks chunk-major (W, R, Z, P, Q and its D, all sidx-indexed)
//
// Start: rows n <= r < ns are padding and stay zero; compact column k < pc is column cmap[k] of G
// (row-major, pitch ld); the other columns are zero.  W = 1/diag with diag = dL/2 - shift_k dB;
// R = G (minus Q, the operator applied to the network's D, when warm); Z = W R; D = 0 (or the
// network's D when warm); rz[k] += R Z; the padding rows of P (and of Q when it is not the warm
// start's input) are zeroed.  Each thread takes (row, 4-column chunk) items in a
// grid-stride loop: consecutive threads take consecutive rows of one chunk, so every write is one
// float4 of a contiguous run; a warp never spans two chunks (ns is a multiple of 32).
// Column sums go warp -> the warp's own row of shared memory (lane 0 adds, in item order) -> the
// block's partial per column (the eight warp rows added in order) -> part[k * gridDim.x + block].
__device__ __forceinline__ void flush_cols(const float (&acc)[4], int q, float (*csw)[MAXLD]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float t = warp_sum_f(acc[i]);
        if ((threadIdx.x & 31) == 0) csw[threadIdx.x >> 5][4 * q + i] += t;
    }
}

__device__ __forceinline__ void cols_out(int w, const float (*csw)[MAXLD], double *part) {
    __syncthreads();
    for (int k = threadIdx.x; k < w; k += blockDim.x) {
        float t = 0.f;
        for (int wp = 0; wp < 8; ++wp) t += csw[wp][k];
        part[(int64_t)k * gridDim.x + blockIdx.x] = (double)t;
    }
}

__global__ void __launch_bounds__(256) k_pcg_init_s(int64_t n, int64_t ns, int pc, int w,
                                                    const float *__restrict__ G, const float *__restrict__ Qn,
                                                    const float *__restrict__ Dn, int ld, const int *__restrict__ cmap,
                                                    const double *__restrict__ dL, const double *__restrict__ dB,
                                                    const double *__restrict__ cb, const int *__restrict__ tmap,
                                                    float *W, float *D, float *R, float *Z, float *P, float *Q,
                                                    double *part, int jac) {
    __shared__ float csw[8][MAXLD];
    __shared__ int scol[MAXLD];
    __shared__ float ssh[MAXLD];
    __shared__ unsigned char swarm[MAXLD];
    for (int k = threadIdx.x; k < 8 * MAXLD; k += blockDim.x) csw[k / MAXLD][k % MAXLD] = 0.f;
    for (int k = threadIdx.x; k < w; k += blockDim.x) {
        scol[k] = k < pc ? cmap[k] : -1;
        ssh[k] = (float)cb[CB_SHIFT * w + k];
        swarm[k] = (Qn && cb[CB_WARM * w + k] != 0.0) ? 1 : 0;
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;    // a multiple of 32
    // one block row (type order) per item, all its chunks in turn: the free row tmap[t] of G (and
    // of Q, D when warm) is read once and the chunk-major writes of one chunk stay contiguous
    // across the warp
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t - (threadIdx.x & 31) < ns; t += stride) {
        const int64_t r = t < ns ? tmap[t] : -1;
        const bool real = r >= 0;
        const float dl = real ? 0.5f * (float)dL[r] : 0.f, db = real ? (float)dB[r] : 0.f;
        for (int q = 0; q < (w >> 2); ++q) {
            float wv[4], rv[4], zv[4], dv[4], acc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * q + i;
                const int col = scol[k];
                float g = 0.f, d = 0.f, ww = 0.f;
                if (real) {
                    if (jac) ww = 1.f / (dl - ssh[k] * db);
                    if (col >= 0) {
                        const int64_t e = r * ld + col;
                        g = G[e];
                        if (swarm[k]) { g -= Qn[e]; d = Dn[e]; }
                    }
                }
                wv[i] = ww; rv[i] = g; zv[i] = g * ww; dv[i] = d;
                acc[i] = g * zv[i];
            }
            if (t < ns) {
                const int64_t o = (q * ns + t) << 2;           // sidx(t, 4 q, ns)
                *reinterpret_cast<float4 *>(R + o) = make_float4(rv[0], rv[1], rv[2], rv[3]);
                *reinterpret_cast<float4 *>(D + o) = make_float4(dv[0], dv[1], dv[2], dv[3]);
                if (jac) {
                    *reinterpret_cast<float4 *>(W + o) = make_float4(wv[0], wv[1], wv[2], wv[3]);
                    *reinterpret_cast<float4 *>(Z + o) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                }
                if (!real) {                                 // padding rows: the apply never writes their P, Q
                    *reinterpret_cast<float4 *>(P + o) = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (Q) *reinterpret_cast<float4 *>(Q + o) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (jac) flush_cols(acc, q, csw);
        }
    }
    if (jac) cols_out(w, csw, part);                         // rz
}

// alpha = rz/pq; D += alpha P; R -= alpha Q; Z = R W; rzn += R Z, per float4 of one row and
// chunk.  On the last iteration only D is needed (last = 1: R, Z and rzn are left alone).
__global__ void __launch_bounds__(256) k_pcg_update_s(int64_t ns, int pc, int w, const double *__restrict__ cb,
                                                      const float *__restrict__ W, const float *__restrict__ P,
                                                      const float *__restrict__ Q, float *D, float *R, float *Z,
                                                      double *part, int last, int jac) {
    __shared__ float csw[8][MAXLD], al[MAXLD];
    for (int k = threadIdx.x; k < 8 * MAXLD; k += blockDim.x) csw[k / MAXLD][k % MAXLD] = 0.f;
    for (int k = threadIdx.x; k < w; k += blockDim.x) al[k] = (float)cb[CB_ALPHA * w + k];
    __syncthreads();
    const int64_t total = ns * (w >> 2);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx - (threadIdx.x & 31) < total;
         idx += stride) {
        const int q = (int)(idx / ns);
        const int64_t o = idx << 2;                  // sidx(r, 4 q, ns) with r = idx - q ns
        const float a0 = al[4 * q], a1 = al[4 * q + 1], a2 = al[4 * q + 2], a3 = al[4 * q + 3];
        const float4 p4 = *reinterpret_cast<const float4 *>(P + o);
        float4 d4 = *reinterpret_cast<const float4 *>(D + o);
        d4.x = fmaf(a0, p4.x, d4.x); d4.y = fmaf(a1, p4.y, d4.y); d4.z = fmaf(a2, p4.z, d4.z); d4.w = fmaf(a3, p4.w, d4.w);
        *reinterpret_cast<float4 *>(D + o) = d4;
        if (last) continue;
        const float4 q4 = *reinterpret_cast<const float4 *>(Q + o);
        float4 r4 = *reinterpret_cast<const float4 *>(R + o);
        r4.x = fmaf(-a0, q4.x, r4.x); r4.y = fmaf(-a1, q4.y, r4.y); r4.z = fmaf(-a2, q4.z, r4.z); r4.w = fmaf(-a3, q4.w, r4.w);
        *reinterpret_cast<float4 *>(R + o) = r4;
        if (!jac) continue;                      // Z and r.z come from the separable preconditioner
        const float4 w4 = *reinterpret_cast<const float4 *>(W + o);
        const float4 z4 = make_float4(r4.x * w4.x, r4.y * w4.y, r4.z * w4.z, r4.w * w4.w);
        *reinterpret_cast<float4 *>(Z + o) = z4;
        const float acc[4] = {r4.x * z4.x, r4.y * z4.y, r4.z * z4.z, r4.w * z4.w};
        flush_cols(acc, q, csw);
    }
    if (last || !jac) return;
    cols_out(w, csw, part);                                  // rzn
}

// The separable preconditioner of the float32 PCG (lattice meshes): R (chunk-major, type-ordered
// rows) -> the bf16 tensor [k][a][b][c~] of the contractions (free row r = (a ny + b) nz + c;
// columns k >= pc are zero), then after the passes Z <- the tensor (chunk-major) with the column
// sums rz = R.Z as per-block partials (as k_pcg_update_s writes them).  Items (block row, 4-column
// chunk) as in the other chunk-major kernels; tmap gives a block row's free row (-1: padding).
__global__ void __launch_bounds__(256) k_psep_gather(int64_t ns, int pc, int w, int nz, int pz, int64_t blk,
                                                     const int *__restrict__ tmap, const float *__restrict__ R,
                                                     __nv_bfloat16 *t) {
    const int64_t total = ns * (w >> 2);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(idx / ns);
        const int64_t r = tmap[idx - (int64_t)q * ns];
        if (r < 0) continue;
        const float4 v = *reinterpret_cast<const float4 *>(R + (idx << 2));
        const float vv[4] = {v.x, v.y, v.z, v.w};
        const int64_t pos = (r / nz) * pz + r % nz;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * q + i;
            t[(int64_t)k * blk + pos] = __float2bfloat16(k < pc ? vv[i] : 0.f);
        }
    }
}

__global__ void __launch_bounds__(256) k_psep_scatter(int64_t ns, int pc, int w, int nz, int pz, int64_t blk,
                                                      const int *__restrict__ tmap, const __nv_bfloat16 *__restrict__ t,
                                                      const float *__restrict__ R, float *Z, double *part) {
    __shared__ float csw[8][MAXLD];
    for (int k = threadIdx.x; k < 8 * MAXLD; k += blockDim.x) csw[k / MAXLD][k % MAXLD] = 0.f;
    __syncthreads();
    const int64_t total = ns * (w >> 2);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;    // a multiple of 32
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx - (threadIdx.x & 31) < total;
         idx += stride) {
        // the warp's first item decides for the whole warp (total is a multiple of 32)
        const int q = (int)(idx / ns);
        const int64_t r = idx < total ? tmap[idx - (int64_t)q * ns] : -1;
        float zv[4] = {0.f, 0.f, 0.f, 0.f}, acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (r >= 0) {
            const float4 rv = *reinterpret_cast<const float4 *>(R + (idx << 2));
            const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
            const int64_t pos = (r / nz) * pz + r % nz;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * q + i;
                zv[i] = k < pc ? __bfloat162float(t[(int64_t)k * blk + pos]) : 0.f;
                acc[i] = rr[i] * zv[i];
            }
        }
        if (idx < total) *reinterpret_cast<float4 *>(Z + (idx << 2)) = make_float4(zv[0], zv[1], zv[2], zv[3]);
        flush_cols(acc, q, csw);
    }
    cols_out(w, csw, part);                                  // rz
}

// the same for row-major PCG blocks of width ld (element type T)
template <class T>
__global__ void __launch_bounds__(256) k_psep_gather_n(int64_t n, int ld, int64_t stride, int pc, int nz, int pz,
                                                       int64_t blk, const T *__restrict__ R, __nv_bfloat16 *t) {
    ELEM_BEGIN
        t[(int64_t)j * blk + (r / nz) * pz + r % nz] = __float2bfloat16(j < pc ? (float)R[e] : 0.f);
    ELEM_END
}

template <class T>
__global__ void __launch_bounds__(256) k_psep_scatter_n(int64_t n, int ld, int64_t stride, int pc, int nz, int pz,
                                                        int64_t blk, const __nv_bfloat16 *__restrict__ t,
                                                        const T *__restrict__ R, T *Z, double *part) {
    T acc = T(0);
    ELEM_BEGIN
        const T z = j < pc ? (T)__bfloat162float(t[(int64_t)j * blk + (r / nz) * pz + r % nz]) : T(0);
        Z[e] = z;
        acc = fma(R[e], z, acc);
    ELEM_END
    col_partial((double)acc, gid < stride, ld, ld, part);      // rz
}

// D (row-major, pitch ld) from the chunk-major PCG result (free row r at block row tinv[r]):
// column j takes compact column cpos[j] of Dc, G when inactive (cpos[j] = -1: T = I in Eq.
// precondition-T), and keeps its D when cpos[j] = -2 (a learned direction the judge accepted)
__global__ void __launch_bounds__(256) k_expand_s(int64_t n, int ld, int64_t stride, int64_t ns,
                                                  const int *__restrict__ cpos, const int *__restrict__ tinv,
                                                  const float *__restrict__ G, const float *__restrict__ Dc, float *D) {
    ELEM_BEGIN
        const int k = cpos[j];
        if (k >= 0) D[e] = Dc[sidx(tinv[r], k, ns)];
        else if (k == -1) D[e] = G[e];
    ELEM_END
}

// D from the compact PCG: column j takes compact column cpos[j] of Dc (width w), G when it is
// inactive (cpos[j] = -1: T = I in Eq. precondition-T), and keeps its D when cpos[j] = -2 (a
// learned direction the judge accepted)
template <class T>
__global__ void __launch_bounds__(256) k_expand(int64_t n, int ld, int64_t stride, int w, const int *__restrict__ cpos,
                                                const T *__restrict__ G, const T *__restrict__ Dc, T *D) {
    ELEM_BEGIN
        const int k = cpos[j];
        if (k >= 0) D[e] = Dc[r * w + k];
        else if (k == -1) D[e] = G[e];
    ELEM_END
}

// columns whose shift is not negative take D = G (T = I in Eq. precondition-T)
template <class T>
__global__ void __launch_bounds__(256) k_select(int64_t n, int ld, int64_t stride, const double *cb,
                                                const T *__restrict__ G, T *D) {
    const int jj = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % ld);
    if (cb[CB_ACTIVE * ld + jj] != 0.0) return;
    ELEM_BEGIN
        D[e] = G[e];
    ELEM_END
}

// Barzilai-Borwein sums: <dX,dD>, <dD,dD>, <dX,dX>, and ||X||^2, ||D||^2
template <class T>
__global__ void __launch_bounds__(256) k_bb(int64_t n, int ld, int64_t stride, const T *__restrict__ X,
                                            const T *__restrict__ Xp, const T *__restrict__ D,
                                            const T *__restrict__ Dp, int have_prev, double *sc, double *gpart,
                                            unsigned *gcount) {
    __shared__ double red[8];
    T sy = 0, yy = 0, ss = 0, xx = 0, dd = 0;
    {
        ELEM_BEGIN
            const T x = X[e], d = D[e];
            xx = fma(x, x, xx); dd = fma(d, d, dd);
            if (have_prev) {
                const T sx = x - Xp[e], yd = d - Dp[e];
                sy = fma(sx, yd, sy); yy = fma(yd, yd, yy); ss = fma(sx, sx, ss);
            }
        ELEM_END
    }
    const double tot[5] = {block_sum((double)sy, red), block_sum((double)yy, red), block_sum((double)ss, red),
                           block_sum((double)xx, red), block_sum((double)dd, red)};
    grid_accumulate<5>(tot, gpart, gcount, [&](int k, double v) {
        sc[k < 3 ? SC_BB + k : (k == 3 ? SC_XNRM2 : SC_DNRM2)] = v;
    });
}

// Y = X - D / eta
template <class T>
__global__ void __launch_bounds__(256) k_step(int64_t n, int ld, int64_t stride, const T *__restrict__ X,
                                              const T *__restrict__ D, const double *sc, T *Y) {
    const T inv = (T)(1.0 / sc[SC_ETA]);
    ELEM_BEGIN
        Y[e] = fma(-inv, D[e], X[e]);
    ELEM_END
}

// X_i = Y_i / ||Y_i||_B and B X_i = B Y_i / ||Y_i||_B   (Eq. PCAL-main)
template <class T>
__global__ void __launch_bounds__(256) k_scale(int64_t n, int p, int ld, int64_t stride, const double *colsum,
                                               T *Y, T *BY) {
    const int jj = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % ld);
    if (jj >= p) return;
    const T s = (T)(1.0 / sqrt(colsum[jj]));
    ELEM_BEGIN
        Y[e] *= s; BY[e] *= s;
    ELEM_END
}

template <class S, class T>
__global__ void k_convert(int64_t count, const S *__restrict__ src, T *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// Y = X M with M (ld x ld, zero padded) staged in KC-row chunks
template <class T, int MC>
__global__ void __launch_bounds__(256) k_block_small(int64_t n, int ld, const T *__restrict__ X,
                                                     const double *__restrict__ M, T *Y, int KC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);   // 32 x ld
    T *ms = xs + 32 * ld;                       // KC x ld
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
    for (int64_t rt = blockIdx.x * 32LL; rt < n; rt += 32LL * gridDim.x) {
        T y[4][MC];
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * ld; idx += 256) {
            const int64_t r = rt + idx / ld;
            xs[idx] = r < n ? X[rt * ld + idx] : T(0);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < MC; ++m) y[a][m] = T(0);
        for (int k0 = 0; k0 < ld; k0 += KC) {
            const int kl = min(KC, ld - k0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < kl * ld; idx += 256) ms[idx] = (T)M[(int64_t)k0 * ld + idx];
            __syncthreads();
            for (int kk = 0; kk < kl; ++kk) {
                T b[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) b[a] = xs[(rg * 4 + a) * ld + k0 + kk];
#pragma unroll
                for (int m = 0; m < MC; ++m) {
                    const int j = lane + 32 * m;
                    const T mv = j < ld ? ms[kk * ld + j] : T(0);
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

// out[j] = the sum of column j's partials part[j * units + u] in unit order (j < kact), 0 for
// kact <= j < gridDim.x
__global__ void __launch_bounds__(256) k_col_fin(int kact, int64_t units, const double *__restrict__ part,
                                                 double *out) {
    __shared__ double sh[8];
    const int j = blockIdx.x;
    const double s = j < kact ? ordered_sum(part + (int64_t)j * units, units, sh) : 0.0;
    if (threadIdx.x == 0) out[j] = s;
}

}  // namespace

void launch_col_fin(ofks_ctx *c, int kact, int ktot, int64_t units, const double *part, double *out) {
    if (ktot <= 0) return;
    k_col_fin<<<(unsigned)ktot, 256, 0, c->stream>>>(kact, units, part, out);
    c->kernels += 1;
}

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

template <class T>
void launch_gram2(ofks_ctx *c, const T *X, const T *A, const T *B, double *XA, double *XB) {
    c->kernels += 2;
    ProfScope ps(c, PF_GRAM);
    const int ld = c->ld, p = c->p;
    cudaMemsetAsync(XA, 0, sizeof(double) * ld * ld, c->stream);    // the padding stays zero
    cudaMemsetAsync(XB, 0, sizeof(double) * ld * ld, c->stream);
    // the split partials are added in split order by k_gram_fin (one warp per upper entry)
    auto fin = [&](int TS, int ntile, int64_t units) {
        const int64_t warps = (int64_t)p * (p + 1);
        k_gram_fin<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(p, ld, TS, ntile, units, c->d_cpart,
                                                                               XA, XB);
    };
    if constexpr (sizeof(T) == 4) {
        int64_t units = 0;
        if (launch_gram_tc(c, (const float *)X, (const float *)A, (const float *)B, c->d_cpart, &units)) {
            fin(ld, 1, units);
            return;
        }
        if (ld > 64 && ld <= 256 && ld % 4 == 0) {
            const int ntile = (p + GM_T - 1) / GM_T, npair = ntile * (ntile + 1) / 2;
            int64_t splits = std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, (152LL * 4) / npair + 1));
            const int64_t rps = ((c->n + splits - 1) / splits + GM_KR - 1) / GM_KR * GM_KR;
            splits = (c->n + rps - 1) / rps;
            k_gram_f32w<<<dim3((unsigned)npair, (unsigned)splits), 256, 0, c->stream>>>(
                c->n, p, ld, ntile, (const float *)X, (const float *)A, (const float *)B, c->d_cpart, rps);
            fin(GM_T, ntile, splits);
            return;
        }
    }
    int RT = p <= 16 ? 1 : (p <= 32 ? 2 : (p <= 48 ? 3 : 4));
    const int TS = 16 * RT, ntile = (p + TS - 1) / TS, npair = ntile * (ntile + 1) / 2;
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, (152LL * 4) / npair + 1));
    const int64_t rps = ((c->n + splits - 1) / splits + 15) / 16 * 16;
    splits = (c->n + rps - 1) / rps;
    dim3 grid((unsigned)npair, (unsigned)splits);
#define G_(rt) k_gram2<T, rt><<<grid, 256, 0, c->stream>>>(c->n, p, ld, ntile, X, A, B, c->d_cpart, rps)
    switch (RT) { case 1: G_(1); break; case 2: G_(2); break; case 3: G_(3); break; default: G_(4); }
#undef G_
    fin(TS, ntile, splits);
}

template <> bool pcg_zc<double>(const ofks_ctx *, int) { return false; }
template <> bool pcg_zc<float>(const ofks_ctx *c, int w) {
    // the staged apply (pcg_staged, widths 8..32) works on row-major blocks of the main SELL
    if (c->prm.pcg_staged && w % 4 == 0 && w >= 8 && w <= 32) return false;
    return c->n_tslices > 0 && w >= 4 && w % 4 == 0;
}

// grid of 256-thread blocks whose total thread count is a multiple of ld
struct ElemGrid { unsigned blocks; int64_t stride; };
static ElemGrid elem_grid(int64_t n, int ld) {
    const int64_t want = std::min<int64_t>((n * ld + 255) / 256, 152LL * 8);
    const int64_t threads = std::max<int64_t>(want * 256, ld);
    const int64_t stride = threads / ld * ld;
    return {(unsigned)((stride + 255) / 256), stride};
}

template <class T>
void launch_grad_update(ofks_ctx *c, Blocks<T> &b) {
    c->kernels += 1;
    ProfScope ps(c, PF_GRAD);
    const int ld = c->ld, KC = kc_of(ld);
    const size_t sm = sizeof(T) * (32 * ld + 2 * KC * ld);
    T *G = b.G[c->cur];
    cudaMemsetAsync(c->d_sc + SC_KKT2, 0, sizeof(double), c->stream);
    if constexpr (sizeof(T) == 4) {
        if (launch_grad_tc(c, (const float *)b.HX, (const float *)b.BX, (float *)G, c->d_sc + SC_KKT2)) return;
        if (ld > 64 && ld <= 256 && ld % 4 == 0) {
            const int nsl = (ld + GW_COLS - 1) / GW_COLS;
            const int smw = (int)(sizeof(float) * (size_t)ld * (2 * GW_COLS + GW_PAD));
            const unsigned gw = (unsigned)(nsl * std::max<int64_t>(1, std::min<int64_t>((c->n + GW_ROWS - 1) / GW_ROWS,
                                                                                      152 / nsl)));
            cudaFuncSetAttribute(k_grad_f32w, cudaFuncAttributeMaxDynamicSharedMemorySize, smw);
            k_grad_f32w<<<gw, 256, smw, c->stream>>>(c->n, c->p, ld, nsl, (const float *)b.HX, (const float *)b.BX,
                                                     c->d_C, c->d_L0, (float *)G, c->d_sc + SC_KKT2, c->d_gpart,
                                                     c->d_gcount);
            return;
        }
        if (ld <= 64) {
            const int smf = (int)(sizeof(float) * (2 * ld * ld + 64 * ld));
            const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>((c->n + 63) / 64, 152 * 4));
#define GF_(k) { cudaFuncSetAttribute(k_grad_f32<k>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf); \
        k_grad_f32<k><<<gf, 256, smf, c->stream>>>(c->n, c->p, ld, (const float *)b.HX, (const float *)b.BX, \
                                                   c->d_C, c->d_L0, (float *)G, c->d_sc + SC_KKT2, c->d_gpart, \
                                                   c->d_gcount); }
            if (ld <= 16) GF_(1) else if (ld <= 32) GF_(2) else if (ld <= 48) GF_(3) else GF_(4)
#undef GF_
            return;
        }
    }
    const unsigned grid = row_grid(32, c->n);
    const int no = (32 * ld + 255) / 256;
#define GR_(k) { cudaFuncSetAttribute(k_grad<T, k>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        k_grad<T, k><<<grid, 256, sm, c->stream>>>(c->n, c->p, ld, b.HX, b.BX, c->d_C, c->d_L0, G, \
                                                  c->d_sc + SC_KKT2, KC, c->d_gpart, c->d_gcount); }
    if (no <= 1) GR_(1) else if (no <= 2) GR_(2) else if (no <= 4) GR_(4) else if (no <= 6) GR_(6)
    else if (no <= 8) GR_(8) else if (no <= 16) GR_(16) else GR_(32)
#undef GR_
}

template <class T>
void launch_pcg_init(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v, bool warm) {
    c->kernels += 1;
    const int w = v.w;
    const T *Qn = warm ? b.Q : nullptr, *Dn = warm ? b.D[c->cur] : nullptr;
    if constexpr (sizeof(T) == 4) {
        if (pcg_zc<T>(c, w)) {
            // a warm start reads T D from the natural-layout Q, so the chunk-major Q (the same
            // buffer) is not cleared here; its padding rows then hold finite values of T D, which
            // the apply never reads and whose products with the zero preconditioner weights of
            // the padding rows add nothing
            const int64_t total = c->n_slots * (w >> 2);
            const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
            const bool jac = !pcg_sep_active(c, w);      // else Z and r.z come from the separable step
            const unsigned rgrid = (unsigned)std::min<int64_t>((c->n_slots + 255) / 256, 152 * 8);
            k_pcg_init_s<<<rgrid, 256, 0, c->stream>>>(
                c->n, c->n_slots, v.pc, w, (const float *)b.G[c->cur], (const float *)Qn, (const float *)Dn, c->ld,
                v.cmap, c->d_dL, c->d_dB, v.cb, c->d_tmap, (float *)b.W, (float *)v.D, (float *)b.R, (float *)b.Z, (float *)b.P,
                warm ? nullptr : (float *)b.Q, c->d_cpart, jac ? 1 : 0);
            if (jac) launch_col_fin(c, v.pc, w, rgrid, c->d_cpart, v.cb + CB_RZ * w);
            return;
        }
    }
    const ElemGrid g = elem_grid(c->n, w);
    k_pcg_init<T><<<g.blocks, 256, 0, c->stream>>>(c->n, v.pc, w, g.stride, b.G[c->cur], c->ld, v.cmap, Qn, Dn,
                                                   c->d_dL, c->d_dB, v.cb, b.W, v.D, b.R, b.Z, c->d_cpart);
    launch_col_fin(c, v.pc, w, g.blocks, c->d_cpart, v.cb + CB_RZ * w);
}

// z = T_sep^-1 r for the float32 PCG's w columns (chunk-major R, Z): the rz partials replace
// those of the Jacobi step (rz_units = this grid); false when the form does not apply (not a
// lattice mesh with the tensor-core separable operator, or not the chunk-major float32 blocks)
// the PCG of width w runs with the separable preconditioner (its buffers are allocated here,
// outside any graph capture, by the PCG start)
bool pcg_sep_active(ofks_ctx *c, int w) {
    if (c->prm.pcg_pc != OFKS_PCGPC_SEPARABLE || !sep_pcg_ready(c, w)) return false;
    const SepState &S = c->sep;
    return (int64_t)S.n[0] * S.n[1] * S.n[2] == c->n;
}

template <class T>
bool launch_pcg_sep(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v) {
    const int w = v.w;
    if (!pcg_sep_active(c, w)) return false;
    const SepState &S = c->sep;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2], pz = (nz + 15) / 16 * 16;
    const int64_t blk = (int64_t)nx * ny * pz;
    __nv_bfloat16 *t = S.pbuf + S.poff[0];
    if constexpr (sizeof(T) == 4) {
        if (pcg_zc<T>(c, w)) {
            const int64_t total = c->n_slots * (w >> 2);
            const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
            k_psep_gather<<<grid, 256, 0, c->stream>>>(c->n_slots, v.pc, w, nz, pz, blk, c->d_tmap, (const float *)b.R,
                                                       t);
            sep_pcg_passes(c, w, v.cb + CB_SHIFT * w);
            k_psep_scatter<<<grid, 256, 0, c->stream>>>(c->n_slots, v.pc, w, nz, pz, blk, c->d_tmap, t,
                                                        (const float *)b.R, (float *)b.Z, c->d_cpart);
            c->rz_units = grid;
            c->kernels += 2;
            return true;
        }
    }
    const ElemGrid g = elem_grid(c->n, w);
    k_psep_gather_n<T><<<g.blocks, 256, 0, c->stream>>>(c->n, w, g.stride, v.pc, nz, pz, blk, b.R, t);
    sep_pcg_passes(c, w, v.cb + CB_SHIFT * w);
    k_psep_scatter_n<T><<<g.blocks, 256, 0, c->stream>>>(c->n, w, g.stride, v.pc, nz, pz, blk, t, b.R, b.Z,
                                                         c->d_cpart);
    c->rz_units = g.blocks;
    c->kernels += 2;
    return true;
}

template <class T>
void launch_judge(ofks_ctx *c, Blocks<T> &b) {
    c->kernels += 1;
    const int ld = c->ld;
    double *cb = c->d_colA;
    const ElemGrid g = elem_grid(c->n, ld);
    k_judge<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->p, ld, g.stride, b.G[c->cur], b.Q, b.D[c->cur], c->d_dL,
                                                c->d_dB, cb, c->d_cpart);
    // |G - T D|^2, |G|^2 (M^{-1} norms) and G.D into the RZ, RZN and PQ rows
    const int64_t set = (int64_t)ld * g.blocks;
    launch_col_fin(c, c->p, ld, g.blocks, c->d_cpart, cb + CB_RZ * ld);
    launch_col_fin(c, c->p, ld, g.blocks, c->d_cpart + set, cb + CB_RZN * ld);
    launch_col_fin(c, c->p, ld, g.blocks, c->d_cpart + 2 * set, cb + CB_PQ * ld);
}

template <class T>
void launch_pcg_update(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v, bool last) {
    c->kernels += 1;
    const int w = v.w;
    double *cb = v.cb;
    // the column sums r.z go to the partials; k_pcg_beta adds them (rz_units per column)
    if constexpr (sizeof(T) == 4) {
        if (pcg_zc<T>(c, w)) {
            const int64_t total = c->n_slots * (w >> 2);
            const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
            k_pcg_update_s<<<grid, 256, 0, c->stream>>>(
                c->n_slots, v.pc, w, cb, (const float *)b.W, (const float *)b.P, (const float *)b.Q, (float *)v.D,
                (float *)b.R, (float *)b.Z, c->d_cpart, last ? 1 : 0, pcg_sep_active(c, w) ? 0 : 1);
            c->rz_units = grid;
            return;
        }
    }
    const ElemGrid g = elem_grid(c->n, w);
    k_pcg_update<T><<<g.blocks, 256, 0, c->stream>>>(c->n, v.pc, w, g.stride, cb, b.W, b.P, b.Q, v.D, b.R,
                                                     b.Z, c->d_cpart);
    c->rz_units = g.blocks;
}

template <class T>
void launch_direction_expand(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v) {
    c->kernels += 1;
    const ElemGrid g = elem_grid(c->n, c->ld);
    if constexpr (sizeof(T) == 4) {
        if (pcg_zc<T>(c, v.w)) {
            k_expand_s<<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, c->n_slots, v.cpos, c->d_tinv,
                                                        (const float *)b.G[c->cur], (const float *)v.D,
                                                        (float *)b.D[c->cur]);
            return;
        }
    }
    k_expand<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, v.w, v.cpos, b.G[c->cur], v.D, b.D[c->cur]);
}

template <class T>
void launch_direction_select(ofks_ctx *c, Blocks<T> &b) {
    c->kernels += 1;
    const ElemGrid g = elem_grid(c->n, c->ld);
    k_select<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, c->d_colA, b.G[c->cur], b.D[c->cur]);
}

// BB sums over the applied directions D, or over the raw gradients G when raw is set; the
// norms used by eta_0 are always those of X and D
template <class T>
void launch_bb_dots(ofks_ctx *c, Blocks<T> &b, bool raw) {
    ProfScope ps(c, PF_BB);
    const int cur = c->cur, prv = cur ^ 1;
    const ElemGrid g = elem_grid(c->n, c->ld);
    T **DD = raw ? b.G : b.D;
    k_bb<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, b.X[cur], b.X[prv], DD[cur], DD[prv],
                                             c->have_prev ? 1 : 0, c->d_sc, c->d_gpart, c->d_gcount);
    c->kernels += 1;
    if (raw && !c->have_prev) {       // eta_0 needs ||D||: rerun the sums on D
        k_bb<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, b.X[cur], b.X[prv], b.D[cur], b.D[prv], 0,
                                                 c->d_sc, c->d_gpart, c->d_gcount);
        c->kernels += 1;
    }
}

template <class T>
void launch_step_y(ofks_ctx *c, Blocks<T> &b, T *Y) {
    c->kernels += 1;
    const ElemGrid g = elem_grid(c->n, c->ld);
    k_step<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->ld, g.stride, b.X[c->cur], b.D[c->cur], c->d_sc, Y);
}

template <class T>
void launch_scale_cols(ofks_ctx *c, T *Y, T *BY, const double *colsum) {
    c->kernels += 1;
    const ElemGrid g = elem_grid(c->n, c->ld);
    k_scale<T><<<g.blocks, 256, 0, c->stream>>>(c->n, c->p, c->ld, g.stride, colsum, Y, BY);
}

template <class T>
void launch_block_times_small(ofks_ctx *c, const T *X, const double *M, T *Y) {
    c->kernels += 1;
    const int ld = c->ld, KC = kc_of(ld);
    const size_t sm = sizeof(T) * (32 * ld + KC * ld);
    const unsigned grid = row_grid(32, c->n);
    MC_DISPATCH(mc_of(ld), {
        cudaFuncSetAttribute(k_block_small<T, M_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_block_small<T, M_><<<grid, 256, sm, c->stream>>>(c->n, ld, X, M, Y, KC);
    });
}

__global__ void __launch_bounds__(256) k_repack(int64_t n, int w, const double *__restrict__ src, int64_t sp,
                                                double *__restrict__ dst, int64_t dp) {
    const int64_t total = n * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / w;
        const int j = (int)(i - r * w);
        dst[r * dp + j] = src[r * sp + j];
    }
}

__global__ void __launch_bounds__(256) k_unpack_f32(int64_t n, int p, int ld, const double *__restrict__ src,
                                                    float *__restrict__ dst) {
    const int64_t total = n * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ld;
        const int j = (int)(i - r * ld);
        dst[i] = j < p ? (float)src[r * p + j] : 0.f;
    }
}

__global__ void __launch_bounds__(256) k_pack_f32(int64_t n, int p, int ld, const float *__restrict__ src,
                                                  double *__restrict__ dst) {
    const int64_t total = n * p;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / p;
        const int j = (int)(i - r * p);
        dst[i] = (double)src[r * ld + j];
    }
}

void launch_unpack_f32(ofks_ctx *c, const double *src, float *dst) {
    c->kernels += 1;
    const int64_t count = c->n * (int64_t)c->ld;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152LL * 16));
    k_unpack_f32<<<g, 256, 0, c->stream>>>(c->n, c->p, c->ld, src, dst);
}

void launch_pack_f32(ofks_ctx *c, const float *src, double *dst) {
    c->kernels += 1;
    const int64_t count = c->n * (int64_t)c->p;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152LL * 16));
    k_pack_f32<<<g, 256, 0, c->stream>>>(c->n, c->p, c->ld, src, dst);
}

void launch_repack(ofks_ctx *c, const double *src, int64_t sp, double *dst, int64_t dp, int64_t n, int w) {
    c->kernels += 1;
    const int64_t count = n * w;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152LL * 16));
    k_repack<<<g, 256, 0, c->stream>>>(n, w, src, sp, dst, dp);
}

template <class S, class T>
void launch_convert(ofks_ctx *c, const S *src, T *dst, int64_t count) {
    c->kernels += 1;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152LL * 16));
    k_convert<S, T><<<g, 256, 0, c->stream>>>(count, src, dst);
}

#define INST(T)                                                                                      \
    template void launch_gram2<T>(ofks_ctx *, const T *, const T *, const T *, double *, double *); \
    template void launch_grad_update<T>(ofks_ctx *, Blocks<T> &);                                    \
    template void launch_pcg_init<T>(ofks_ctx *, Blocks<T> &, const PcgView<T> &, bool);             \
    template void launch_pcg_update<T>(ofks_ctx *, Blocks<T> &, const PcgView<T> &, bool);           \
    template void launch_direction_expand<T>(ofks_ctx *, Blocks<T> &, const PcgView<T> &);           \
    template void launch_judge<T>(ofks_ctx *, Blocks<T> &);                                          \
    template bool launch_pcg_sep<T>(ofks_ctx *, Blocks<T> &, const PcgView<T> &);                    \
    template void launch_direction_select<T>(ofks_ctx *, Blocks<T> &);                               \
    template void launch_bb_dots<T>(ofks_ctx *, Blocks<T> &, bool);                                  \
    template void launch_step_y<T>(ofks_ctx *, Blocks<T> &, T *);                                    \
    template void launch_scale_cols<T>(ofks_ctx *, T *, T *, const double *);                        \
    template void launch_block_times_small<T>(ofks_ctx *, const T *, const double *, T *);
INST(double)
INST(float)
#undef INST
template void launch_convert<double, float>(ofks_ctx *, const double *, float *, int64_t);
template void launch_convert<float, double>(ofks_ctx *, const float *, double *, int64_t);
