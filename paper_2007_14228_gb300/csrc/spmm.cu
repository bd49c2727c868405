// SELL-C-sigma sparse times tall-skinny block products for the P2 matrices (paper Sec. 2.2:
// H X, B X; Eq. precondition-T: (L/2 - lambda_i B) z_i).
//
// Layout: rows of the free pattern are sorted by length inside windows of sigma rows and cut
// into slices of 32; entry j of lane l of slice s sits at slice_ptr[s] + 32 j + l, so the 32
// lanes of a warp read 32 consecutive column ids and values.  X and Y are row-major n x ld
// with ld a multiple of the chunk width W; a warp handles one (slice, W-column chunk) pair,
// each lane one row, and gathers W consecutive doubles of each neighbour row with vector
// loads.  Padding entries carry value 0 and repeat the row's last column id.
#include "common.cuh"
#include "internal.h"

namespace {

template <int W>
__device__ __forceinline__ void load_w(const double *__restrict__ p, double (&v)[W]) {
    if constexpr (W == 1) {
        v[0] = __ldg(p);
    } else {
#pragma unroll
        for (int w = 0; w < W; w += 2) {
            double2 t = __ldg(reinterpret_cast<const double2 *>(p + w));
            v[w] = t.x; v[w + 1] = t.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void store_w(double *p, const double (&v)[W]) {
    if constexpr (W == 1) {
        p[0] = v[0];
    } else {
#pragma unroll
        for (int w = 0; w < W; w += 2) *reinterpret_cast<double2 *>(p + w) = make_double2(v[w], v[w + 1]);
    }
}

// MODE 0: Y = A X.  MODE 1: also colsum[c] += sum_rows X[r,c] Y[r,c].
template <int W, int MODE>
__global__ void __launch_bounds__(256) k_sell_spmm(int64_t nwarps, int nchunks, int p, int ld,
                                                   const int *__restrict__ slice_ptr,
                                                   const int *__restrict__ slice_w,
                                                   const int *__restrict__ cols,
                                                   const int *__restrict__ perm,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ X, double *__restrict__ Y,
                                                   double *colsum) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nwarps) return;                       // whole warp leaves together
    const int chunk = (int)(wg % nchunks);
    const int64_t s = wg / nchunks;
    const int c0 = chunk * W;
    const int base = slice_ptr[s], width = slice_w[s];
    const int r = perm[s * SELL_C + lane];
    double acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0.0;
    int e = base + lane;
    for (int j = 0; j < width; ++j, e += SELL_C) {
        const int c = __ldg(cols + e);
        const double v = __ldg(val + e);
        double x[W];
        load_w<W>(X + (int64_t)c * ld + c0, x);
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = fma(v, x[w], acc[w]);
    }
    if (r >= 0) store_w<W>(Y + (int64_t)r * ld + c0, acc);
    if constexpr (MODE == 1) {
        double xr[W];
        if (r >= 0) load_w<W>(X + (int64_t)r * ld + c0, xr);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            double t = (r >= 0) ? xr[w] * acc[w] : 0.0;
            t = warp_sum(t);
            if (lane == 0 && c0 + w < p) atomicAdd(colsum + c0 + w, t);
        }
    }
}

// One Jacobi-PCG operator apply for all columns at once (Eq. precondition-T):
//   TZ = (L/2) Z - B Z diag(shift)  gathered over the neighbours of each row, then for the
//   own row  P <- Z + beta P,  Q <- TZ + beta Q  (so T P = Q), and pq[c] += P.Q.
// With first = 1: P = Z, Q = TZ.
template <int W>
__global__ void __launch_bounds__(256) k_pcg_apply(int64_t nwarps, int nchunks, int p, int ld,
                                                   const int *__restrict__ slice_ptr,
                                                   const int *__restrict__ slice_w,
                                                   const int *__restrict__ cols,
                                                   const int *__restrict__ perm,
                                                   const double *__restrict__ valL,
                                                   const double *__restrict__ valB,
                                                   const double *__restrict__ Z, double *P, double *Q,
                                                   const double *__restrict__ beta_col,
                                                   const double *__restrict__ shift, double *pq,
                                                   int first) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nwarps) return;
    const int chunk = (int)(wg % nchunks);
    const int64_t s = wg / nchunks;
    const int c0 = chunk * W;
    const int base = slice_ptr[s], width = slice_w[s];
    const int r = perm[s * SELL_C + lane];
    double aL[W], aB[W];
#pragma unroll
    for (int w = 0; w < W; ++w) { aL[w] = 0.0; aB[w] = 0.0; }
    int e = base + lane;
    for (int j = 0; j < width; ++j, e += SELL_C) {
        const int c = __ldg(cols + e);
        const double vl = __ldg(valL + e), vb = __ldg(valB + e);
        double x[W];
        load_w<W>(Z + (int64_t)c * ld + c0, x);
#pragma unroll
        for (int w = 0; w < W; ++w) { aL[w] = fma(vl, x[w], aL[w]); aB[w] = fma(vb, x[w], aB[w]); }
    }
    double contrib[W];
    if (r >= 0) {
        double zr[W], pr[W], qr[W];
        load_w<W>(Z + (int64_t)r * ld + c0, zr);
        if (!first) {
            load_w<W>(P + (int64_t)r * ld + c0, pr);
            load_w<W>(Q + (int64_t)r * ld + c0, qr);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const double tz = 0.5 * aL[w] - shift[c0 + w] * aB[w];
            const double b = first ? 0.0 : beta_col[c0 + w];
            const double pn = first ? zr[w] : fma(b, pr[w], zr[w]);
            const double qn = first ? tz : fma(b, qr[w], tz);
            pr[w] = pn; qr[w] = qn;
            contrib[w] = pn * qn;
        }
        store_w<W>(P + (int64_t)r * ld + c0, pr);
        store_w<W>(Q + (int64_t)r * ld + c0, qr);
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) contrib[w] = 0.0;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        double t = warp_sum(contrib[w]);
        if (lane == 0 && c0 + w < p) atomicAdd(pq + c0 + w, t);
    }
}

inline int chunk_width(int ld) { return (ld % 4 == 0) ? 4 : (ld % 2 == 0 ? 2 : 1); }

}  // namespace

void launch_sell_spmm(ofks_ctx *c, const double *val, const double *X, double *Y) {
    const int W = chunk_width(c->ld), nch = c->ld / W;
    const int64_t nw = (int64_t)c->n_slices * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_sell_spmm<w, 0><<<grid, 256, 0, c->stream>>>(nw, nch, c->p, c->ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, nullptr)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
}

void launch_sell_spmm_colnorm(ofks_ctx *c, const double *val, const double *X, double *Y, double *colsum) {
    const int W = chunk_width(c->ld), nch = c->ld / W;
    const int64_t nw = (int64_t)c->n_slices * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_sell_spmm<w, 1><<<grid, 256, 0, c->stream>>>(nw, nch, c->p, c->ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, colsum)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
}

void launch_pcg_apply(ofks_ctx *c, const double *Zin, double *P, double *Q, const double *beta_col,
                      const double *shift, double *pq, int first) {
    const int W = chunk_width(c->ld), nch = c->ld / W;
    const int64_t nw = (int64_t)c->n_slices * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_pcg_apply<w><<<grid, 256, 0, c->stream>>>(nw, nch, c->p, c->ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, c->d_valL, c->d_valB, Zin, P, Q, beta_col, shift, pq, first)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
}
