// SELL-C-sigma sparse times tall-skinny block products for the P2 matrices (paper Sec. 2.2:
// H X, B X; Eq. precondition-T: (L/2 - lambda_i B) z_i).
//
// Layout: rows of the free pattern are sorted by length inside windows of sigma rows and cut
// into slices of 32; entry j of lane l of slice s sits at slice_ptr[s] + 32 j + l, so the 32
// lanes of a warp read 32 consecutive column ids and values.  X and Y are row-major n x ld
// with ld a multiple of the chunk width W; a warp handles one (slice, W-column chunk) pair,
// each lane one row, and gathers W consecutive doubles of each neighbour row with vector
// loads.  Padding entries carry value 0 and repeat the row's last column id.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <class T, int W>
__device__ __forceinline__ void load_w(const T *__restrict__ p, T (&v)[W]) {
    if constexpr (W == 1) {
        v[0] = __ldg(p);
    } else if constexpr (sizeof(T) == 4 && W == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        using V2 = typename Vec2<T>::type;
#pragma unroll
        for (int w = 0; w < W; w += 2) {
            const V2 t = __ldg(reinterpret_cast<const V2 *>(p + w));
            v[w] = t.x; v[w + 1] = t.y;
        }
    }
}

template <class T, int W>
__device__ __forceinline__ void store_w(T *p, const T (&v)[W]) {
    if constexpr (W == 1) {
        p[0] = v[0];
    } else if constexpr (sizeof(T) == 4 && W == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        using V2 = typename Vec2<T>::type;
#pragma unroll
        for (int w = 0; w < W; w += 2) {
            V2 t;
            t.x = v[w]; t.y = v[w + 1];
            *reinterpret_cast<V2 *>(p + w) = t;
        }
    }
}

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Slices a warp takes in turn for one column chunk in the kernels that add column sums: the
// sums go out by one set of float64 atomics per warp instead of one per slice (measured on the
// float32 PCG apply: 1, 2, 4, 8, 16 slices -> 1170, 927, 911, 971, 982 us per launch on the
// 1.25 M-row chain; the plain product keeps one slice per warp, which measured faster).  Small
// problems keep one slice per warp so that the grid still fills the GPU (spw_for).
constexpr int SPW = 4;

inline int spw_for(int64_t units) {
    const int64_t fill = 152LL * 48;              // resident warps of one wave at ~40 registers
    return units / SPW >= fill ? SPW : (units / 2 >= fill ? 2 : 1);
}

// MODE 0: Y = A X.  MODE 1: also the column sums sum_rows X[r,c] Y[r,c] of the warp's slices,
// written (float64) to part[c * nsg + g] for slice group g (nsg groups of spw slices), to be
// added in group order (launch_col_fin).  T is the element type of the values and blocks; sums
// run in T.
template <class T, int W, int MODE>
__global__ void __launch_bounds__(256) k_sell_spmm(int64_t nwarps, int nchunks, int64_t n_slices, int spw_, int p, int ld,
                                                   const int *__restrict__ slice_ptr,
                                                   const int *__restrict__ slice_w,
                                                   const int *__restrict__ cols,
                                                   const int *__restrict__ perm,
                                                   const T *__restrict__ val,
                                                   const T *__restrict__ X, T *__restrict__ Y,
                                                   double *part) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nwarps) return;                       // whole warp leaves together
    const int spw = MODE == 1 ? spw_ : 1;           // without column sums one slice is faster
    const int chunk = (int)(wg % nchunks);
    const int64_t s0 = (wg / nchunks) * spw;
    const int64_t s1 = s0 + spw < n_slices ? s0 + spw : n_slices;
    const int c0 = chunk * W;
    T cs[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cs[w] = T(0);
    for (int64_t s = s0; s < s1; ++s) {
        const int base = slice_ptr[s], width = slice_w[s];
        const int r = perm[s * SELL_C + lane];
        T acc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = T(0);
        int e = base + lane;
        for (int j = 0; j < width; ++j, e += SELL_C) {
            const int c = __ldg(cols + e);
            const T v = __ldg(val + e);
            T x[W];
            load_w<T, W>(X + (int64_t)c * ld + c0, x);
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] = fma(v, x[w], acc[w]);
        }
        if (r >= 0) {
            store_w<T, W>(Y + (int64_t)r * ld + c0, acc);
            if constexpr (MODE == 1) {
                T xr[W];
                load_w<T, W>(X + (int64_t)r * ld + c0, xr);
#pragma unroll
                for (int w = 0; w < W; ++w) cs[w] = fma(xr[w], acc[w], cs[w]);
            }
        }
    }
    if constexpr (MODE == 1) {
        const int64_t nsg = (n_slices + spw - 1) / spw, g = wg / nchunks;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const T t = warp_sum_t(cs[w]);
            if (lane == 0) part[(int64_t)(c0 + w) * nsg + g] = (double)t;
        }
    }
}

// One Jacobi-PCG operator apply for all columns at once (Eq. precondition-T):
//   TZ = (L/2) Z - B Z diag(shift)  gathered over the neighbours of each row, then for the
//   own row  P <- Z + beta P,  Q <- TZ + beta Q  (so T P = Q), and the column sums P.Q of the
// warp's slices to part[c * nsg + g] (slice group g; added in group order by k_pcg_alpha).
// With first = 1: P = Z, Q = TZ.
template <class T, int W>
__global__ void __launch_bounds__(256) k_pcg_apply(int64_t nwarps, int nchunks, int64_t n_slices, int spw, int p, int ld,
                                                   const int *__restrict__ slice_ptr,
                                                   const int *__restrict__ slice_w,
                                                   const int *__restrict__ cols,
                                                   const int *__restrict__ perm,
                                                   const T *__restrict__ valL,
                                                   const T *__restrict__ valB,
                                                   const T *__restrict__ Z, T *P, T *Q,
                                                   const double *__restrict__ beta_col,
                                                   const double *__restrict__ shift, double *part,
                                                   int first) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nwarps) return;
    const int chunk = (int)(wg % nchunks);
    const int64_t s0 = (wg / nchunks) * spw;
    const int64_t s1 = s0 + spw < n_slices ? s0 + spw : n_slices;
    const int c0 = chunk * W;
    T sh[W], bt[W], contrib[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        sh[w] = T(shift[c0 + w]);
        bt[w] = first ? T(0) : T(beta_col[c0 + w]);
        contrib[w] = T(0);
    }
    for (int64_t s = s0; s < s1; ++s) {
        const int base = slice_ptr[s], width = slice_w[s];
        const int r = perm[s * SELL_C + lane];
        T aL[W], aB[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { aL[w] = T(0); aB[w] = T(0); }
        int e = base + lane;
        for (int j = 0; j < width; ++j, e += SELL_C) {
            const int c = __ldg(cols + e);
            const T vl = __ldg(valL + e), vb = __ldg(valB + e);
            T x[W];
            load_w<T, W>(Z + (int64_t)c * ld + c0, x);
#pragma unroll
            for (int w = 0; w < W; ++w) { aL[w] = fma(vl, x[w], aL[w]); aB[w] = fma(vb, x[w], aB[w]); }
        }
        if (r >= 0) {
            T zr[W], pr[W], qr[W];
            load_w<T, W>(Z + (int64_t)r * ld + c0, zr);
            if (!first) {
                load_w<T, W>(P + (int64_t)r * ld + c0, pr);
                load_w<T, W>(Q + (int64_t)r * ld + c0, qr);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const T tz = T(0.5) * aL[w] - sh[w] * aB[w];
                const T pn = first ? zr[w] : fma(bt[w], pr[w], zr[w]);
                const T qn = first ? tz : fma(bt[w], qr[w], tz);
                pr[w] = pn; qr[w] = qn;
                contrib[w] = fma(pn, qn, contrib[w]);
            }
            store_w<T, W>(P + (int64_t)r * ld + c0, pr);
            store_w<T, W>(Q + (int64_t)r * ld + c0, qr);
        }
    }
    const int64_t nsg = (n_slices + spw - 1) / spw, g = wg / nchunks;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const T t = warp_sum_t(contrib[w]);
        if (lane == 0) part[(int64_t)(c0 + w) * nsg + g] = (double)t;
    }
}

// The float32 PCG apply on the type-grouped SELL with every PCG block chunk-major: element
// (r, c) at ((c / 4) ns + r) 4 + c % 4 (ns = n rounded up to 32), rows in type order.  A warp
// takes spw consecutive slices in turn for one 4-column chunk and writes its column sums P.Q once
// at the end.  Its lanes are 32 consecutive rows of one lattice node type, so for one entry index
// their neighbours are (mostly) 32 consecutive rows of one type: each 16-byte gather of the warp
// reads 512 contiguous bytes, and the lanes' own P and Q pieces are contiguous too.
__global__ void __launch_bounds__(256, 4) k_pcg_apply_zc(int64_t nwarps, int nchunks, int64_t n_slices, int spw, int p,
                                                      int64_t n, int64_t ns, const int *__restrict__ slice_ptr,
                                                      const int *__restrict__ slice_w,
                                                      const int *__restrict__ cols,
                                                      const float *__restrict__ valL,
                                                      const float *__restrict__ valB,
                                                      const float *__restrict__ Zc, float *P, float *Q,
                                                      const double *__restrict__ beta_col,
                                                      const double *__restrict__ shift, double *part, int first) {
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= nwarps) return;
    const int chunk = (int)(wg % nchunks);
    const int64_t s0 = (wg / nchunks) * spw;
    const int64_t s1 = s0 + spw < n_slices ? s0 + spw : n_slices;
    const int c0 = chunk * 4;
    const int64_t cbase = (int64_t)chunk * ns * 4;
    const float *Zk = Zc + cbase;
    float *Pk = P + cbase, *Qk = Q + cbase;
    float sh[4], bt[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        sh[w] = (float)shift[c0 + w];
        bt[w] = first ? 0.f : (float)beta_col[c0 + w];
    }
    float contrib[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t s = s0; s < s1; ++s) {
        const int base = slice_ptr[s], width = slice_w[s];
        const int64_t r = s * SELL_C + lane;
        float aL[4] = {0.f, 0.f, 0.f, 0.f}, aB[4] = {0.f, 0.f, 0.f, 0.f};
        // four entries per pass with all their loads issued before the first multiply-add: four
        // gathers in flight per lane (with the register cap of four CTAs per SM this measured
        // 0.195 ms per launch against 0.34 ms for one entry per pass on the 60x32x30 chain)
        int e = base + lane, j = 0;
        for (; j + 4 <= width; j += 4, e += 4 * SELL_C) {
            int cc[4];
            float vl[4], vb[4];
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cc[u] = __ldg(cols + e + u * SELL_C);
#pragma unroll
            for (int u = 0; u < 4; ++u) { vl[u] = __ldg(valL + e + u * SELL_C); vb[u] = __ldg(valB + e + u * SELL_C); }
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __ldg(reinterpret_cast<const float4 *>(Zk + (int64_t)cc[u] * 4));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                aL[0] = fmaf(vl[u], x[u].x, aL[0]); aL[1] = fmaf(vl[u], x[u].y, aL[1]);
                aL[2] = fmaf(vl[u], x[u].z, aL[2]); aL[3] = fmaf(vl[u], x[u].w, aL[3]);
                aB[0] = fmaf(vb[u], x[u].x, aB[0]); aB[1] = fmaf(vb[u], x[u].y, aB[1]);
                aB[2] = fmaf(vb[u], x[u].z, aB[2]); aB[3] = fmaf(vb[u], x[u].w, aB[3]);
            }
        }
        for (; j < width; ++j, e += SELL_C) {
            const int c = __ldg(cols + e);
            const float vl = __ldg(valL + e), vb = __ldg(valB + e);
            const float4 x = __ldg(reinterpret_cast<const float4 *>(Zk + (int64_t)c * 4));
            aL[0] = fmaf(vl, x.x, aL[0]); aL[1] = fmaf(vl, x.y, aL[1]); aL[2] = fmaf(vl, x.z, aL[2]); aL[3] = fmaf(vl, x.w, aL[3]);
            aB[0] = fmaf(vb, x.x, aB[0]); aB[1] = fmaf(vb, x.y, aB[1]); aB[2] = fmaf(vb, x.z, aB[2]); aB[3] = fmaf(vb, x.w, aB[3]);
        }
        if (r >= n) continue;
        const int64_t o = r * 4;
        const float4 z4 = __ldg(reinterpret_cast<const float4 *>(Zk + o));
        const float zr[4] = {z4.x, z4.y, z4.z, z4.w};
        float pr[4] = {0.f, 0.f, 0.f, 0.f}, qr[4] = {0.f, 0.f, 0.f, 0.f};
        if (!first) {
            const float4 p4 = *reinterpret_cast<const float4 *>(Pk + o), q4 = *reinterpret_cast<const float4 *>(Qk + o);
            pr[0] = p4.x; pr[1] = p4.y; pr[2] = p4.z; pr[3] = p4.w;
            qr[0] = q4.x; qr[1] = q4.y; qr[2] = q4.z; qr[3] = q4.w;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float tz = 0.5f * aL[w] - sh[w] * aB[w];
            const float pn = first ? zr[w] : fmaf(bt[w], pr[w], zr[w]);
            const float qn = first ? tz : fmaf(bt[w], qr[w], tz);
            pr[w] = pn; qr[w] = qn;
            contrib[w] = fmaf(pn, qn, contrib[w]);
        }
        *reinterpret_cast<float4 *>(Pk + o) = make_float4(pr[0], pr[1], pr[2], pr[3]);
        *reinterpret_cast<float4 *>(Qk + o) = make_float4(qr[0], qr[1], qr[2], qr[3]);
    }
    const int64_t nsg = (n_slices + spw - 1) / spw, g = wg / nchunks;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const float t = warp_sum_t(contrib[w]);
        if (lane == 0) part[(int64_t)(c0 + w) * nsg + g] = (double)t;
    }
}

inline int chunk_width(int ld) { return (ld % 4 == 0) ? 4 : (ld % 2 == 0 ? 2 : 1); }

// ---- float32 SpMM with the neighbour rows staged through shared memory (ld = 4 NC <= 64)
//
// One warp per SELL slice (lane = row).  For each entry index j the warp copies the 32 neighbour
// rows X[c_l, 0:ld] into a shared tile with 16-byte asynchronous copies (cp.async, straight from
// L2 into shared memory): flat item i = (row k, 16-byte chunk q) with consecutive lanes on
// consecutive chunks of one row, so one copy instruction covers about three whole rows (~6 cache
// lines) instead of 32 rows' pieces; each lane then multiplies its own row from the tile.  The
// copies run WS_STAGES - 1 entries ahead of the multiply-adds (a ring of WS_STAGES tiles per
// warp, row stride ws_stride(NC) floats: an odd multiple of 4 modulo 32 words, so the 16-byte
// reads of 8 lanes at a time hit distinct banks), and the column ids and values of 8 entries
// are loaded together.  The result rows leave through a tile as whole-row coalesced stores.
// MODE 1 also forms the column sums X[r,c] Y[r,c] of the slice (per warp, in lane order) into
// part[c * n_slices + slice].
constexpr int WS_WARPS = 2;                       // warps per block
constexpr int WS_STAGES = 3;                      // tiles in flight per warp
constexpr int WS_BATCH = 8;                       // entries whose column ids and values load together

__host__ __device__ constexpr int ws_stride(int nc) { return (nc % 2 == 1) ? 4 * nc : 4 * nc + 4; }
// shared memory of one block: per warp WS_STAGES tiles of 32 rows and WS_STAGES x 32 values
__host__ __device__ constexpr int ws_smem(int nc) { return WS_WARPS * WS_STAGES * 32 * (ws_stride(nc) + 1) * 4; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

template <int NC, int MODE>
__global__ void __launch_bounds__(WS_WARPS * 32) k_spmm_ws(int64_t n_slices, int p, const int *__restrict__ slice_ptr,
                                                          const int *__restrict__ slice_w, const int *__restrict__ cols,
                                                          const int *__restrict__ perm, const float *__restrict__ val,
                                                          const float *__restrict__ X, float *__restrict__ Y,
                                                          double *part) {
    constexpr int LD = 4 * NC, STR = ws_stride(NC), TS = 32 * STR;
    extern __shared__ __align__(16) float wsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = blockIdx.x * (int64_t)WS_WARPS + warp;
    if (s >= n_slices) return;                      // whole warp leaves together
    float *T = wsm + (size_t)warp * WS_STAGES * (TS + 32);
    float *V = T + WS_STAGES * TS;                  // the lane's value of each staged entry
    const int base = slice_ptr[s], width = slice_w[s];
    const int r = perm[s * SELL_C + lane];
    float acc[LD];
#pragma unroll
    for (int k = 0; k < LD; ++k) acc[k] = 0.f;
    // iteration j copies entry j's rows and multiplies entry j - (WS_STAGES - 1); the copy groups
    // are committed one per iteration (empty past the last entry), so waiting until at most
    // WS_STAGES - 1 groups are pending completes the group of the entry multiplied
    for (int j0 = 0; j0 < width + WS_STAGES - 1; j0 += WS_BATCH) {
        int cc[WS_BATCH];
        float vv[WS_BATCH];
#pragma unroll
        for (int u = 0; u < WS_BATCH; ++u) {
            const int j = j0 + u;
            cc[u] = j < width ? __ldg(cols + base + j * SELL_C + lane) : 0;
            vv[u] = j < width ? __ldg(val + base + j * SELL_C + lane) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < WS_BATCH; ++u) {
            const int j = j0 + u;
            if (j >= width + WS_STAGES - 1) break;  // warp-uniform
            if (j < width) {
                const int st = j % WS_STAGES;
                float *Ts = T + st * TS;
                V[st * 32 + lane] = vv[u];
#pragma unroll
                for (int it = 0; it < NC; ++it) {
                    const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
                    const int ck = __shfl_sync(0xffffffffu, cc[u], k);
                    cp_async16(Ts + k * STR + 4 * q, X + (int64_t)ck * LD + 4 * q);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            const int jc = j - (WS_STAGES - 1);
            if (jc < 0) continue;
            asm volatile("cp.async.wait_group %0;" ::"n"(WS_STAGES - 1) : "memory");
            __syncwarp();
            const int st = jc % WS_STAGES;
            const float *Ts = T + st * TS;
            const float vl = V[st * 32 + lane];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                const float4 x = *reinterpret_cast<const float4 *>(Ts + lane * STR + 4 * q);
                acc[4 * q] = fmaf(vl, x.x, acc[4 * q]);
                acc[4 * q + 1] = fmaf(vl, x.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(vl, x.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(vl, x.w, acc[4 * q + 3]);
            }
            __syncwarp();                           // the tile is refilled WS_STAGES entries later
        }
    }
    // the slice's rows out through the tile as whole-row stores
#pragma unroll
    for (int q = 0; q < NC; ++q)
        *reinterpret_cast<float4 *>(T + lane * STR + 4 * q) =
            make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (int it = 0; it < NC; ++it) {
        const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
        const int rk = __shfl_sync(0xffffffffu, r, k);
        if (rk >= 0)
            *reinterpret_cast<float4 *>(Y + (int64_t)rk * LD + 4 * q) = *reinterpret_cast<const float4 *>(T + k * STR + 4 * q);
    }
    if constexpr (MODE == 1) {
        // column sums X[r, c] Y[r, c] over the slice's rows: the own rows of X through the tile
        __syncwarp();
#pragma unroll
        for (int it = 0; it < NC; ++it) {
            const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
            const int rk = __shfl_sync(0xffffffffu, r, k);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rk >= 0) v = __ldg(reinterpret_cast<const float4 *>(X + (int64_t)rk * LD) + q);
            *reinterpret_cast<float4 *>(T + k * STR + 4 * q) = v;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const float4 x = *reinterpret_cast<const float4 *>(T + lane * STR + 4 * q);
            const float c4[4] = {x.x * acc[4 * q], x.y * acc[4 * q + 1], x.z * acc[4 * q + 2], x.w * acc[4 * q + 3]};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const float t = warp_sum_t(c4[w]);
                if (lane == 0) part[(int64_t)(4 * q + w) * n_slices + s] = (double)t;
            }
        }
    }
}

// The float32 PCG operator apply of k_pcg_apply with the same staging, on row-major blocks of
// width w = 4 NC <= 32: for each entry index the 32 neighbour rows of Z go through the warp's
// tile, each lane accumulates L Z and B Z for its row; then the lane's own rows of Z, P and Q are
// staged (coalesced) and P <- Z + beta P, Q <- (L/2 - shift B) Z + beta Q are formed and written
// back through the tiles, with the column sums P.Q of the slice into part[c * n_slices + slice].
template <int NC>
__global__ void __launch_bounds__(WS_WARPS * 32) k_pcg_apply_ws(int64_t n_slices, int pc, const int *__restrict__ slice_ptr,
                                                               const int *__restrict__ slice_w, const int *__restrict__ cols,
                                                               const int *__restrict__ perm, const float *__restrict__ valL,
                                                               const float *__restrict__ valB, const float *__restrict__ Z,
                                                               float *P, float *Q, const double *__restrict__ beta_col,
                                                               const double *__restrict__ shift, double *part, int first) {
    constexpr int LD = 4 * NC, STR = ws_stride(NC);
    __shared__ __align__(16) float tile[WS_WARPS][3][32 * STR];
    __shared__ float ssh[LD], sbt[LD];
    for (int k = threadIdx.x; k < LD; k += blockDim.x) {
        ssh[k] = (float)shift[k];
        sbt[k] = first ? 0.f : (float)beta_col[k];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = blockIdx.x * (int64_t)WS_WARPS + warp;
    if (s >= n_slices) return;                      // whole warp leaves together
    float *T0 = tile[warp][0], *T1 = tile[warp][1], *T2 = tile[warp][2];
    const int base = slice_ptr[s], width = slice_w[s];
    const int r = perm[s * SELL_C + lane];
    float aL[LD], aB[LD];
#pragma unroll
    for (int k = 0; k < LD; ++k) { aL[k] = 0.f; aB[k] = 0.f; }
    for (int j = 0; j < width; ++j) {
        const int e = base + j * SELL_C + lane;
        const int cl = __ldg(cols + e);
        const float vl = __ldg(valL + e), vb = __ldg(valB + e);
#pragma unroll
        for (int it = 0; it < NC; ++it) {
            const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
            const int ck = __shfl_sync(0xffffffffu, cl, k);
            *reinterpret_cast<float4 *>(T0 + k * STR + 4 * q) = __ldg(reinterpret_cast<const float4 *>(Z + (int64_t)ck * LD) + q);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const float4 x = *reinterpret_cast<const float4 *>(T0 + lane * STR + 4 * q);
            const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                aL[4 * q + w] = fmaf(vl, xs[w], aL[4 * q + w]);
                aB[4 * q + w] = fmaf(vb, xs[w], aB[4 * q + w]);
            }
        }
        __syncwarp();
    }
    // own rows of Z, P, Q (zero for the padding rows of the last slice)
#pragma unroll
    for (int it = 0; it < NC; ++it) {
        const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
        const int rk = __shfl_sync(0xffffffffu, r, k);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4 *>(T0 + k * STR + 4 * q) = rk >= 0 ? __ldg(reinterpret_cast<const float4 *>(Z + (int64_t)rk * LD) + q) : z;
        *reinterpret_cast<float4 *>(T1 + k * STR + 4 * q) = (rk >= 0 && !first) ? *(reinterpret_cast<const float4 *>(P + (int64_t)rk * LD) + q) : z;
        *reinterpret_cast<float4 *>(T2 + k * STR + 4 * q) = (rk >= 0 && !first) ? *(reinterpret_cast<const float4 *>(Q + (int64_t)rk * LD) + q) : z;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const float4 z4 = *reinterpret_cast<const float4 *>(T0 + lane * STR + 4 * q);
        const float4 p4 = *reinterpret_cast<const float4 *>(T1 + lane * STR + 4 * q);
        const float4 q4 = *reinterpret_cast<const float4 *>(T2 + lane * STR + 4 * q);
        const float zs[4] = {z4.x, z4.y, z4.z, z4.w}, ps[4] = {p4.x, p4.y, p4.z, p4.w}, qs[4] = {q4.x, q4.y, q4.z, q4.w};
        float pn[4], qn[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int col = 4 * q + w;
            const float tz = 0.5f * aL[col] - ssh[col] * aB[col];
            pn[w] = fmaf(sbt[col], ps[w], zs[w]);
            qn[w] = fmaf(sbt[col], qs[w], tz);
            const float t = warp_sum_t(r >= 0 ? pn[w] * qn[w] : 0.f);
            if (lane == 0) part[(int64_t)col * n_slices + s] = (double)t;
        }
        *reinterpret_cast<float4 *>(T1 + lane * STR + 4 * q) = make_float4(pn[0], pn[1], pn[2], pn[3]);
        *reinterpret_cast<float4 *>(T2 + lane * STR + 4 * q) = make_float4(qn[0], qn[1], qn[2], qn[3]);
    }
    __syncwarp();
#pragma unroll
    for (int it = 0; it < NC; ++it) {
        const int i = it * 32 + lane, k = i / NC, q = i - k * NC;
        const int rk = __shfl_sync(0xffffffffu, r, k);
        if (rk >= 0) {
            *(reinterpret_cast<float4 *>(P + (int64_t)rk * LD) + q) = *reinterpret_cast<const float4 *>(T1 + k * STR + 4 * q);
            *(reinterpret_cast<float4 *>(Q + (int64_t)rk * LD) + q) = *reinterpret_cast<const float4 *>(T2 + k * STR + 4 * q);
        }
    }
}

// the staged PCG apply applies at widths 8..32 (multiples of 4) of float32 blocks on the main SELL
inline bool pcg_ws_fits(int w) { return w % 4 == 0 && w >= 8 && w <= 32; }

template <int MODE>
bool launch_spmm_ws(ofks_ctx *c, int ld, const float *val, const float *X, float *Y, double *colsum) {
    if (ld % 4 || ld < 8 || ld > 64) return false;
    const unsigned grid = (unsigned)((c->n_slices + WS_WARPS - 1) / WS_WARPS);
#define WS_(nc) { cudaFuncSetAttribute(k_spmm_ws<nc, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, ws_smem(nc)); \
        k_spmm_ws<nc, MODE><<<grid, WS_WARPS * 32, ws_smem(nc), c->stream>>>(c->n_slices, c->p, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, c->d_cpart); }
    switch (ld / 4) {
        case 2: WS_(2); break; case 3: WS_(3); break; case 4: WS_(4); break; case 5: WS_(5); break;
        case 6: WS_(6); break; case 7: WS_(7); break; case 8: WS_(8); break; case 9: WS_(9); break;
        case 10: WS_(10); break; case 11: WS_(11); break; case 12: WS_(12); break; case 13: WS_(13); break;
        case 14: WS_(14); break; case 15: WS_(15); break; default: WS_(16); break;
    }
#undef WS_
    c->kernels += 1;
    if (MODE == 1) launch_col_fin(c, c->p, c->p, c->n_slices, c->d_cpart, colsum);
    return true;
}

// ---- half-warp-per-row forms for float32 blocks (the mixed form)
//
// With float32 blocks the lane-per-row kernels above are limited by L1 wavefronts, not by
// HBM: each lane gathers a 16-byte piece of a different neighbour row, so one load instruction
// touches 32 cache lines.  Here each half-warp takes one row and its 16 lanes split the row's
// ld columns (VPL consecutive floats each), so one gather instruction reads two contiguous
// neighbour rows; both half-warps share the slice, whose column ids and values are read with
// half-warp broadcasts and stay in L1 for the slice's other rows.  Warps stride over
// (slice, row pair) items; column sums are reduced in the block and written once per block.
constexpr int RW = 8;                  // warps per block

template <int VPL>
__device__ __forceinline__ void ldf(const float *__restrict__ p, float (&v)[VPL]) {
#pragma unroll
    for (int w = 0; w < VPL; w += 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p + w));
        v[w] = t.x; v[w + 1] = t.y; v[w + 2] = t.z; v[w + 3] = t.w;
    }
}

template <int VPL>
__device__ __forceinline__ void stf(float *p, const float (&v)[VPL]) {
#pragma unroll
    for (int w = 0; w < VPL; w += 4) *reinterpret_cast<float4 *>(p + w) = make_float4(v[w], v[w + 1], v[w + 2], v[w + 3]);
}

// epilogue of one row (own-row loads, stores, column sums) for the three modes
template <int VPL, int MODE>
__device__ __forceinline__ void rows_epilogue(int r, int ld, int c0, int first, const float *__restrict__ X, float *Y,
                                              float *Y2, const float (&aA)[VPL], const float (&aB)[VPL],
                                              const float (&sh)[VPL], const float (&bt)[VPL], float (&csum)[VPL]) {
    float *yr = Y + (int64_t)r * ld + c0;
    if (MODE == 0) {
        stf<VPL>(yr, aA);
    } else if (MODE == 1) {
        float xr[VPL];
        ldf<VPL>(X + (int64_t)r * ld + c0, xr);
        stf<VPL>(yr, aA);
#pragma unroll
        for (int v = 0; v < VPL; ++v) csum[v] = fmaf(xr[v], aA[v], csum[v]);
    } else {
        float zr[VPL], pr[VPL], qr[VPL];
        ldf<VPL>(X + (int64_t)r * ld + c0, zr);
        float *q = Y2 + (int64_t)r * ld + c0;
        if (!first) { ldf<VPL>(yr, pr); ldf<VPL>(q, qr); }
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const float tz = 0.5f * aA[v] - sh[v] * aB[v];
            const float pn = first ? zr[v] : fmaf(bt[v], pr[v], zr[v]);
            const float qn = first ? tz : fmaf(bt[v], qr[v], tz);
            pr[v] = pn; qr[v] = qn;
            csum[v] = fmaf(pn, qn, csum[v]);
        }
        stf<VPL>(yr, pr);
        stf<VPL>(q, qr);
    }
}

// MODE 0: Y = A X.  MODE 1: Y = A X and the block's column sums X[:,c].Y[:,c] into part[c grid +
// block].  MODE 2: the PCG apply of
// k_pcg_apply (X = Z, Y = P, Y2 = Q, A = L values, B = B values).  Each half-warp carries two
// rows of the same slice, so two independent gathers are in flight per step of the entry loop.
template <int VPL, int MODE>
__global__ void __launch_bounds__(RW * 32) k_rows_f32(int n_slices, int p, int ld, const int *__restrict__ slice_ptr,
                                                      const int *__restrict__ slice_w, const int *__restrict__ cols,
                                                      const int *__restrict__ perm, const float *__restrict__ valA,
                                                      const float *__restrict__ valB, const float *__restrict__ X,
                                                      float *Y, float *Y2, const double *__restrict__ beta_col,
                                                      const double *__restrict__ shift, double *part, int first) {
    __shared__ float red[RW][VPL * 16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4;
    const int c0 = (lane & 15) * VPL;
    const bool on = c0 < ld;
    float csum[VPL], sh[VPL], bt[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        csum[v] = 0.f;
        sh[v] = (MODE == 2 && on) ? (float)shift[c0 + v] : 0.f;
        bt[v] = (MODE == 2 && on && !first) ? (float)beta_col[c0 + v] : 0.f;
    }
    const int64_t items = (int64_t)n_slices * (SELL_C / 4);
    for (int64_t w = blockIdx.x * (int64_t)RW + warp; w < items; w += (int64_t)gridDim.x * RW) {
        const int s = (int)(w / (SELL_C / 4));
        const int l0 = (int)(w % (SELL_C / 4)) * 4 + half * 2, l1 = l0 + 1;
        const int r0 = perm[s * SELL_C + l0], r1 = perm[s * SELL_C + l1];
        if (!on || (r0 < 0 && r1 < 0)) continue;
        const int width = slice_w[s];
        const int64_t e0 = slice_ptr[s] + l0;          // row l1's entries sit one further
        float a0[VPL], b0[VPL], a1[VPL], b1[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) { a0[v] = 0.f; b0[v] = 0.f; a1[v] = 0.f; b1[v] = 0.f; }
#pragma unroll 4
        for (int j = 0; j < width; ++j) {
            const int64_t e = e0 + (int64_t)j * SELL_C;
            const int2 cc = *reinterpret_cast<const int2 *>(cols + e);      // rows l0, l1 (8-byte aligned: l0 even)
            const float2 va = *reinterpret_cast<const float2 *>(valA + e);
            float2 vb = make_float2(0.f, 0.f);
            if (MODE == 2) vb = *reinterpret_cast<const float2 *>(valB + e);
            float x0[VPL], x1[VPL];
            ldf<VPL>(X + (int64_t)cc.x * ld + c0, x0);
            ldf<VPL>(X + (int64_t)cc.y * ld + c0, x1);
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                a0[v] = fmaf(va.x, x0[v], a0[v]);
                a1[v] = fmaf(va.y, x1[v], a1[v]);
                if (MODE == 2) { b0[v] = fmaf(vb.x, x0[v], b0[v]); b1[v] = fmaf(vb.y, x1[v], b1[v]); }
            }
        }
        if (r0 >= 0) rows_epilogue<VPL, MODE>(r0, ld, c0, first, X, Y, Y2, a0, b0, sh, bt, csum);
        if (r1 >= 0) rows_epilogue<VPL, MODE>(r1, ld, c0, first, X, Y, Y2, a1, b1, sh, bt, csum);
    }
    if (MODE == 0) return;
#pragma unroll
    for (int v = 0; v < VPL; ++v) csum[v] += __shfl_down_sync(0xffffffffu, csum[v], 16);
    if (half == 0)
#pragma unroll
        for (int v = 0; v < VPL; ++v) red[warp][c0 + v] = on ? csum[v] : 0.f;
    __syncthreads();
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < RW; ++w) t += red[w][c];
        part[(int64_t)c * gridDim.x + blockIdx.x] = (double)t;
    }
}

// half-warp-per-row launch for float32 blocks; false when the shapes do not suit it.  MODE 1 adds
// the column sums into colsum; MODE 2 leaves its column partials for k_pcg_alpha (pq_units).
template <int MODE>
bool launch_rows_f32(ofks_ctx *c, int ld, int pc, const float *valA, const float *valB, const float *X, float *Y, float *Y2,
                     const double *beta_col, const double *shift, double *colsum, int first) {
    if (!c->prm.spmm_f32_rows || ld < 16 || ld % 4 || ld > 256) return false;
    const int64_t items = (int64_t)c->n_slices * (SELL_C / 4);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + RW - 1) / RW, 152 * 8));
#define R_(v)                                                                                                      \
    k_rows_f32<v, MODE><<<grid, RW * 32, 0, c->stream>>>(c->n_slices, pc, ld, c->d_slice_ptr, c->d_slice_w,     \
                                                         c->d_cols, c->d_perm, valA, valB, X, Y, Y2, beta_col,    \
                                                         shift, c->d_cpart, first)
    if (ld <= 64) R_(4);
    else if (ld <= 128) R_(8);
    else R_(16);
#undef R_
    c->kernels += 1;
    if (MODE == 1) launch_col_fin(c, pc, pc, grid, c->d_cpart, colsum);
    if (MODE == 2) c->pq_units = grid;
    return true;
}

}  // namespace

template <class T>
void launch_sell_spmm(ofks_ctx *c, const T *val, const T *X, T *Y) {
    if constexpr (sizeof(T) == 4) {
        if (launch_rows_f32<0>(c, c->ld, c->p, val, nullptr, X, Y, nullptr, nullptr, nullptr, nullptr, 0)) return;
        if (c->prm.spmm_f32_rows == 0 && launch_spmm_ws<0>(c, c->ld, val, X, Y, nullptr)) return;
    }
    const int W = chunk_width(c->ld), nch = c->ld / W;
    const int64_t nw = (int64_t)c->n_slices * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_sell_spmm<T, w, 0><<<grid, 256, 0, c->stream>>>(nw, nch, (int64_t)c->n_slices, 1, c->p, c->ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, nullptr)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
}

template <class T>
void launch_sell_spmm_colnorm(ofks_ctx *c, const T *val, const T *X, T *Y, double *colsum) {
    if constexpr (sizeof(T) == 4) {
        if (launch_rows_f32<1>(c, c->ld, c->p, val, nullptr, X, Y, nullptr, nullptr, nullptr, colsum, 0)) return;
        if (c->prm.spmm_f32_rows == 0 && launch_spmm_ws<1>(c, c->ld, val, X, Y, colsum)) return;
    }
    const int W = chunk_width(c->ld), nch = c->ld / W;
    const int spw = spw_for((int64_t)c->n_slices * nch);
    const int64_t nsg = ((int64_t)c->n_slices + spw - 1) / spw, nw = nsg * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_sell_spmm<T, w, 1><<<grid, 256, 0, c->stream>>>(nw, nch, (int64_t)c->n_slices, spw, c->p, c->ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, c->d_cpart)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
    launch_col_fin(c, c->p, c->p, nsg, c->d_cpart, colsum);
}

template <class T>
void launch_pcg_apply(ofks_ctx *c, const T *valL, const T *valB, const T *Zin, int zc, T *P, T *Q, const double *beta_col,
                      const double *shift, double *pq, int first, int w, int pc) {
    if constexpr (sizeof(T) == 4) {
        if (!zc && c->prm.pcg_staged && pcg_ws_fits(w)) {
            const unsigned grid = (unsigned)((c->n_slices + WS_WARPS - 1) / WS_WARPS);
#define PW_(nc) k_pcg_apply_ws<nc><<<grid, WS_WARPS * 32, 0, c->stream>>>(c->n_slices, pc, c->d_slice_ptr, c->d_slice_w, \
        c->d_cols, c->d_perm, (const float *)valL, (const float *)valB, (const float *)Zin, (float *)P, (float *)Q, beta_col, \
        shift, c->d_cpart, first)
            switch (w / 4) {
                case 2: PW_(2); break; case 3: PW_(3); break; case 4: PW_(4); break; case 5: PW_(5); break;
                case 6: PW_(6); break; case 7: PW_(7); break; default: PW_(8); break;
            }
#undef PW_
            c->kernels += 1;
            c->pq_units = c->n_slices;
            return;
        }
        if (zc) {
            const int nch = w / 4;
            const int spw = spw_for((int64_t)c->n_tslices * nch);
            const int64_t nsg = ((int64_t)c->n_tslices + spw - 1) / spw, nw = nsg * nch;
            k_pcg_apply_zc<<<(unsigned)((nw * 32 + 255) / 256), 256, 0, c->stream>>>(
                nw, nch, (int64_t)c->n_tslices, spw, pc, c->n, c->n_slots, c->d_tslice_ptr, c->d_tslice_w, c->d_tcols,
                c->d_tvalL, c->d_tvalB, (const float *)Zin, (float *)P, (float *)Q, beta_col, shift,
                c->d_cpart, first);
            c->kernels += 1;
            c->pq_units = nsg;
            return;
        }
    }
    if constexpr (sizeof(T) == 4)
        if (launch_rows_f32<2>(c, w, pc, valL, valB, Zin, P, Q, beta_col, shift, pq, first)) return;
    const int W = chunk_width(w), nch = w / W;
    const int spw = spw_for((int64_t)c->n_slices * nch);
    const int64_t nsg = ((int64_t)c->n_slices + spw - 1) / spw, nw = nsg * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(v) k_pcg_apply<T, v><<<grid, 256, 0, c->stream>>>(nw, nch, (int64_t)c->n_slices, spw, pc, w, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, valL, valB, Zin, P, Q, beta_col, shift, c->d_cpart, first)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
    c->pq_units = nsg;
}

template <class T>
void launch_sell_spmm_ld(ofks_ctx *c, const T *val, const T *X, T *Y, int ld) {
    const int W = chunk_width(ld), nch = ld / W;
    const int64_t nw = (int64_t)c->n_slices * nch;
    const unsigned grid = (unsigned)((nw * 32 + 255) / 256);
#define L_(w) k_sell_spmm<T, w, 0><<<grid, 256, 0, c->stream>>>(nw, nch, (int64_t)c->n_slices, 1, ld, ld, c->d_slice_ptr, \
        c->d_slice_w, c->d_cols, c->d_perm, val, X, Y, nullptr)
    if (W == 4) L_(4); else if (W == 2) L_(2); else L_(1);
#undef L_
    c->kernels += 1;
}

template void launch_sell_spmm_ld<float>(ofks_ctx *, const float *, const float *, float *, int);
template void launch_sell_spmm<double>(ofks_ctx *, const double *, const double *, double *);
template void launch_sell_spmm<float>(ofks_ctx *, const float *, const float *, float *);
template void launch_sell_spmm_colnorm<double>(ofks_ctx *, const double *, const double *, double *, double *);
template void launch_sell_spmm_colnorm<float>(ofks_ctx *, const float *, const float *, float *, double *);
template void launch_pcg_apply<double>(ofks_ctx *, const double *, const double *, const double *, int, double *,
                                       double *, const double *, const double *, double *, int, int, int);
template void launch_pcg_apply<float>(ofks_ctx *, const float *, const float *, const float *, int, float *, float *,
                                      const double *, const double *, double *, int, int, int);
