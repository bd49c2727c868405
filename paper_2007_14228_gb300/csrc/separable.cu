// Separable preconditioner for the Hartree CG on lattice meshes (fast diagonalization).
//
// On a tensor-product lattice the P2 stiffness of the Poisson problem (paper Sec. 2.2) is
// spectrally equivalent, with constants independent of the grading and of the cells' aspect
// ratios, to the separable operator
//     A_sep = Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz
// built from the 1-D piecewise-linear stiffness K_d and lumped mass M_d on the lattice
// coordinates of each axis (Dirichlet ends removed).  With the per-axis generalized
// eigenvectors K_d S_d = M_d S_d diag(lam_d), S_d^T M_d S_d = I,
//     A_sep^-1 = (Sx (x) Sy (x) Sz) diag(1 / (lam_x,i + lam_y,j + lam_z,k)) (Sx (x) Sy (x) Sz)^T,
// i.e. three dense contractions along the axes, a pointwise scaling and three more.  The CG
// keeps its iteration count near twenty whatever the mesh size (the point Jacobi
// preconditioner needs hundreds to thousands on these graded meshes).  The contractions run in
// float32 (the preconditioner only has to be a fixed symmetric positive definite operator;
// the CG itself stays in float64).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace {

// Eigen-decomposition of a dense symmetric n x n matrix (row-major, overwritten) by cyclic
// Jacobi rotations: on return a holds the eigenvalues on its diagonal and v the eigenvectors
// in its columns.  Returns false if the sweeps did not converge.
bool jacobi_eigen(int n, std::vector<double> &a, std::vector<double> &v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    double norm = 0.0;
    for (double x : a) norm += x * x;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (off <= 1e-30 * norm) return true;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) <= 1e-300) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                // rotation angle that zeroes a_pq: tan(2 phi) = 2 a_pq / (a_qq - a_pp)
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {            // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = cs * akp - sn * akq;
                    a[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {            // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = cs * apk - sn * aqk;
                    a[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    v[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    return false;
}

// One axis: coordinates x_0 .. x_{L-1} (Dirichlet ends), n = L - 2 interior points.
// S (n x n, row-major S[a][i]: interior point a, mode i) and lam (n) with K S = M S diag(lam).
bool axis_modes(const std::vector<double> &x, std::vector<double> &S, std::vector<double> &lam) {
    const int L = (int)x.size(), n = L - 2;
    if (n < 1) return false;
    std::vector<double> h(L - 1), m(n), T((size_t)n * n, 0.0);
    for (int e = 0; e < L - 1; ++e) {
        h[e] = x[e + 1] - x[e];
        if (!(h[e] > 0.0)) return false;
    }
    for (int a = 0; a < n; ++a) m[a] = 0.5 * (h[a] + h[a + 1]);
    // T = M^-1/2 K M^-1/2 for the tridiagonal stiffness K
    for (int a = 0; a < n; ++a) {
        T[(size_t)a * n + a] = (1.0 / h[a] + 1.0 / h[a + 1]) / m[a];
        if (a + 1 < n) {
            const double o = -1.0 / (h[a + 1] * std::sqrt(m[a] * m[a + 1]));
            T[(size_t)a * n + a + 1] = o;
            T[(size_t)(a + 1) * n + a] = o;
        }
    }
    std::vector<double> Q;
    if (!jacobi_eigen(n, T, Q)) return false;
    lam.resize(n);
    S.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) lam[i] = T[(size_t)i * n + i];
    for (int a = 0; a < n; ++a)
        for (int i = 0; i < n; ++i) S[(size_t)a * n + i] = Q[(size_t)a * n + i] / std::sqrt(m[a]);
    return true;
}

// Interior lattice tensor (a, b, c) <- the CG residual (element type E, innermost axis stored
// with stride ldc >= nz; with tlo the value is split in two, t + tlo, the low part the rounding
// error of the high one).  With it >= 0 the CG update of iteration it is fused in first (the
// scalars protocol of the Hartree CG in fields.cu): alpha = rz/pq, U += alpha p, r -= alpha q,
// rr' += r.r, and the next pq slot is cleared.
template <class E>
__global__ void __launch_bounds__(256) k_sep_gather(int nx, int ny, int nz, int ldc, int Ly, int Lz,
                                                    const double *__restrict__ pv, const double *__restrict__ qv,
                                                    double *U, double *r, E *t, E *tlo, double *sc, int it,
                                                    double *gpart, unsigned *gcount) {
    __shared__ double sh[8];
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_alpha = 0.0;
        if (it >= 0) {
            const double rz = sc[it & 1], pq = sc[2 + (it & 1)];
            s_alpha = pq > 0.0 ? rz / pq : 0.0;     // one float64 division per block
        }
    }
    __syncthreads();
    const double alpha = s_alpha;
    const int64_t n = (int64_t)nx * ny * nz;
    double rr = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ab = q / nz, c = q - ab * nz, a = ab / ny, b = ab - a * ny;
        const int64_t i = ((a + 1) * Ly + (b + 1)) * Lz + (c + 1);
        double ri = r[i];
        if (it >= 0) {
            U[i] += alpha * pv[i];
            ri -= alpha * qv[i];
            r[i] = ri;
            rr = fma(ri, ri, rr);
        }
        const E hi = (E)(float)ri;
        t[ab * ldc + c] = hi;
        if (tlo) tlo[ab * ldc + c] = (E)((float)ri - (float)hi);
    }
    if (it >= 0) {
        if (threadIdx.x == 0 && blockIdx.x == 0) sc[2 + ((it + 1) & 1)] = 0.0;
        const double tot[1] = {block_sum(rr, sh)};
        grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[4 + ((it + 1) & 1)] += v; });
    }
}

// z <- the interior tensor (float64; t + tlo when tlo is given), rz[slot] += r.z; with pv also
// p = z (CG start), and with pf p as float32 pairs too
template <class E>
__global__ void __launch_bounds__(256) k_sep_scatter(int nx, int ny, int nz, int ldc, int Ly, int Lz,
                                                     const E *__restrict__ t, const E *__restrict__ tlo,
                                                     const double *__restrict__ r, double *z, double *pv, float2 *pf,
                                                     double *sc, int slot, double *gpart, unsigned *gcount) {
    __shared__ double sh[8];
    const int64_t n = (int64_t)nx * ny * nz;
    double rz = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ab = q / nz, c = q - ab * nz, a = ab / ny, b = ab - a * ny;
        const int64_t i = ((a + 1) * Ly + (b + 1)) * Lz + (c + 1);
        const double zi = (double)(float)t[ab * ldc + c] + (tlo ? (double)(float)tlo[ab * ldc + c] : 0.0);
        z[i] = zi;
        if (pv) pv[i] = zi;
        if (pf) pf[i] = ff_split(zi);
        rz = fma(r[i], zi, rz);
    }
    const double tot[1] = {block_sum(rz, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[slot] += v; });
}

// Batched row-major GEMM C_z = A_z B_z (M x K times K x N), float32, 64 x 64 tiles, 256
// threads with 4 x 4 outputs each, K in steps of 16 through shared memory.  Batch strides may
// be zero (a shared operand).  With lam_r / lam_c the epilogue divides by lam_r[m] + lam_c[n].
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_sep_gemm(int M, int N, int K, const float *__restrict__ A, int64_t sA,
                                                  const float *__restrict__ B, int64_t sB, float *C, int64_t sC,
                                                  const float *__restrict__ lam_r, const float *__restrict__ lam_c) {
    __shared__ float As[GK][GT + 4];    // As[k][m]
    __shared__ float Bs[GK][GT + 4];    // Bs[k][n]
    const int z = blockIdx.z;
    A += z * sA; B += z * sB; C += z * sC;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;     // 16 x 16 threads
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        // 64 x 16 of A and 16 x 64 of B, four elements per thread each
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int mm = e / GK, kk = e % GK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * K + gk] : 0.f;
            const int kb = e / GT, nn = e % GT;
            const int gkb = k0 + kb, gn = n0 + nn;
            Bs[kb][nn] = (gkb < K && gn < N) ? B[(int64_t)gkb * N + gn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float v = acc[i][j];
            if (lam_r) v /= (lam_r[gm] + lam_c[gn]);
            C[(int64_t)gm * N + gn] = v;
        }
    }
}

void gemm(ofks_ctx *c, int batch, int M, int N, int K, const float *A, int64_t sA, const float *B, int64_t sB,
          float *C, int64_t sC, const float *lr = nullptr, const float *lc = nullptr) {
    dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT), (unsigned)batch);
    k_sep_gemm<<<grid, 256, 0, c->stream>>>(M, N, K, A, sA, B, sB, C, sC, lr, lc);
    c->kernels += 1;
}


// ---- tensor-core form (tcgen05, bf16 operands, float32 accumulation in tensor memory)
//
// Each of the six contractions is one GEMM  D[m][n] = sum_k A[m][k] Bt[n][k]  whose A is the
// current tensor with the contracted axis innermost (rows m = the other two axes) and whose Bt
// is an axis matrix or its transpose.  The output is written with n outermost, which rotates the
// axes so that the next contraction is again over the innermost one: [a][b][c] -> [k][a][b] ->
// [j][k][a] -> [i][j][k] (scaled) -> [c][i][j] -> [b][c][i] -> [a][b][c].  Intermediate tensors
// are bf16 with the innermost axis padded to a multiple of 16 (zero padding, written never), so
// every A row is a whole number of 16-byte core-matrix rows.  One CTA of four warps computes a
// 128-row tile: the operands go to shared memory in the no-swizzle K-major core-matrix layout,
// one thread issues the MMAs (M = 128, N = NP, K = 16 each) into tensor memory and commits them
// to an mbarrier, and each warp reads its 32 rows back with tcgen05.ld for the epilogue.
// Waits are bounded: on timeout the CTA flags an error, frees its tensor memory and returns.
constexpr int STM = 128;
constexpr long long SEP_WAIT = 1LL << 20;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// element (r, k) of a tile with KP columns: core matrix (r / 8, k / 8), 8 x 8 elements, cores
// adjacent along K 128 B apart and along rows KP / 8 * 128 B apart
__device__ __forceinline__ int coff(int r, int k, int KP) {
    return ((r >> 3) * (KP >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (rows past the end)
__device__ __forceinline__ void cp16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes) : "memory");
}

struct SepPass {
    const __nv_bfloat16 *A;        // M x KP row-major (zero padding beyond K)
    const __nv_bfloat16 *Alo;      // SPLIT: the low parts of A (A + Alo is the operand)
    const __nv_bfloat16 *Bt;       // NP x KP row-major, zero padded
    int M, K, KP, N, NP, tcols;    // tcols: tensor-memory columns (power of two >= NS)
    int NS;                        // output columns per CTA (NP / gridDim.y, a multiple of 16)
    __nv_bfloat16 *out;            // element (n, m) at (n M1 + m / M2) KPo + m % M2
    __nv_bfloat16 *outlo;          // SPLIT: the low parts of the output (same layout)
    int M1, M2, KPo;
    const float *lr, *lc;          // SCALE: multiply by f / (lr[n] + lc[m] + h_b)
    // batches of Mb rows (Mb = 0: one batch of M): row m is row m' = m mod Mb of batch
    // b = m / Mb, whose output starts at b * ob; in the scaling h_b = -2 shd[b] (shd null: 0)
    int Mb;
    int64_t ob;
    const double *shd;
    float f;
    int nst;                       // A stages in shared memory (1 or 2)
    int *err;
};

// SPLIT: the A operand and the output are pairs of bf16 parts (high + low), and the MMAs add
// both parts' products with Bt, so the passes carry ~16 significant bits instead of 8.
//
// Persistent: CTA (x, y) takes the 128-row tiles x, x + gridDim.x, ... of output columns
// [y NS, (y + 1) NS).  Bt's NS x KP slice is loaded once; the A tiles go through P.nst stages
// (two: the next tile's copies are issued before this tile's MMAs, so they overlap the MMAs and
// the epilogue; one: issued once this tile's MMAs are done, overlapping the epilogue).  One
// thread issues each tile's MMAs into the tensor-memory accumulator and commits them to the
// mbarrier (one phase per tile); the four warps read their 32 rows back after the wait.
template <int SCALE, int SPLIT>
__global__ void __launch_bounds__(128, 1) k_sep_tc(const SepPass P) {
    extern __shared__ __align__(128) unsigned char dsm[];
    constexpr int NA = SPLIT ? 2 : 1;                                // parts of A
    const int KP = P.KP, kc8 = KP >> 3;
    __nv_bfloat16 *sB = reinterpret_cast<__nv_bfloat16 *>(dsm);     // NS x KP
    __nv_bfloat16 *sA = sB + P.NS * KP;                              // nst stages of NA x STM x KP
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * P.NS;                                // this CTA's output columns
    const int ntiles = (P.M + STM - 1) / STM;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(P.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    // operands: rows of 8 elements (16 B) copied asynchronously into their core-matrix rows
    auto load_a = [&](int tile, int stage) {
        const int m0 = tile * STM;
        __nv_bfloat16 *dst = sA + (size_t)stage * NA * STM * KP;
        for (int e = tid; e < STM * kc8; e += blockDim.x) {
            const int rr = e / kc8, k = (e - rr * kc8) * 8;
            const bool in = m0 + rr < P.M;
            const int64_t off = in ? (int64_t)(m0 + rr) * KP + k : 0;
            cp16(dst + coff(rr, k, KP), P.A + off, in ? 16 : 0);
            if (SPLIT) cp16(dst + STM * KP + coff(rr, k, KP), P.Alo + off, in ? 16 : 0);
        }
    };
    for (int e = tid; e < P.NS * kc8; e += blockDim.x) {
        const int n = e / kc8, k = (e - n * kc8) * 8;
        cp16(sB + coff(n, k, KP), P.Bt + (int64_t)(n0 + n) * KP + k, 16);
    }
    int tile = blockIdx.x;
    if (tile < ntiles) load_a(tile, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(P.NS >> 3) << 17) |
                           ((uint32_t)(STM >> 4) << 24);
    const uint32_t sbo = (uint32_t)kc8 * 128u;
    int last = -1;                                                   // iteration of the last commit
    for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
        const int st = P.nst == 2 ? (i & 1) : 0;
        const int next = tile + gridDim.x;
        if (P.nst == 2) {
            if (next < ntiles) load_a(next, st ^ 1);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a0 = su32(sA + (size_t)st * NA * STM * KP), b0 = su32(sB);
            for (int part = 0; part < NA; ++part)
                for (int kk = 0; kk < KP / 16; ++kk) {
                    const uint64_t ad = sdesc(a0 + (uint32_t)(part * STM * KP * 2) + kk * 256, 128, sbo);
                    const uint64_t bd = sdesc(b0 + kk * 256, 128, sbo);
                    const uint32_t accum = (part > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(&mbar)));
        }
        last = i;
        uint32_t done = 0;
        for (long long w = 0; w < SEP_WAIT && !done; ++w) {
            asm volatile(
                "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(done)
                : "r"(su32(&mbar)), "r"((uint32_t)(i & 1)));
        }
        if (!done) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;                                       // uniform: read after the barrier
        if (P.nst == 1) {                                            // the stage is free again
            if (next < ntiles) load_a(next, 0);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int m = tile * STM + warp * 32 + lane;
        const int bt = P.Mb ? m / P.Mb : 0, mm = m - bt * P.Mb;
        const int m1 = mm / P.M2, m2 = mm - m1 * P.M2;
        const float lcm = (SCALE && m < P.M) ? P.lc[mm] + (P.shd ? (float)(-2.0 * P.shd[bt]) : 0.f) : 0.f;
        __nv_bfloat16 *outb = P.out + (int64_t)bt * P.ob;
        __nv_bfloat16 *outl = SPLIT ? P.outlo + (int64_t)bt * P.ob : nullptr;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < P.NS; cb += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr + cb));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (m >= P.M) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int n = n0 + cb + q;
                if (n >= P.N) break;
                float x = __uint_as_float(v[q]);
                if (SCALE) x = __fdividef(P.f * x, P.lr[n] + lcm);
                const int64_t o = ((int64_t)n * P.M1 + m1) * P.KPo + m2;
                const __nv_bfloat16 hi = __float2bfloat16(x);
                outb[o] = hi;
                if (SPLIT) outl[o] = __float2bfloat16(x - __bfloat162float(hi));
            }
        }
        // the accumulator is read: the next tile's MMAs (issued after the next barrier) may overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (abort_flag && tid == 0) {
        atomicExch(P.err, 1);
        // the MMAs of the last commit may still be running: wait for them once more (bounded)
        // before the tensor memory is released
        uint32_t done = 0;
        for (long long w = 0; w < SEP_WAIT && !done && last >= 0; ++w)
            asm volatile(
                "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(done)
                : "r"(su32(&mbar)), "r"((uint32_t)(last & 1)));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");                 // no copy left in flight
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tcols));
}

template <int SCALE, int SPLIT = 0>
void sep_tc_launch(ofks_ctx *c, SepPass P) {
    // the output columns split over gridDim.y (each a multiple of 16) until the tiles cover the
    // 152 SMs: the passes are latency-bound, and short axes give few 128-row tiles
    const int tiles = (P.M + STM - 1) / STM, nb = P.NP / 16;
    int d = 1;
    for (int cand = 1; cand <= nb; ++cand) {
        if (nb % cand) continue;
        d = cand;
        // enough tiles for the SMs, and at most 128 output columns per CTA: 128 tensor-memory
        // columns let several CTAs share an SM
        if ((int64_t)tiles * cand >= 152 && P.NP / cand <= 128) break;
    }
    P.NS = P.NP / d;
    P.tcols = P.NS <= 32 ? 32 : (P.NS <= 64 ? 64 : (P.NS <= 128 ? 128 : 256));
    P.err = c->d_flag + 1;
    const int NA = SPLIT ? 2 : 1, kmax = 227 * 1024;
    // shared memory of at least 228 KB * tcols / 512 per CTA keeps the CTAs resident on one SM
    // within its 512 tensor-memory columns, so no allocation ever has to wait
    const int floor_ = 228 * 1024 / (512 / P.tcols) + 1024;
    auto need = [&](int nst) { return (P.NS + nst * NA * STM) * P.KP * (int)sizeof(__nv_bfloat16); };
    auto smem_for = [&](int nst) { return std::min(kmax, std::max(need(nst), floor_)); };
    // persistent CTAs: one wave over the SMs, each walking its share of the tiles
    auto grid_for = [&](int smem) {
        const int per_sm = std::max(1, std::min(512 / P.tcols, 228 * 1024 / (smem + 1024)));
        return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (152LL * per_sm + d - 1) / d));
    };
    // a second A stage only where a CTA has more than one tile (it costs residency)
    P.nst = 1;
    int smem = smem_for(1), gx = grid_for(smem);
    if (tiles > gx && need(2) <= kmax) {
        P.nst = 2;
        smem = smem_for(2);
        gx = grid_for(smem);
    }
    cudaFuncSetAttribute(k_sep_tc<SCALE, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_sep_tc<SCALE, SPLIT><<<dim3((unsigned)gx, (unsigned)d), 128, smem, c->stream>>>(P);
    c->kernels += 1;
}

inline int pad16(int x) { return (x + 15) / 16 * 16; }
}  // namespace

void sep_free(ofks_ctx *c) {
    SepState &S = c->sep;
    for (float *p : {S.S[0], S.S[1], S.S[2], S.St[0], S.St[1], S.St[2], S.lx, S.lyz, S.t0, S.t1})
        if (p) cudaFree(p);
    for (void *p : {(void *)S.hS[0], (void *)S.hS[1], (void *)S.hS[2], (void *)S.hSt[0], (void *)S.hSt[1],
                    (void *)S.hSt[2], (void *)S.hbuf, (void *)S.hlo, (void *)S.pbuf})
        if (p) cudaFree(p);
    S = SepState{};
}

// Per-axis modes on the host; OFKS_OK with c->sep.on = false when the mesh is not a lattice
// whose faces are the Dirichlet boundary, or an axis is too long for the dense eigen-solver.
int sep_setup(ofks_ctx *c, const double *xyz, const uint8_t *dirichlet) {
    sep_free(c);
    if (!c->st.on) return OFKS_OK;
    const int L[3] = {c->st.Lx, c->st.Ly, c->st.Lz};
    for (int d = 0; d < 3; ++d)
        if (L[d] < 3 || L[d] > 770) return OFKS_OK;    // dense O(n^3) eigen-solver per axis
    const int64_t N = (int64_t)L[0] * L[1] * L[2];
    for (int64_t i = 0; i < N; ++i) {
        const int64_t a = i / ((int64_t)L[1] * L[2]), b = (i / L[2]) % L[1], cz = i % L[2];
        const bool face = a == 0 || a == L[0] - 1 || b == 0 || b == L[1] - 1 || cz == 0 || cz == L[2] - 1;
        if (face != (dirichlet[i] != 0)) return OFKS_OK;
    }
    std::vector<double> x[3];
    for (int a = 0; a < L[0]; ++a) x[0].push_back(xyz[3 * ((int64_t)a * L[1] * L[2])]);
    for (int b = 0; b < L[1]; ++b) x[1].push_back(xyz[3 * ((int64_t)b * L[2]) + 1]);
    for (int cz = 0; cz < L[2]; ++cz) x[2].push_back(xyz[3 * (int64_t)cz + 2]);
    std::vector<double> Sd[3], lam[3];
    for (int d = 0; d < 3; ++d)
        if (!axis_modes(x[d], Sd[d], lam[d])) return OFKS_OK;
    SepState &S = c->sep;
    const int n[3] = {L[0] - 2, L[1] - 2, L[2] - 2};
    const int64_t nt = (int64_t)n[0] * n[1] * n[2];
    std::vector<float> lyz((size_t)n[1] * n[2]), lx(n[0]);
    for (int i = 0; i < n[0]; ++i) lx[i] = (float)lam[0][i];
    for (int j = 0; j < n[1]; ++j)
        for (int k = 0; k < n[2]; ++k) lyz[(size_t)j * n[2] + k] = (float)(lam[1][j] + lam[2][k]);
    cudaError_t e = cudaSuccess;
    auto upf = [&](float **dst, const std::vector<float> &h) {
        if (e == cudaSuccess) e = cudaMalloc((void **)dst, sizeof(float) * std::max<size_t>(h.size(), 1));
        if (e == cudaSuccess) e = cudaMemcpy(*dst, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
    };
    for (int d = 0; d < 3; ++d) {
        std::vector<float> s((size_t)n[d] * n[d]), st((size_t)n[d] * n[d]);
        for (int a = 0; a < n[d]; ++a)
            for (int i = 0; i < n[d]; ++i) {
                s[(size_t)a * n[d] + i] = (float)Sd[d][(size_t)a * n[d] + i];
                st[(size_t)i * n[d] + a] = (float)Sd[d][(size_t)a * n[d] + i];
            }
        upf(&S.S[d], s);
        upf(&S.St[d], st);
    }
    upf(&S.lx, lx);
    upf(&S.lyz, lyz);
    // tensor-core operands: bf16 axis matrices padded to multiples of 16, and five zeroed
    // intermediate tensors whose innermost axis is padded the same way
    S.tc = n[0] <= 256 && n[1] <= 256 && n[2] <= 256;
    if (S.tc && e == cudaSuccess) {
        for (int d = 0; d < 3; ++d) {
            const int P16 = pad16(n[d]);
            std::vector<__nv_bfloat16> s((size_t)P16 * P16, __float2bfloat16(0.f)), st(s);
            for (int a = 0; a < n[d]; ++a)
                for (int i = 0; i < n[d]; ++i) {
                    s[(size_t)a * P16 + i] = __float2bfloat16((float)Sd[d][(size_t)a * n[d] + i]);
                    st[(size_t)i * P16 + a] = __float2bfloat16((float)Sd[d][(size_t)a * n[d] + i]);
                }
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
                __nv_bfloat16 **dst = w == 0 ? &S.hS[d] : &S.hSt[d];
                const std::vector<__nv_bfloat16> &h = w == 0 ? s : st;
                e = cudaMalloc((void **)dst, sizeof(__nv_bfloat16) * h.size());
                if (e == cudaSuccess) e = cudaMemcpy(*dst, h.data(), sizeof(__nv_bfloat16) * h.size(), cudaMemcpyHostToDevice);
            }
        }
        // [a][b][c~], [k][a][b~], [j][k][a~], [i][j][k~], [c][i][j~], [b][c][i~]  (~ = padded to 16)
        const int64_t len[6] = {(int64_t)n[0] * n[1] * pad16(n[2]), (int64_t)n[2] * n[0] * pad16(n[1]),
                                (int64_t)n[1] * n[2] * pad16(n[0]), (int64_t)n[0] * n[1] * pad16(n[2]),
                                (int64_t)n[2] * n[0] * pad16(n[1]), (int64_t)n[1] * n[2] * pad16(n[0])};
        int64_t tot = 0;
        for (int q = 0; q < 6; ++q) { S.hoff[q] = tot; tot += (len[q] + 63) / 64 * 64; }
        if (e == cudaSuccess) e = cudaMalloc((void **)&S.hbuf, sizeof(__nv_bfloat16) * tot);
        if (e == cudaSuccess) e = cudaMemset(S.hbuf, 0, sizeof(__nv_bfloat16) * tot);
        if (e == cudaSuccess) e = cudaMalloc((void **)&S.hlo, sizeof(__nv_bfloat16) * tot);
        if (e == cudaSuccess) e = cudaMemset(S.hlo, 0, sizeof(__nv_bfloat16) * tot);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.t0, sizeof(float) * nt);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.t1, sizeof(float) * nt);
    if (e != cudaSuccess) {
        sep_free(c);
        return ofks_fail(c, OFKS_ENOMEM, "set_mesh: separable preconditioner: %s", cudaGetErrorString(e));
    }
    S.n[0] = n[0]; S.n[1] = n[1]; S.n[2] = n[2];
    S.on = true;
    if (std::getenv("OFKS_VERBOSE"))
        std::fprintf(stderr, "[ofks sep] interior %d x %d x %d, lam_x in [%.3e, %.3e]\n", n[0], n[1], n[2],
                     lam[0].front(), lam[0].back());
    return OFKS_OK;
}

// One preconditioned step of the Hartree CG on the interior nodes (full-node vectors, Dirichlet
// entries untouched): with it >= 0 first the CG update of iteration it (see k_sep_gather), then
// z = A_sep^-1 r, rz[slot] += r.z, and with first != 0 also p = z.
void sep_cg_step(ofks_ctx *c, int it, int slot, int first) {
    SepState &S = c->sep;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int64_t nt = (int64_t)nx * ny * nz;
    const unsigned g = (unsigned)std::min<int64_t>((nt + 255) / 256, 152 * 8);
    double *sc = c->d_sc + SC_CG;
    if (S.tc && c->prm.poisson_sep_tc) {
        // every tensor as a high and a low bf16 part: the rounding of the intermediates to 8 bits
        // made the preconditioner visibly nonlinear and cost the CG about a quarter more iterations
        const int px = pad16(nx), py = pad16(ny), pz = pad16(nz);
        __nv_bfloat16 *B[6], *Bl[6];
        for (int q = 0; q < 6; ++q) { B[q] = S.hbuf + S.hoff[q]; Bl[q] = S.hlo + S.hoff[q]; }
        SepPass P{};
        P.f = 1.f;
        auto pass = [&](int q, const __nv_bfloat16 *Bt, int M, int K, int N, int qo, int M1, int M2, int KPo) {
            P.A = B[q]; P.Alo = Bl[q]; P.Bt = Bt; P.M = M; P.K = K; P.KP = pad16(K); P.N = N; P.NP = pad16(N);
            P.out = B[qo]; P.outlo = Bl[qo]; P.M1 = M1; P.M2 = M2; P.KPo = KPo;
        };
        k_sep_gather<__nv_bfloat16><<<g, 256, 0, c->stream>>>(nx, ny, nz, pz, c->st.Ly, c->st.Lz, c->d_cp, c->d_cq,
                                                              c->d_U, c->d_cr, B[0], Bl[0], sc, it, c->d_gpart,
                                                              c->d_gcount);
        pass(0, S.hSt[2], nx * ny, nz, nz, 1, nx, ny, py);                 // [a][b][c] -> [k][a][b]
        sep_tc_launch<0, 1>(c, P);
        pass(1, S.hSt[1], nz * nx, ny, ny, 2, nz, nx, px);                 // -> [j][k][a]
        sep_tc_launch<0, 1>(c, P);
        pass(2, S.hSt[0], ny * nz, nx, nx, 3, ny, nz, pz);                 // -> [i][j][k] / lam
        P.lr = S.lx; P.lc = S.lyz;
        sep_tc_launch<1, 1>(c, P);
        pass(3, S.hS[2], nx * ny, nz, nz, 4, nx, ny, py);                  // -> [c][i][j]
        sep_tc_launch<0, 1>(c, P);
        pass(4, S.hS[1], nz * nx, ny, ny, 5, nz, nx, px);                  // -> [b][c][i]
        sep_tc_launch<0, 1>(c, P);
        pass(5, S.hS[0], ny * nz, nx, nx, 0, ny, nz, pz);                  // -> [a][b][c]
        sep_tc_launch<0, 1>(c, P);
        k_sep_scatter<__nv_bfloat16><<<g, 256, 0, c->stream>>>(nx, ny, nz, pz, c->st.Ly, c->st.Lz, B[0], Bl[0],
                                                               c->d_cr, c->d_cz, first ? c->d_cp : nullptr,
                                                               first && c->hartree_ff ? c->d_cpff : nullptr, sc, slot,
                                                               c->d_gpart, c->d_gcount);
        c->kernels += 2;
        return;
    }
    k_sep_gather<float><<<g, 256, 0, c->stream>>>(nx, ny, nz, nz, c->st.Ly, c->st.Lz, c->d_cp, c->d_cq, c->d_U,
                                                  c->d_cr, S.t0, nullptr, sc, it, c->d_gpart, c->d_gcount);
    // forward: T1[ab][k] = sum_c R[ab][c] Sz[c][k]
    gemm(c, 1, nx * ny, nz, nz, S.t0, 0, S.S[2], 0, S.t1, 0);
    // T2[a][j][k] = sum_b Sy^T[j][b] T1[a][b][k]
    gemm(c, nx, ny, nz, ny, S.St[1], 0, S.t1, (int64_t)ny * nz, S.t0, (int64_t)ny * nz);
    // T3[i][jk] = sum_a Sx^T[i][a] T2[a][jk] / (lam_x,i + lam_y,j + lam_z,k)
    gemm(c, 1, nx, ny * nz, nx, S.St[0], 0, S.t0, 0, S.t1, 0, S.lx, S.lyz);
    // back: U1[a][jk] = sum_i Sx[a][i] T3[i][jk]
    gemm(c, 1, nx, ny * nz, nx, S.S[0], 0, S.t1, 0, S.t0, 0);
    // U2[a][b][k] = sum_j Sy[b][j] U1[a][j][k]
    gemm(c, nx, ny, nz, ny, S.S[1], 0, S.t0, (int64_t)ny * nz, S.t1, (int64_t)ny * nz);
    // Z[ab][c] = sum_k U2[ab][k] Sz^T[k][c]
    gemm(c, 1, nx * ny, nz, nz, S.t1, 0, S.St[2], 0, S.t0, 0);
    k_sep_scatter<float><<<g, 256, 0, c->stream>>>(nx, ny, nz, nz, c->st.Ly, c->st.Lz, S.t0, nullptr, c->d_cr, c->d_cz,
                                                   first ? c->d_cp : nullptr, first && c->hartree_ff ? c->d_cpff : nullptr,
                                                   sc, slot, c->d_gpart, c->d_gcount);
    c->kernels += 2;
}

// ---- the PCG of Eq. (precondition-T) preconditioned by the separable operator
//
// T_k = L/2 - shift_k B is approximated, like the Hartree stiffness above, by
//     T_sep,k = A_sep / 2 - shift_k B_sep,   B_sep = Mx (x) My (x) Mz,
// which the same modes diagonalize (S^T A_sep S = diag(lam), S^T B_sep S = I):
//     T_sep,k^-1 = S diag(2 / (lam_x,i + lam_y,j + lam_z,k - 2 shift_k)) S^T.
// The w columns of a PCG block go through the six contractions at once: column b's tensors are
// consecutive blocks, so each pass is one GEMM over w times the rows (batches of Mb rows, the
// output of batch b at b * ob), and the scaling adds -2 shift_b of its batch.  Six bf16 tensors
// per column, zero-initialized, padding never written (as for the Hartree solve).

// buffers for PCG blocks of width w (kept for smaller w); false when the form does not apply
bool sep_pcg_ready(ofks_ctx *c, int w) {
    SepState &S = c->sep;
    if (!S.on || !S.tc) return false;
    if (S.pbuf && S.pw >= w) return true;
    if (S.pbuf) cudaFree(S.pbuf);
    S.pbuf = nullptr;
    S.pw = 0;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int64_t len[6] = {(int64_t)nx * ny * pad16(nz), (int64_t)nz * nx * pad16(ny), (int64_t)ny * nz * pad16(nx),
                            (int64_t)nx * ny * pad16(nz), (int64_t)nz * nx * pad16(ny), (int64_t)ny * nz * pad16(nx)};
    // room for the widest block (ld columns) at once, so that a growing active set neither
    // reallocates (a device-wide synchronization) nor invalidates the captured PCG graphs; the
    // exact width when that does not fit
    for (const int wa : {std::max(w, c->ld), w}) {
        int64_t tot = 0;
        for (int q = 0; q < 6; ++q) { S.poff[q] = tot; tot += (len[q] * wa + 63) / 64 * 64; }
        if (cudaMalloc((void **)&S.pbuf, sizeof(__nv_bfloat16) * tot) == cudaSuccess) {
            if (cudaMemset(S.pbuf, 0, sizeof(__nv_bfloat16) * tot) == cudaSuccess) {
                S.pw = wa;
                return true;
            }
            cudaFree(S.pbuf);
        }
        cudaGetLastError();
        S.pbuf = nullptr;
    }
    // without room for the buffers the PCG keeps the Jacobi preconditioner (the failed call's
    // error is cleared so that no later check reports it)
    return false;
}

// z = T_sep^-1 r for the w columns in the input tensor (buffer 0, [b][a][b][c~]), result in the
// same buffer; shift: the PCG's per-column shifts (w doubles)
void sep_pcg_passes(ofks_ctx *c, int w, const double *shift) {
    SepState &S = c->sep;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int px = pad16(nx), py = pad16(ny), pz = pad16(nz);
    __nv_bfloat16 *B[6];
    for (int q = 0; q < 6; ++q) B[q] = S.pbuf + S.poff[q];
    SepPass P{};
    P.f = 1.f;
    auto pass = [&](const __nv_bfloat16 *A, const __nv_bfloat16 *Bt, int Mb, int K, int N, __nv_bfloat16 *out,
                    int M1, int M2, int KPo) {
        P.A = A; P.Bt = Bt; P.M = w * Mb; P.K = K; P.KP = pad16(K); P.N = N; P.NP = pad16(N);
        P.out = out; P.M1 = M1; P.M2 = M2; P.KPo = KPo;
        P.Mb = Mb; P.ob = (int64_t)N * M1 * KPo;
    };
    pass(B[0], S.hSt[2], nx * ny, nz, nz, B[1], nx, ny, py);           // [a][b][c] -> [k][a][b]
    sep_tc_launch<0>(c, P);
    pass(B[1], S.hSt[1], nz * nx, ny, ny, B[2], nz, nx, px);           // -> [j][k][a]
    sep_tc_launch<0>(c, P);
    pass(B[2], S.hSt[0], ny * nz, nx, nx, B[3], ny, nz, pz);           // -> [i][j][k] scaled
    P.lr = S.lx; P.lc = S.lyz; P.shd = shift; P.f = 2.f;
    sep_tc_launch<1>(c, P);
    P.shd = nullptr; P.f = 1.f;
    pass(B[3], S.hS[2], nx * ny, nz, nz, B[4], nx, ny, py);            // -> [c][i][j]
    sep_tc_launch<0>(c, P);
    pass(B[4], S.hS[1], nz * nx, ny, ny, B[5], nz, nx, px);            // -> [b][c][i]
    sep_tc_launch<0>(c, P);
    pass(B[5], S.hS[0], ny * nz, nx, nx, B[0], ny, nz, pz);            // -> [a][b][c]
    sep_tc_launch<0>(c, P);
}
