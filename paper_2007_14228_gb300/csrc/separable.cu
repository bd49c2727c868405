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

// interior lattice tensor (a, b, c) <- full-node vector, float32
__global__ void k_sep_gather(int nx, int ny, int nz, int Ly, int Lz, const double *__restrict__ full, float *t) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = q / ((int64_t)ny * nz), b = (q / nz) % ny, c = q % nz;
        t[q] = (float)full[((a + 1) * Ly + (b + 1)) * Lz + (c + 1)];
    }
}

__global__ void k_sep_scatter(int nx, int ny, int nz, int Ly, int Lz, const float *__restrict__ t, double *full) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = q / ((int64_t)ny * nz), b = (q / nz) % ny, c = q % nz;
        full[((a + 1) * Ly + (b + 1)) * Lz + (c + 1)] = (double)t[q];
    }
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

}  // namespace

void sep_free(ofks_ctx *c) {
    SepState &S = c->sep;
    for (float *p : {S.S[0], S.S[1], S.S[2], S.St[0], S.St[1], S.St[2], S.lx, S.lyz, S.t0, S.t1})
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

// z = A_sep^-1 r on the interior nodes (full-node vectors; Dirichlet entries of z untouched)
void sep_apply(ofks_ctx *c, const double *r_full, double *z_full) {
    SepState &S = c->sep;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int64_t nt = (int64_t)nx * ny * nz;
    const unsigned g = (unsigned)std::min<int64_t>((nt + 255) / 256, 152 * 8);
    k_sep_gather<<<g, 256, 0, c->stream>>>(nx, ny, nz, c->st.Ly, c->st.Lz, r_full, S.t0);
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
    k_sep_scatter<<<g, 256, 0, c->stream>>>(nx, ny, nz, c->st.Ly, c->st.Lz, S.t0, z_full);
    c->kernels += 2;
}
