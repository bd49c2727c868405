// Quadrature-point fields: density (paper Sec. 2.2, rho = f tr(X^T calB X)), the Hartree
// potential by the FEM Poisson equation (Sec. 2.2) with multipole boundary data, the LDA
// potential (Slater exchange + Perdew-Zunger 1981 correlation), and the refresh of the
// Hamiltonian values H = L/2 + M_ext + M_Har + M_xc (Eq. hamiltonian).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr double PI = 3.14159265358979323846264338327950288;
constexpr double RHO_MIN = 1e-14;

// Spin-unpolarized LDA: returns eps_xc, writes V_xc.
// Exchange: eps_x = -(3/4)(3 rho/pi)^(1/3), V_x = (4/3) eps_x.
// Correlation (PZ81, r_s = (3/(4 pi rho))^(1/3)):
//   r_s >= 1: eps_c = g/(1 + b1 sqrt(r_s) + b2 r_s),
//             V_c = eps_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s)/(1 + b1 sqrt(r_s) + b2 r_s)
//   r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
//             V_c = A ln r_s + (B - A/3) + (2/3) C r_s ln r_s + (2 D - C)/3 r_s
__device__ __forceinline__ double lda(double rho, double &vxc) {
    if (!(rho >= RHO_MIN)) { vxc = 0.0; return 0.0; }
    const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
    const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
    double t = cbrt(3.0 * rho / PI);
    double ex = -0.75 * t, vx = -t;
    double rs = cbrt(3.0 / (4.0 * PI * rho));
    double ec, vc;
    if (rs >= 1.0) {
        double sq = sqrt(rs), den = 1.0 + b1 * sq + b2 * rs;
        ec = g / den;
        vc = ec * (1.0 + (7.0 / 6.0) * b1 * sq + (4.0 / 3.0) * b2 * rs) / den;
    } else {
        double lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        vc = A * lr + (B - A / 3.0) + (2.0 / 3.0) * C * rs * lr + (2.0 * D - C) / 3.0 * rs;
    }
    vxc = vx + vc;
    return ex + ec;
}

// One group of G lanes per tetrahedron; lane j of the group covers columns j, j+G, ...
// psi_{q,l} = sum_a N_a(x_q) X_{a,l}; rho_q = f sum_l psi_{q,l}^2.  The group leader writes
// rho_q, scatters the Poisson load 4 pi sum_q w rho_q N_i(x_q) to the 10 nodes and adds the
// tetrahedron's multipole moments to the block sums.
template <int G>
__global__ void __launch_bounds__(256) k_density(int64_t T, int p, int ld, double occ,
                                                 const double *__restrict__ X,
                                                 const int *__restrict__ tetf,
                                                 const int *__restrict__ tetn,
                                                 const double *__restrict__ wq,
                                                 const double *__restrict__ yq, double *rho,
                                                 double *rhs, double *mom, int do_hartree) {
    __shared__ double smom[10];
    if (threadIdx.x < 10) smom[threadIdx.x] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x % G;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double s[4] = {0, 0, 0, 0};
    if (t < T) {
        int f[10];
#pragma unroll
        for (int a = 0; a < 10; ++a) f[a] = tetf[t * 10 + a];
        for (int l = lane; l < p; l += G) {
            double x[10];
#pragma unroll
            for (int a = 0; a < 10; ++a) x[a] = f[a] >= 0 ? X[(int64_t)f[a] * ld + l] : 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double psi = 0.0;
#pragma unroll
                for (int a = 0; a < 10; ++a) psi += p2N(q, a) * x[a];
                s[q] += psi * psi;
            }
        }
    }
    // every lane of the warp takes part in the group reduction
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o, G);
    if (t < T) {
        if (lane == 0) {
            const double w = wq[t];
            double r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { r[q] = occ * s[q]; rho[t * 4 + q] = r[q]; }
            if (do_hartree) {
#pragma unroll
                for (int a = 0; a < 10; ++a) {
                    double v = 0.0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) v += p2N(q, a) * r[q];
                    atomicAdd(rhs + tetn[t * 10 + a], 4.0 * PI * w * v);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double *y = yq + (t * 4 + q) * 3;
                    double wr = w * r[q], y2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
                    m[0] += wr;
                    m[1] += wr * y[0]; m[2] += wr * y[1]; m[3] += wr * y[2];
                    m[4] += wr * (3.0 * y[0] * y[0] - y2);
                    m[5] += wr * (3.0 * y[1] * y[1] - y2);
                    m[6] += wr * (3.0 * y[2] * y[2] - y2);
                    m[7] += wr * 3.0 * y[0] * y[1];
                    m[8] += wr * 3.0 * y[0] * y[2];
                    m[9] += wr * 3.0 * y[1] * y[2];
                }
            }
        }
    }
    if (do_hartree) {
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            double v = warp_sum(m[i]);
            if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(smom + i, v);
        }
        __syncthreads();
        if (threadIdx.x < 10) atomicAdd(mom + threadIdx.x, smom[threadIdx.x]);
    }
}

// Multipole boundary values V_B(r) = Q/|r| + d.r/|r|^3 + (1/2) sum Q_ij r_i r_j/|r|^5
__global__ void k_boundary(int nb, const int *__restrict__ bnd, const double *__restrict__ bxyz,
                           const double *__restrict__ mom, int lmax, double *U) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    double x = bxyz[3 * k], y = bxyz[3 * k + 1], z = bxyz[3 * k + 2];
    double r2 = x * x + y * y + z * z, r = sqrt(r2);
    double v = 0.0;
    if (lmax >= 0) v = mom[0] / r;
    if (lmax >= 1) v += (mom[1] * x + mom[2] * y + mom[3] * z) / (r2 * r);
    if (lmax >= 2) {
        double qq = mom[4] * x * x + mom[5] * y * y + mom[6] * z * z +
                    2.0 * (mom[7] * x * y + mom[8] * x * z + mom[9] * y * z);
        v += 0.5 * qq / (r2 * r2 * r);
    }
    U[bnd[k]] = v;
}

// Poisson CG on the interior nodes with the full-node CSR stiffness; boundary entries of
// r, z, p stay zero (minv = 0 there), so L p restricted to the interior is L_II p_I.
__global__ void __launch_bounds__(256) k_cg_init(int64_t N, const int *__restrict__ ptr,
                                                 const int *__restrict__ col,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ minv,
                                                 const double *__restrict__ rhs,
                                                 const double *__restrict__ U, double *r, double *z,
                                                 double *pv, double *sc) {
    __shared__ double sh[8];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rz = 0.0, rr = 0.0, bb = 0.0;
    if (i < N) {
        double mi = minv[i], ri = 0.0, zi = 0.0;
        if (mi != 0.0) {
            double s = 0.0;
            for (int k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * U[col[k]];
            ri = rhs[i] - s;
            zi = mi * ri;
            bb = rhs[i] * rhs[i];
        }
        r[i] = ri; z[i] = zi; pv[i] = zi;
        rz = ri * zi; rr = ri * ri;
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        atomicAdd(sc + 0, rz);     // rz[0]
        atomicAdd(sc + 4, rr);     // rr[0]
        atomicAdd(sc + 6, bb);     // rhs2
    }
}

// q = L p, pq += p.q  (slot it&1); zero the retired rz slot
__global__ void __launch_bounds__(256) k_cg_spmv(int64_t N, const int *__restrict__ ptr,
                                                 const int *__restrict__ col,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ minv,
                                                 const double *__restrict__ pv, double *qv,
                                                 double *sc, int it) {
    __shared__ double sh[8];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double pq = 0.0;
    if (i < N && minv[i] != 0.0) {
        double s = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * pv[col[k]];
        qv[i] = s;
        pq = pv[i] * s;
    }
    pq = block_sum(pq, sh);
    if (threadIdx.x == 0) {
        atomicAdd(sc + 2 + (it & 1), pq);
        if (blockIdx.x == 0) {
            sc[0 + ((it + 1) & 1)] = 0.0;    // rz slot of the next "new" value
            sc[4 + ((it + 1) & 1)] = 0.0;    // rr slot
        }
    }
}

// alpha = rz/pq; U += alpha p; r -= alpha q; z = minv r; rz', rr' into the other slots
__global__ void __launch_bounds__(256) k_cg_update(int64_t N, const double *__restrict__ minv,
                                                   const double *__restrict__ pv,
                                                   const double *__restrict__ qv, double *U,
                                                   double *r, double *z, double *sc, int it) {
    __shared__ double sh[8];
    const int o = it & 1, nn = (it + 1) & 1;
    const double rz = sc[0 + o], pq = sc[2 + o];
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rz2 = 0.0, rr = 0.0;
    if (i < N) {
        double mi = minv[i];
        if (mi != 0.0) {
            U[i] += alpha * pv[i];
            double ri = r[i] - alpha * qv[i];
            double zi = mi * ri;
            r[i] = ri; z[i] = zi;
            rz2 = ri * zi; rr = ri * ri;
        }
    }
    rz2 = block_sum(rz2, sh);
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        atomicAdd(sc + 0 + nn, rz2);
        atomicAdd(sc + 4 + nn, rr);
        if (blockIdx.x == 0) sc[2 + nn] = 0.0;   // next pq slot
    }
}

// beta = rz'/rz; p = z + beta p
__global__ void k_cg_dir(int64_t N, const double *__restrict__ z, double *pv, const double *sc, int it) {
    const int o = it & 1, nn = (it + 1) & 1;
    const double rz = sc[0 + o], rz2 = sc[0 + nn];
    const double beta = rz > 0.0 ? rz2 / rz : 0.0;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) pv[i] = z[i] + beta * pv[i];
}

__global__ void k_half_copy(int64_t n, const double *__restrict__ a, double *b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = 0.5 * a[i];
}

// Per tetrahedron: V_H(x_q) from the nodal U, LDA at rho_q, V_q = V_ext + V_H + V_xc,
// the double-counting sum w (V_H/2 + V_xc - eps_xc) rho, and the local potential matrix
// sum_q w V_q N_a N_b added to the Hamiltonian values (which hold L/2 on entry).
__global__ void __launch_bounds__(128) k_potential(int64_t T, const int *__restrict__ tetn,
                                                   const int *__restrict__ emap,
                                                   const double *__restrict__ wq,
                                                   const double *__restrict__ vext,
                                                   const double *__restrict__ rho,
                                                   const double *__restrict__ U, int do_h, int do_xc,
                                                   double *vh, double *vxc, double *exc,
                                                   double *valH, double *edc) {
    __shared__ double sh[4];
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (t < T) {
        const double w = wq[t];
        double V[4];
        for (int q = 0; q < 4; ++q) {
            double h = 0.0;
            if (do_h)
                for (int a = 0; a < 10; ++a) h += p2N(q, a) * U[tetn[t * 10 + a]];
            double r = rho[t * 4 + q], vx = 0.0, ex = 0.0;
            if (do_xc) ex = lda(r, vx);
            vh[t * 4 + q] = h; vxc[t * 4 + q] = vx; exc[t * 4 + q] = ex;
            V[q] = w * (vext[t * 4 + q] + h + vx);
            e += w * (0.5 * h + vx - ex) * r;
        }
        const int *em = emap + t * 100;
        for (int a = 0; a < 10; ++a)
            for (int b = 0; b < 10; ++b) {
                int pos = em[a * 10 + b];
                if (pos < 0) continue;
                double m = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) m += V[q] * p2N(q, a) * p2N(q, b);
                atomicAdd(valH + pos, m);
            }
    }
    e = block_sum(e, sh);
    if (threadIdx.x == 0) atomicAdd(edc, e);
}

}  // namespace

int launch_density(ofks_ctx *c, const double *X) {
    ProfScope ps(c, PF_DENSITY);
    const int64_t T = c->n_tets;
    const int do_h = c->prm.hartree ? 1 : 0;
    if (do_h) {
        cudaMemsetAsync(c->d_rhs, 0, sizeof(double) * c->n_nodes, c->stream);
        cudaMemsetAsync(c->d_sc + SC_MOM, 0, sizeof(double) * 10, c->stream);
    }
    int G = 1;
    while (G < 32 && G < (c->p + 1) / 2) G <<= 1;
    const int B = 256;
    unsigned grid = (unsigned)((T * G + B - 1) / B);
#define DENS(g) k_density<g><<<grid, B, 0, c->stream>>>(T, c->p, c->ld, c->prm.occ, X, c->d_tetf, \
        c->d_tetn, c->d_wq, c->d_yq, c->d_rho, c->d_rhs, c->d_sc + SC_MOM, do_h)
    switch (G) {
        case 1: DENS(1); break;
        case 2: DENS(2); break;
        case 4: DENS(4); break;
        case 8: DENS(8); break;
        case 16: DENS(16); break;
        default: DENS(32); break;
    }
#undef DENS
    c->kernels += 1;
    return ofks_cuda_check(c, cudaGetLastError(), "density kernel");
}

int run_hartree(ofks_ctx *c) {
    if (!c->prm.hartree) return OFKS_OK;
    ProfScope ps(c, PF_POISSON);
    const int64_t N = c->n_nodes;
    const unsigned gN = (unsigned)((N + 255) / 256);
    double *sc = c->d_sc + SC_CG;
    k_boundary<<<(c->n_bnd + 255) / 256, 256, 0, c->stream>>>(c->n_bnd, c->d_bnd, c->d_bxyz,
                                                               c->d_sc + SC_MOM, c->prm.multipole_lmax,
                                                               c->d_U);
    cudaMemsetAsync(sc, 0, sizeof(double) * 8, c->stream);
    k_cg_init<<<gN, 256, 0, c->stream>>>(N, c->d_fptr, c->d_fcol, c->d_fval, c->d_minv, c->d_rhs, c->d_U,
                                         c->d_cr, c->d_cz, c->d_cp, sc);
    c->kernels += 2;
    const double tol2 = c->prm.poisson_tol * c->prm.poisson_tol;
    const int chunk = 16;
    int it = 0;
    double h[8];
    for (;;) {
        cudaError_t e = cudaMemcpyAsync(h, sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ofks_cuda_check(c, e, "Hartree CG");
        const double rr = h[4 + (it & 1)], bb = h[6];
        if (!std::isfinite(rr)) return ofks_fail(c, OFKS_ENONFINITE, "Hartree CG residual is not finite");
        if (rr <= tol2 * bb || bb == 0.0) break;
        if (it >= c->prm.poisson_max_iter)
            return ofks_fail(c, OFKS_ETIMEOUT, "Hartree CG: %d iterations, relative residual %.3e",
                             it, std::sqrt(rr / bb));
        for (int j = 0; j < chunk; ++j, ++it) {
            k_cg_spmv<<<gN, 256, 0, c->stream>>>(N, c->d_fptr, c->d_fcol, c->d_fval, c->d_minv, c->d_cp,
                                                 c->d_cq, sc, it);
            k_cg_update<<<gN, 256, 0, c->stream>>>(N, c->d_minv, c->d_cp, c->d_cq, c->d_U, c->d_cr,
                                                   c->d_cz, sc, it);
            k_cg_dir<<<gN, 256, 0, c->stream>>>(N, c->d_cz, c->d_cp, sc, it);
            c->kernels += 3;
        }
    }
    return ofks_cuda_check(c, cudaGetLastError(), "Hartree CG");
}

int launch_potential_refresh(ofks_ctx *c) {
    ProfScope ps(c, PF_POTENTIAL);
    const int64_t T = c->n_tets;
    k_half_copy<<<(unsigned)((c->sell_len + 255) / 256), 256, 0, c->stream>>>(c->sell_len, c->d_valL,
                                                                                 c->d_valH);
    cudaMemsetAsync(c->d_sc + SC_EDC, 0, sizeof(double), c->stream);
    k_potential<<<(unsigned)((T + 127) / 128), 128, 0, c->stream>>>(
        T, c->d_tetn, c->d_emap, c->d_wq, c->d_vext, c->d_rho, c->d_U, c->prm.hartree ? 1 : 0,
        c->prm.xc ? 1 : 0, c->d_vh, c->d_vxc, c->d_exc, c->d_valH, c->d_sc + SC_EDC);
    c->kernels += 2;
    return ofks_cuda_check(c, cudaGetLastError(), "potential kernel");
}
