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
// With t = (3 rho/pi)^(1/3), t^3 r_s^3 = 9/(4 pi^2), so r_s = K_RS / t and one cube root
// serves both terms.  F is the arithmetic type: float64, or float32 for the float32 iterations
// (the FP64 pipe is the limit of this kernel on GB300; the potential enters float32 H values).
constexpr double K_RS = 0.610887057710857191300739313402;   // (9/(4 pi^2))^(1/3)

template <class F>
__device__ __forceinline__ F lda(F rho, F &vxc) {
    if (!(rho >= F(RHO_MIN))) { vxc = F(0); return F(0); }
    const F g = F(-0.1423), b1 = F(1.0529), b2 = F(0.3334);
    const F A = F(0.0311), B = F(-0.048), C = F(0.0020), D = F(-0.0116);
    F t;
    if constexpr (sizeof(F) == 4) t = cbrtf(F(3.0 / PI) * rho);
    else t = cbrt(F(3.0 / PI) * rho);
    const F ex = F(-0.75) * t, vx = -t;
    const F rs = F(K_RS) / t;
    F ec, vc;
    if (rs >= F(1)) {
        F sq;
        if constexpr (sizeof(F) == 4) sq = sqrtf(rs);
        else sq = sqrt(rs);
        const F den = F(1) + b1 * sq + b2 * rs;
        ec = g / den;
        vc = ec * (F(1) + F(7.0 / 6.0) * b1 * sq + F(4.0 / 3.0) * b2 * rs) / den;
    } else {
        F lr;
        if constexpr (sizeof(F) == 4) lr = logf(rs);
        else lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        vc = A * lr + (B - A / F(3)) + F(2.0 / 3.0) * C * rs * lr + (F(2) * D - C) / F(3) * rs;
    }
    vxc = vx + vc;
    return ex + ec;
}

// Density at the quadrature points (a1).  A group of G lanes works on one tetrahedron; lane
// j of the group covers columns j, j+G, ...:  psi_{q,l} = sum_a N_a(x_q) X_{a,l},
// rho_q = f sum_l psi_{q,l}^2 (group xor-reduction).  The per-tetrahedron epilogue is spread
// over the group's lanes (float64 warp instructions cost the same with one active lane):
// lane k writes rho_k (k < 4).  The Poisson load is gathered per node from rho (k_rhs_gather) and
// the multipole moments follow from it (k_moments).
template <class E, int G>
__global__ void __launch_bounds__(256) k_density(int64_t T, int p, int ld, double occ,
                                                 const E *__restrict__ X,
                                                 const int *__restrict__ tetf, double *rho) {
    constexpr int TPW = 32 / G;                       // tetrahedra per warp and pass
    const int lane = threadIdx.x & (G - 1), grp = (threadIdx.x & 31) / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * TPW; t0 < T; t0 += nwarp * TPW) {
        const int64_t t = t0 + grp;
        const bool ok = t < T;
        E se[4] = {E(0), E(0), E(0), E(0)};
        if (ok) {
            int f[10];
#pragma unroll
            for (int a = 0; a < 10; ++a) f[a] = tetf[t * 10 + a];
            for (int l = lane; l < p; l += G) {
                E x[10];
#pragma unroll
                for (int a = 0; a < 10; ++a) x[a] = f[a] >= 0 ? X[(int64_t)f[a] * ld + l] : E(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    E psi = E(0);
#pragma unroll
                    for (int a = 0; a < 10; ++a) psi = fma((E)p2N(q, a), x[a], psi);
                    se[q] = fma(psi, psi, se[q]);
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) se[q] += __shfl_xor_sync(0xffffffffu, se[q], o, G);
        double s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = (double)se[q];
        if (!ok) continue;
        for (int k = lane; k < 4; k += G) rho[t * 4 + k] = occ * s[k];
    }
}

// Density for blocks whose leading dimension is a multiple of 4 (p > 2): a group of G lanes per
// tetrahedron, lane j taking the 4-column chunks j, j + G, ... of the 10 rows with one 16-byte
// (float32) or two (float64) loads per row and chunk.  At the symmetric 4-point rule a P2 basis
// value is one of four numbers (vertex at q, other vertex, edge touching q, edge away from q), so
//   psi_q = (N_A - N_B) x_q + (N_C - N_D) e_q + N_B S_v + N_D S_e
// with S_v, S_e the sums of the vertex and edge values and e_q the sum of the three edges at
// vertex q: 30 operations per column instead of the 44 of the ten-term sums.
template <class E, int G>
__global__ void __launch_bounds__(256, sizeof(E) == 4 ? 4 : 2) k_density4(int64_t T, int ld, double occ,
                                                                          const E *__restrict__ X,
                                                                          const int *__restrict__ tetf, double *rho) {
    constexpr int TPW = 32 / G;
    const E nA = (E)p2N(0, 0), nB = (E)p2N(1, 0), nC = (E)p2N(0, 4), nD = (E)p2N(0, 9);
    const E dA = nA - nB, dC = nC - nD;
    const int lane = threadIdx.x & (G - 1), grp = (threadIdx.x & 31) / G;
    const int nch = ld >> 2;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * TPW; t0 < T; t0 += nwarp * TPW) {
        const int64_t t = t0 + grp;
        const bool ok = t < T;
        E se[4] = {E(0), E(0), E(0), E(0)};
        if (ok) {
            int f[10];
#pragma unroll
            for (int a = 0; a < 10; ++a) f[a] = tetf[t * 10 + a];
            for (int ch = lane; ch < nch; ch += G) {
                E x[10][4];
#pragma unroll
                for (int a = 0; a < 10; ++a) {
                    const int64_t base_a = (int64_t)f[a] * ld;
                    if (f[a] >= 0) {
                        if constexpr (sizeof(E) == 4) {
                            const float4 v = __ldg(reinterpret_cast<const float4 *>(X + base_a) + ch);
                            x[a][0] = v.x; x[a][1] = v.y; x[a][2] = v.z; x[a][3] = v.w;
                        } else {
                            const double2 v0 = __ldg(reinterpret_cast<const double2 *>(X + base_a) + 2 * ch);
                            const double2 v1 = __ldg(reinterpret_cast<const double2 *>(X + base_a) + 2 * ch + 1);
                            x[a][0] = v0.x; x[a][1] = v0.y; x[a][2] = v1.x; x[a][3] = v1.y;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) x[a][k] = E(0);
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // vertices 0..3, edges 01 02 03 12 13 23 at local ids 4..9
                    const E sv = (x[0][k] + x[1][k]) + (x[2][k] + x[3][k]);
                    const E se6 = (x[4][k] + x[5][k]) + (x[6][k] + x[7][k]) + (x[8][k] + x[9][k]);
                    const E base_q = fma(nB, sv, nD * se6);
                    const E eq[4] = {x[4][k] + x[5][k] + x[6][k], x[4][k] + x[7][k] + x[8][k],
                                     x[5][k] + x[7][k] + x[9][k], x[6][k] + x[8][k] + x[9][k]};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const E psi = fma(dC, eq[q], fma(dA, x[q][k], base_q));
                        se[q] = fma(psi, psi, se[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) se[q] += __shfl_xor_sync(0xffffffffu, se[q], o, G);
        if (!ok) continue;
        for (int k = lane; k < 4; k += G) rho[t * 4 + k] = occ * (double)se[k];
    }
}

// Poisson load rhs_i = 4 pi sum_T w_T sum_q N_a(x_q) rho_q over the element entries (T, a) of
// node i, gathered in list order (a fixed order: the same value on every run)
__global__ void __launch_bounds__(256) k_rhs_gather(int64_t N, const int *__restrict__ ptr, const int *__restrict__ list,
                                                    const double *__restrict__ wq, const double *__restrict__ rho,
                                                    double *rhs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int code = list[k], t = code / 10, a = code - 10 * t;
        const double *r = rho + (int64_t)t * 4;
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) v = fma(p2N(q, a), r[q], v);
        acc = fma(wq[t], v, acc);
    }
    rhs[i] = (4.0 * PI) * acc;
}

// Multipole moments of the density about the centre (Sec. 2.2 boundary data): for each of
// f = 1, y_0, y_1, y_2, 3 y_0^2 - |y|^2, 3 y_1^2 - |y|^2, 3 y_2^2 - |y|^2, 3 y_0 y_1, 3 y_0 y_2,
// 3 y_1 y_2, mom_k = sum_T w_T sum_q rho_q f_k(y_q).  Every f_k is quadratic and the P2 basis on
// a straight-sided tetrahedron interpolates quadratics exactly (sum_i f_k(y_i) N_i(x) = f_k(x),
// y_i the node positions), so mom_k = sum_i f_k(y_i) rhs_i / (4 pi) with the assembled Poisson
// load rhs_i = 4 pi sum_T w_T sum_q N_i(x_q) rho_q: one pass over the nodes instead of ten
// functions at every quadrature point.
__global__ void __launch_bounds__(256) k_moments(int64_t N, const double *__restrict__ ynode,
                                                 const double *__restrict__ rhs, double *mom, double *gpart,
                                                 unsigned *gcount) {
    __shared__ double sh[8];
    double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = rhs[i] * (1.0 / (4.0 * PI));
        const double y0 = ynode[3 * i], y1 = ynode[3 * i + 1], y2 = ynode[3 * i + 2];
        const double y2s = y0 * y0 + y1 * y1 + y2 * y2;
        m[0] += r;
        m[1] = fma(r, y0, m[1]);
        m[2] = fma(r, y1, m[2]);
        m[3] = fma(r, y2, m[3]);
        m[4] = fma(r, 3.0 * y0 * y0 - y2s, m[4]);
        m[5] = fma(r, 3.0 * y1 * y1 - y2s, m[5]);
        m[6] = fma(r, 3.0 * y2 * y2 - y2s, m[6]);
        m[7] = fma(r, 3.0 * y0 * y1, m[7]);
        m[8] = fma(r, 3.0 * y0 * y2, m[8]);
        m[9] = fma(r, 3.0 * y1 * y2, m[9]);
    }
    double tot[10];
#pragma unroll 1
    for (int k = 0; k < 10; ++k) tot[k] = block_sum(m[k], sh);
    grid_accumulate<10>(tot, gpart, gcount, [&](int k, double v) { mom[k] = v; });
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

// CG start after a residual r = rhs - L U from the lattice-stencil kernel (which leaves the
// Dirichlet rows unwritten): r = 0 there, z = p = minv r, and rz, rr, |rhs|^2 as k_cg_init
__global__ void __launch_bounds__(256) k_cg_init_vec(int64_t N, const double *__restrict__ minv,
                                                     const double *__restrict__ rhs, double *r, double *z,
                                                     double *pv, double *sc, double *gpart, unsigned *gcount) {
    __shared__ double sh[8];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rz = 0.0, rr = 0.0, bb = 0.0;
    if (i < N) {
        const double mi = minv[i];
        const double ri = mi != 0.0 ? r[i] : 0.0, zi = mi * ri;
        if (mi != 0.0) bb = rhs[i] * rhs[i];
        r[i] = ri; z[i] = zi; pv[i] = zi;
        rz = ri * zi; rr = ri * ri;
    }
    const double tot[3] = {block_sum(rz, sh), block_sum(rr, sh), block_sum(bb, sh)};
    grid_accumulate<3>(tot, gpart, gcount, [&](int k, double v) { sc[k == 0 ? 0 : (k == 1 ? 4 : 6)] += v; });
}

// Poisson CG on the interior nodes with the full-node CSR stiffness; boundary entries of
// r, z, p stay zero (minv = 0 there), so L p restricted to the interior is L_II p_I.
__global__ void __launch_bounds__(256) k_cg_init(int64_t N, const int *__restrict__ ptr,
                                                 const int *__restrict__ col,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ minv,
                                                 const double *__restrict__ rhs,
                                                 const double *__restrict__ U, double *r, double *z,
                                                 double *pv, double *sc, double *gpart, unsigned *gcount) {
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
    // rz[0], rr[0], |rhs|^2
    const double tot[3] = {block_sum(rz, sh), block_sum(rr, sh), block_sum(bb, sh)};
    grid_accumulate<3>(tot, gpart, gcount, [&](int k, double v) { sc[k == 0 ? 0 : (k == 1 ? 4 : 6)] += v; });
}

// q = L p, pq += p.q  (slot it&1); zero the retired rz slot.  One thread per row: on GB300 a
// float64 warp instruction costs the same with any number of active lanes, so lane-split rows
// (which add shuffle-reductions in float64) measured slower than this form.
__global__ void __launch_bounds__(256) k_cg_spmv(int64_t N, const int *__restrict__ ptr,
                                                 const int *__restrict__ col,
                                                 const double *__restrict__ val,
                                                 const double *__restrict__ minv,
                                                 const double *__restrict__ pv, double *qv,
                                                 double *sc, int it, double *gpart, unsigned *gcount) {
    __shared__ double sh[8];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double pq = 0.0;
    if (i < N && minv[i] != 0.0) {
        double s = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) s = fma(val[k], pv[col[k]], s);
        qv[i] = s;
        pq = pv[i] * s;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc[0 + ((it + 1) & 1)] = 0.0;        // rz slot of the next "new" value
        sc[4 + ((it + 1) & 1)] = 0.0;        // rr slot
    }
    const double tot[1] = {block_sum(pq, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[2 + (it & 1)] += v; });
}

// alpha = rz/pq; U += alpha p; r -= alpha q; z = minv r; rz', rr' into the other slots
__global__ void __launch_bounds__(256) k_cg_update(int64_t N, const double *__restrict__ minv,
                                                   const double *__restrict__ pv,
                                                   const double *__restrict__ qv, double *U,
                                                   double *r, double *z, double *sc, int it, double *gpart,
                                                   unsigned *gcount) {
    __shared__ double sh[8];
    __shared__ double s_alpha;
    const int nn = (it + 1) & 1;
    // one float64 division per block (a division per thread costs as much as the whole update)
    if (threadIdx.x == 0) {
        const double rz = sc[it & 1], pq = sc[2 + (it & 1)];
        s_alpha = pq > 0.0 ? rz / pq : 0.0;
    }
    __syncthreads();
    const double alpha = s_alpha;
    double rz2 = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double mi = minv[i];
        if (mi != 0.0) {
            U[i] += alpha * pv[i];
            double ri = r[i] - alpha * qv[i];
            double zi = mi * ri;
            r[i] = ri; z[i] = zi;
            rz2 = fma(ri, zi, rz2); rr = fma(ri, ri, rr);
        }
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) sc[2 + nn] = 0.0;   // next pq slot
    const double tot[2] = {block_sum(rz2, sh), block_sum(rr, sh)};
    grid_accumulate<2>(tot, gpart, gcount, [&](int k, double v) { sc[(k == 0 ? 0 : 4) + nn] += v; });
}

// preconditioned variant of k_cg_update: alpha = rz/pq; U += alpha p; r -= alpha q; rr'
__global__ void __launch_bounds__(256) k_cg_update_r(int64_t N, const double *__restrict__ minv,
                                                     const double *__restrict__ pv,
                                                     const double *__restrict__ qv, double *U, double *r,
                                                     double *sc, int it, double *gpart, unsigned *gcount) {
    __shared__ double sh[8];
    __shared__ double s_alpha;
    const int nn = (it + 1) & 1;
    if (threadIdx.x == 0) {
        const double rz = sc[it & 1], pq = sc[2 + (it & 1)];
        s_alpha = pq > 0.0 ? rz / pq : 0.0;
    }
    __syncthreads();
    const double alpha = s_alpha;
    double rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (minv[i] != 0.0) {
            U[i] += alpha * pv[i];
            const double ri = r[i] - alpha * qv[i];
            r[i] = ri;
            rr = fma(ri, ri, rr);
        }
    if (threadIdx.x == 0 && blockIdx.x == 0) sc[2 + nn] = 0.0;
    const double tot[1] = {block_sum(rr, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[4 + nn] += v; });
}

// sc[slot] += r.z; with first = 1 also p = z
__global__ void __launch_bounds__(256) k_cg_rz(int64_t N, const double *__restrict__ r, const double *__restrict__ z,
                                               double *pv, double *sc, int slot, int first, double *gpart,
                                               unsigned *gcount) {
    __shared__ double sh[8];
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        v = fma(r[i], z[i], v);
        if (first) pv[i] = z[i];
    }
    const double tot[1] = {block_sum(v, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double x) { sc[slot] += x; });
}

// beta = rz'/rz; p = z + beta p
// p = z + beta p (beta = rz'/rz); with pf also p as float32 pairs
__global__ void k_cg_dir(int64_t N, const double *__restrict__ z, double *pv, float2 *pf, const double *sc, int it) {
    __shared__ double s_beta;
    if (threadIdx.x == 0) {
        const double rz = sc[it & 1], rz2 = sc[(it + 1) & 1];
        s_beta = rz > 0.0 ? rz2 / rz : 0.0;
    }
    __syncthreads();
    const double beta = s_beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = z[i] + beta * pv[i];
        pv[i] = v;
        if (pf) pf[i] = ff_split(v);
    }
}

// Per tetrahedron: V_H(x_q) from the nodal U, LDA at rho_q, V_q = V_ext + V_H + V_xc, the
// weighted values w V_q of the local potential matrix (ve, in the precision of the H values: the
// float64 products cost as much as the rest of the kernel on GB300's FP64 pipe), and the
// double-counting sum w (V_H/2 + V_xc - eps_xc) rho.
template <class E>
__global__ void __launch_bounds__(128) k_potential(int64_t T, const int *__restrict__ tetn,
                                                   const double *__restrict__ wq,
                                                   const double *__restrict__ vext,
                                                   const double *__restrict__ rho,
                                                   const double *__restrict__ U, int do_h, int do_xc,
                                                   double *vh, double *vxc, double *exc,
                                                   E *ve, double *edc, double *gpart, unsigned *gcount) {
    __shared__ double sh[4];
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (t < T) {
        const double w = wq[t];
        for (int q = 0; q < 4; ++q) {
            double h = 0.0;
            if (do_h)
                for (int a = 0; a < 10; ++a) h += p2N(q, a) * U[tetn[t * 10 + a]];
            double r = rho[t * 4 + q], vx = 0.0, ex = 0.0;
            if (do_xc) {
                if constexpr (sizeof(E) == 4) {
                    float vf;
                    ex = (double)lda<float>((float)r, vf);
                    vx = (double)vf;
                } else {
                    ex = lda<double>(r, vx);
                }
            }
            vh[t * 4 + q] = h; vxc[t * 4 + q] = vx; exc[t * 4 + q] = ex;
            ve[t * 4 + q] = (E)(w * (vext[t * 4 + q] + h + vx));
            e += w * (0.5 * h + vx - ex) * r;
        }
    }
    const double tot[1] = {block_sum(e, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { *edc = v; });
}

// H = L/2 + sum over the element entries (T, a, b) that land on each SELL position of
// sum_q (w V_q)_T N_a(x_q) N_b(x_q) (Eq. hamiltonian), gathered in list order in the precision of
// the H values (the same value on every run).  The 100 x 4 products N_a(x_q) N_b(x_q) sit in shared
// memory in the precision of H, so an entry costs one list load, one 4-vector load of w V and four
// multiply-adds (no float64 arithmetic in the float32 form).
template <class E>
__global__ void __launch_bounds__(256) k_h_gather(int64_t npos, const int *__restrict__ ptr, const int *__restrict__ list,
                                                  const E *__restrict__ ve, const E *__restrict__ valL, E *valH) {
    __shared__ E tab[100 * 4];
    for (int i = threadIdx.x; i < 400; i += blockDim.x) {
        const int ab = i >> 2, q = i & 3, a = ab / 10, b = ab - 10 * a;
        tab[i] = (E)(p2N(q, a) * p2N(q, b));
    }
    __syncthreads();
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    E acc = E(0.5) * valL[pos];
    const int k1 = ptr[pos + 1];
    for (int k = ptr[pos]; k < k1; ++k) {
        const int code = __ldg(list + k), t = code / 100, ab = code - 100 * t;
        E v[4];
        if constexpr (sizeof(E) == 4) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(ve) + t);
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else {
            const double2 x0 = __ldg(reinterpret_cast<const double2 *>(ve) + 2 * (int64_t)t);
            const double2 x1 = __ldg(reinterpret_cast<const double2 *>(ve) + 2 * (int64_t)t + 1);
            v[0] = x0.x; v[1] = x0.y; v[2] = x1.x; v[3] = x1.y;
        }
        const E *w = tab + ab * 4;
        E m = E(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) m += v[q] * w[q];
        acc += m;
    }
    valH[pos] = acc;
}

}  // namespace

// Poisson load and multipole moments from the density (Hartree on)
static int density_tail(ofks_ctx *c, int do_h) {
    if (do_h) {
        const int64_t N = c->n_nodes;
        k_rhs_gather<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(N, c->d_nptr, c->d_nlist, c->d_wq, c->d_rho,
                                                                         c->d_rhs);
        const unsigned gm = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 152LL * 4));
        k_moments<<<gm, 256, 0, c->stream>>>(N, c->d_ynode, c->d_rhs, c->d_sc + SC_MOM, c->d_gpart, c->d_gcount);
        c->kernels += 2;
    }
    return ofks_cuda_check(c, cudaGetLastError(), "density kernel");
}

template <class E>
int launch_density(ofks_ctx *c, const E *X) {
    ProfScope ps(c, PF_DENSITY);
    const int64_t T = c->n_tets;
    const int do_h = c->prm.hartree ? 1 : 0;
    if (c->ld % 4 == 0) {
        // lanes per tetrahedron: up to three 4-column chunks per lane, at most 8 lanes
        const int nch = c->ld / 4;
        int G4 = 1;
        while (G4 < 8 && G4 * 3 < nch) G4 *= 2;
        const int64_t warps4 = (T + 32 / G4 - 1) / (32 / G4);
        const unsigned grid4 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps4 * 32 + 255) / 256, 152LL * 16));
#define DENS4(g) k_density4<E, g><<<grid4, 256, 0, c->stream>>>(T, c->ld, c->prm.occ, X, c->d_tetf, c->d_rho)
        switch (G4) {
            case 1: DENS4(1); break;
            case 2: DENS4(2); break;
            case 4: DENS4(4); break;
            default: DENS4(8); break;
        }
#undef DENS4
        c->kernels += 1;
        return density_tail(c, do_h);
    }
    // group width: the fewest wasted column slots ceil(p/G) G, preferring wide groups on ties
    int G = c->p <= 2 ? c->p : 4;
    if (c->p > 2)
        for (int g = 8; g <= 32; g <<= 1)
            if ((c->p + g - 1) / g * g <= (c->p + G - 1) / G * G) G = g;
    const int B = 256;
    const int64_t warps = (T + 32 / G - 1) / (32 / G);
    unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps * 32 + B - 1) / B, 152LL * 16));
#define DENS(g) k_density<E, g><<<grid, B, 0, c->stream>>>(T, c->p, c->ld, c->prm.occ, X, c->d_tetf, c->d_rho)
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
    return density_tail(c, do_h);
}

int hartree_pc(ofks_ctx *c) {
    if (c->prm.poisson_pc == OFKS_HPC_SEPARABLE && c->sep.on) return OFKS_HPC_SEPARABLE;
    if (c->prm.poisson_pc == OFKS_HPC_MULTIGRID && !c->amg_tried && c->n_nodes > 0) {
        // optional: without the hierarchy the CG runs with the Jacobi preconditioner
        c->amg_tried = true;
        const std::string keep = c->err;
        if (amg_setup(c, c->h_tetn.data(), c->n_tets, c->h_xyz.data()) != OFKS_OK) { amg_free(c); c->err = keep; }
    }
    if (c->prm.poisson_pc == OFKS_HPC_MULTIGRID && !c->amg.empty()) return OFKS_HPC_MULTIGRID;
    return OFKS_HPC_JACOBI;
}

int run_hartree(ofks_ctx *c) {
    if (!c->prm.hartree) return OFKS_OK;
    ProfScope ps(c, PF_POISSON);
    const int64_t N = c->n_nodes;
    const unsigned gN = (unsigned)((N + 255) / 256);
    const unsigned gU = std::min(gN, 152u * 8u);   // grid-stride: fewer same-address atomics
    double *sc = c->d_sc + SC_CG;
    k_boundary<<<(c->n_bnd + 255) / 256, 256, 0, c->stream>>>(c->n_bnd, c->d_bnd, c->d_bxyz,
                                                               c->d_sc + SC_MOM, c->prm.multipole_lmax,
                                                               c->d_U);
    cudaMemsetAsync(sc, 0, sizeof(double) * 8, c->stream);
    if (c->st.on && !c->prm.poisson_csr) {   // the lattice-stencil residual, then the CG start
        launch_stencil_residual(c, c->d_U, c->d_rhs, c->d_cr);
        k_cg_init_vec<<<gN, 256, 0, c->stream>>>(N, c->d_minv, c->d_rhs, c->d_cr, c->d_cz, c->d_cp, sc, c->d_gpart,
                                                 c->d_gcount);
    } else {
        k_cg_init<<<gN, 256, 0, c->stream>>>(N, c->d_fptr, c->d_fcol, c->d_fval, c->d_minv, c->d_rhs, c->d_U,
                                             c->d_cr, c->d_cz, c->d_cp, sc, c->d_gpart, c->d_gcount);
    }
    c->kernels += 2;
    const int pc = hartree_pc(c);
    const bool amg = pc != OFKS_HPC_JACOBI;             // a preconditioner other than the diagonal
    auto precond = [&]() {
        ProfScope pp(c, PF_POISSON_PC);
        amg_apply(c, c->d_cr, c->d_cz);
    };
    const bool sep = pc == OFKS_HPC_SEPARABLE;
    const bool lat = c->st.on && !c->prm.poisson_csr;
    // during the float32 iterations the lattice SpMV of the separable CG runs in float-float
    // arithmetic (~48 bits, its tolerance is at least poisson_tol_mixed); float64 otherwise
    c->hartree_ff = sep && lat && c->phase == 32 && c->st.valff != nullptr;
    auto spmv = [&](int it) {
        ProfScope pv(c, PF_POISSON_SPMV);
        if (lat) { launch_stencil_spmv(c, c->d_cp, c->d_cq, sc, it); return; }
        k_cg_spmv<<<gN, 256, 0, c->stream>>>(N, c->d_fptr, c->d_fcol, c->d_fval, c->d_minv, c->d_cp, c->d_cq, sc,
                                              it, c->d_gpart, c->d_gcount);
        c->kernels += 1;
    };
    if (sep) {          // z = A_sep^-1 r, rz[0] = r.z, p = z
        cudaMemsetAsync(sc, 0, sizeof(double), c->stream);
        ProfScope pp(c, PF_POISSON_PC);
        sep_cg_step(c, -1, 0, 1);
    } else if (amg) {   // z = M^-1 r by the multigrid cycle, rz[0] = r.z, p = z
        cudaMemsetAsync(sc, 0, sizeof(double), c->stream);
        precond();
        k_cg_rz<<<gU, 256, 0, c->stream>>>(N, c->d_cr, c->d_cz, c->d_cp, sc, 0, 1, c->d_gpart, c->d_gcount);
        c->kernels += 1;
    }
    double ptol = c->phase == 32 ? std::max(c->prm.poisson_tol, c->prm.poisson_tol_mixed) : c->prm.poisson_tol;
    if (c->hartree_tol > 0.0) ptol = std::max(ptol, c->hartree_tol);
    const double tol2 = ptol * ptol;
    int chunk = amg ? 4 : 32;
    int it = 0, it_prev = 0;
    double h[8], rr_prev = 0.0;
    for (;;) {
        cudaError_t e = cudaMemcpyAsync(h, sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ofks_cuda_check(c, e, "Hartree CG");
        const double rr = h[4 + (it & 1)], bb = h[6];
        if (!std::isfinite(rr)) return ofks_fail(c, OFKS_ENONFINITE, "Hartree CG residual is not finite");
        if (rr <= tol2 * bb || bb == 0.0) {
            if (sep && it > it_prev && rr_prev > 0.0 && rr > 0.0 && rr < rr_prev)
                c->cg_rate = std::pow(rr / rr_prev, 1.0 / (it - it_prev));
            c->cg_last = it;
            c->cg_total += it;
            break;
        }
        if (it >= c->prm.poisson_max_iter)
            return ofks_fail(c, OFKS_ETIMEOUT, "Hartree CG: %d iterations, relative residual %.3e",
                             it, std::sqrt(rr / bb));
        // with the separable preconditioner the squared residual falls by a steady factor per
        // iteration: run the count that factor predicts to the target (1 to 8) before the next
        // check, not a fixed 4 (the first chunk uses the last solve's factor)
        if (sep) {
            double f = c->cg_rate;
            if (it > 0 && rr_prev > 0.0 && rr < rr_prev) f = std::pow(rr / rr_prev, 1.0 / (it - it_prev));
            chunk = 4;
            if (f > 0.0 && f < 1.0) {
                c->cg_rate = f;
                const double need = std::log(tol2 * bb / rr) / std::log(f);
                chunk = (int)std::min(8.0, std::max(1.0, std::ceil(need)));
            }
            rr_prev = rr;
            it_prev = it;
        }
        if (sep) {
            // `chunk` CG iterations between residual checks; their kernels use the iteration
            // number only through its parity (it >= 0), so one captured graph per chunk length
            // and parity of its first iteration serves every chunk
            struct Chunk { ofks_ctx *c; int it0, n; bool lat, ff; unsigned gN, gU; int64_t N; double *sc; };
            Chunk C{c, it, chunk, lat, c->hartree_ff, gN, gU, N, sc};
            auto body = [](void *a) {
                Chunk &K = *static_cast<Chunk *>(a);
                ofks_ctx *c = K.c;
                for (int it = K.it0; it < K.it0 + K.n; ++it) {
                    {
                        ProfScope pv(c, PF_POISSON_SPMV);
                        if (K.ff) launch_stencil_spmv_ff(c, c->d_cpff, c->d_cp, c->d_cq, K.sc, it);
                        else if (K.lat) launch_stencil_spmv(c, c->d_cp, c->d_cq, K.sc, it);
                        else {
                            k_cg_spmv<<<K.gN, 256, 0, c->stream>>>(K.N, c->d_fptr, c->d_fcol, c->d_fval, c->d_minv,
                                                                   c->d_cp, c->d_cq, K.sc, it, c->d_gpart,
                                                                   c->d_gcount);
                            c->kernels += 1;
                        }
                    }
                    {
                        ProfScope pp(c, PF_POISSON_PC);
                        sep_cg_step(c, it, (it + 1) & 1, 0);    // update, precondition, r.z
                    }
                    {
                        ProfScope pu(c, PF_POISSON_VEC);
                        k_cg_dir<<<K.gU, 256, 0, c->stream>>>(K.N, c->d_cz, c->d_cp, K.ff ? c->d_cpff : nullptr, K.sc, it);
                    }
                    c->kernels += 1;
                }
            };
            int rc;
            if ((rc = run_graph(c, {2, chunk, it & 1, lat ? 1 : 0, (c->sep.tc && c->prm.poisson_sep_tc) ? 1 : 0,
                                    c->hartree_ff ? 1 : 0},
                                body, &C)))
                return rc;
            it += chunk;
        }
        for (int j = 0; j < chunk && amg && !sep; ++j, ++it) {
            spmv(it);
            {
                ProfScope pu(c, PF_POISSON_VEC);
                k_cg_update_r<<<gU, 256, 0, c->stream>>>(N, c->d_minv, c->d_cp, c->d_cq, c->d_U, c->d_cr, sc, it,
                                                         c->d_gpart, c->d_gcount);
            }
            precond();
            {
                ProfScope pu(c, PF_POISSON_VEC);
                k_cg_rz<<<gU, 256, 0, c->stream>>>(N, c->d_cr, c->d_cz, c->d_cp, sc, (it + 1) & 1, 0, c->d_gpart,
                                                   c->d_gcount);
                k_cg_dir<<<gU, 256, 0, c->stream>>>(N, c->d_cz, c->d_cp, nullptr, sc, it);
            }
            c->kernels += 3;
        }
        for (int j = 0; j < chunk && !amg; ++j, ++it) {
            spmv(it);
            {
                ProfScope pu(c, PF_POISSON_VEC);
                k_cg_update<<<gU, 256, 0, c->stream>>>(N, c->d_minv, c->d_cp, c->d_cq, c->d_U, c->d_cr,
                                                       c->d_cz, sc, it, c->d_gpart, c->d_gcount);
                k_cg_dir<<<gU, 256, 0, c->stream>>>(N, c->d_cz, c->d_cp, nullptr, sc, it);
            }
            c->kernels += 2;
        }
    }
    if (sep && c->sep.tc && c->prm.poisson_sep_tc) {   // a tensor-core wait that timed out
        int hf = 0;
        cudaError_t e = cudaMemcpyAsync(&hf, c->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ofks_cuda_check(c, e, "Hartree CG");
        if (hf) {
            cudaMemsetAsync(c->d_flag + 1, 0, sizeof(int), c->stream);
            return ofks_fail(c, OFKS_ETIMEOUT, "Hartree preconditioner: tensor-core wait timed out");
        }
    }
    return ofks_cuda_check(c, cudaGetLastError(), "Hartree CG");
}

template <class E>
int launch_potential_refresh(ofks_ctx *c, E *valH, const E *valL) {
    ProfScope ps(c, PF_POTENTIAL);
    const int64_t T = c->n_tets;
    E *ve = reinterpret_cast<E *>(c->d_ve);
    k_potential<E><<<(unsigned)((T + 127) / 128), 128, 0, c->stream>>>(
        T, c->d_tetn, c->d_wq, c->d_vext, c->d_rho, c->d_U, c->prm.hartree ? 1 : 0, c->prm.xc ? 1 : 0, c->d_vh,
        c->d_vxc, c->d_exc, ve, c->d_sc + SC_EDC, c->d_gpart, c->d_gcount);
    k_h_gather<E><<<(unsigned)((c->sell_len + 255) / 256), 256, 0, c->stream>>>(c->sell_len, c->d_hptr, c->d_hlist,
                                                                               ve, valL, valH);
    c->kernels += 2;
    return ofks_cuda_check(c, cudaGetLastError(), "potential kernel");
}

template int launch_density<double>(ofks_ctx *, const double *);
template int launch_density<float>(ofks_ctx *, const float *);
template int launch_potential_refresh<double>(ofks_ctx *, double *, const double *);
template int launch_potential_refresh<float>(ofks_ctx *, float *, const float *);
