// p x p work of one PCAL iteration and of the set-up / post-processing, each on a single CTA:
//   * multipliers Lambda = Lambda0 + Theta(Lambda0 - S Lambda0 + beta S (S - I))  (Eq. lambda2;
//     Lambda = Lambda0 for PLAM, Eq. multi, and MOptQR), C = beta (S - I) - Lambda (C = -Lambda0 for
//     MOptQR), preconditioner shifts (Eq. precondition-T), fea and E
//   * the step parameter eta (Barzilai-Borwein, Sec. 4.4)
//   * Cholesky S = R^T R and R^{-1} for the initial guess (Sec. 4.2)
//   * Rayleigh-Ritz (Sec. 4.3): Cholesky, R^{-T} A R^{-1}, parallel cyclic Jacobi, V = R^{-1} W
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace {

// method: OFKS_METHOD_PCAL adds Theta(.) to Lambda0 (Eq. lambda2); PLAM keeps Lambda = Lambda0
// (Eq. multi); MOptQR keeps Lambda = Lambda0 and has no penalty, so C = -Lambda0 and the gradient
// is the antigradient H X - B X Lambda0
__global__ void __launch_bounds__(256) k_small_update(int p, int ld, const double *__restrict__ L0,
                                                      const double *__restrict__ S, double beta, int method,
                                                      int precond, double occ, double e_nuc, const double *sc,
                                                      double *Lam, double *C, double *cb, double *rec) {
    const bool theta_on = method == OFKS_METHOD_PCAL;
    const double beta_c = method == OFKS_METHOD_MOPTQR ? 0.0 : beta;
    __shared__ double red[8];
    double fea2 = 0.0, tr = 0.0;
    for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
        const int i = idx / ld, j = idx % ld;
        if (i >= p || j >= p) { Lam[idx] = 0.0; C[idx] = 0.0; continue; }
        const double sij = S[idx] - (i == j ? 1.0 : 0.0);
        fea2 += sij * sij;
        double lam = L0[idx];
        if (i == j) tr += lam;
        if (i == j && theta_on) {
            // diagonal of Lambda0 - S Lambda0 + beta S (S - I)
            double sl = 0.0, ss = 0.0;
            for (int k = 0; k < p; ++k) {
                const double sik = S[(int64_t)i * ld + k];
                sl += sik * L0[(int64_t)k * ld + i];
                ss += sik * (S[(int64_t)k * ld + i] - (k == i ? 1.0 : 0.0));
            }
            lam += L0[idx] - sl + beta * ss;
        }
        Lam[idx] = lam;
        C[idx] = beta_c * sij - lam;
    }
    fea2 = block_sum(fea2, red);
    tr = block_sum(tr, red);
    __syncthreads();
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        const double ljj = j < p ? Lam[(int64_t)j * ld + j] : 0.0;
        const bool act = precond && j < p && ljj < 0.0;
        cb[CB_SHIFT * ld + j] = act ? ljj : 0.0;
        cb[CB_ACTIVE * ld + j] = act ? 1.0 : 0.0;
        cb[CB_ACC * ld + j] = 0.0;
        cb[CB_WARM * ld + j] = 0.0;
    }
    if (threadIdx.x == 0) {
        rec[0] = occ * tr - sc[SC_EDC] + e_nuc;   // E_KS in the double-counting form
        rec[1] = sqrt(fea2);
    }
}

__global__ void k_record_kkt(const double *sc, double *rec) { rec[2] = sqrt(sc[SC_KKT2]); }

// eta_k by the selected rule, clamped to [eta_min, eta_max]
__global__ void k_eta(int rule, int k, int have_prev, double eta_fixed, double eta_min, double eta_max,
                      double *sc, double *rec) {
    double eta;
    const double sy = sc[SC_BB], yy = sc[SC_BB + 1], ss = sc[SC_BB + 2];
    if (rule == OFKS_ETA_FIXED) {
        eta = eta_fixed;
    } else if (!have_prev) {
        eta = sqrt(sc[SC_DNRM2]) / (1e-3 * sqrt(sc[SC_XNRM2]));
    } else {
        int r = rule;
        if (r == OFKS_ETA_ABB1) r = (k % 2 == 1) ? OFKS_ETA_BB1 : OFKS_ETA_BB2;
        else if (r == OFKS_ETA_ABB2) r = (k % 2 == 1) ? OFKS_ETA_BB2 : OFKS_ETA_BB1;
        if (sy == 0.0) eta = sc[SC_ETA];
        else if (r == OFKS_ETA_BB1) eta = fabs(sy) / ss;
        else eta = yy / fabs(sy);
    }
    eta = fmin(fmax(eta, eta_min), eta_max);
    sc[SC_ETA] = eta;
    rec[3] = eta;
}

// one block per column j: pq_j = the operator apply's partials of column j added in unit order
// (0 for j >= pc); alpha_j = rz_j / pq_j (0 if pq_j <= 0); clear rzn
__global__ void __launch_bounds__(256) k_pcg_alpha(int ld, int pc, int64_t units, const double *__restrict__ part,
                                                   double *cb) {
    __shared__ double sh[8];
    const int j = blockIdx.x;
    const double pq = j < pc ? ordered_sum(part + (int64_t)j * units, units, sh) : 0.0;
    if (threadIdx.x == 0) {
        const double rz = cb[CB_RZ * ld + j];
        cb[CB_PQ * ld + j] = pq;
        cb[CB_ALPHA * ld + j] = (pq > 0.0 && cb[CB_ACC * ld + j] == 0.0) ? rz / pq : 0.0;
        cb[CB_RZN * ld + j] = 0.0;
    }
}

// per-column arrays of the compact PCG (stride w): compact column k < nact is column cmap[k]
// (stride ld in colA) and keeps its shift and warm-start flag; every other entry starts at zero
__global__ void k_pcg_compact_cols(int ld, int w, int nact, const int *__restrict__ cmap, const double *__restrict__ colA,
                                   double *colC) {
    for (int i = threadIdx.x; i < CB_COUNT * w; i += blockDim.x) colC[i] = 0.0;
    __syncthreads();
    for (int k = threadIdx.x; k < nact; k += blockDim.x) {
        colC[CB_SHIFT * w + k] = colA[CB_SHIFT * ld + cmap[k]];
        colC[CB_ACTIVE * w + k] = 1.0;
        colC[CB_WARM * w + k] = colA[CB_WARM * ld + cmap[k]];
    }
}

// one block per column j: rzn_j = the vector update's partials of column j added in unit order
// (0 for j >= pc); beta_j = rzn_j / rz_j (0 if rz_j <= 0); rz <- rzn; clear pq
__global__ void __launch_bounds__(256) k_pcg_beta(int ld, int pc, int64_t units, const double *__restrict__ part,
                                                  double *cb) {
    __shared__ double sh[8];
    const int j = blockIdx.x;
    const double rzn = j < pc ? ordered_sum(part + (int64_t)j * units, units, sh) : 0.0;
    if (threadIdx.x == 0) {
        const double rz = cb[CB_RZ * ld + j];
        cb[CB_RZN * ld + j] = rzn;
        cb[CB_BETA * ld + j] = rz > 0.0 ? rzn / rz : 0.0;
        cb[CB_RZ * ld + j] = rzn;
        cb[CB_PQ * ld + j] = 0.0;
    }
}

// S = R^T R (R upper); R and Rinv = R^{-1} written zero-padded (ld x ld).  flag = 1 if S is
// not positive definite.
__device__ void chol_upper(int p, int ld, const double *S, double *R, double *Rinv, double *A, int *flag) {
    for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
        A[idx] = S[idx];
        R[idx] = 0.0;
        Rinv[idx] = 0.0;
    }
    __syncthreads();
    __shared__ double piv;
    for (int j = 0; j < p; ++j) {
        if (threadIdx.x == 0) {
            // a pivot that lost all but ~13 digits of the original diagonal counts as zero
            const double d = A[(int64_t)j * ld + j];
            if (!(d > 1e-13 * fabs(S[(int64_t)j * ld + j]))) { *flag = 1; piv = 1.0; } else piv = sqrt(d);
            R[(int64_t)j * ld + j] = piv;
        }
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < p; c += blockDim.x) R[(int64_t)j * ld + c] = A[(int64_t)j * ld + c] / piv;
        __syncthreads();
        const int m = p - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int r = j + 1 + idx / m, c = j + 1 + idx % m;
            if (c >= r) A[(int64_t)r * ld + c] -= R[(int64_t)j * ld + r] * R[(int64_t)j * ld + c];
        }
        __syncthreads();
    }
    // columns of R^{-1} by back substitution, one column per thread
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        Rinv[(int64_t)c * ld + c] = 1.0 / R[(int64_t)c * ld + c];
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k) s += R[(int64_t)i * ld + k] * Rinv[(int64_t)k * ld + c];
            Rinv[(int64_t)i * ld + c] = -s / R[(int64_t)i * ld + i];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(512) k_cholesky_inv(int p, int ld, const double *S, double *scratch,
                                                      double *Rinv, int *flag) {
    chol_upper(p, ld, S, scratch, Rinv, scratch + (int64_t)ld * ld, flag);
}

// C = op(A) * B for p x p blocks (ld stride); ta: use A^T
__device__ void small_gemm(int p, int ld, const double *A, bool ta, const double *B, double *C) {
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
        const int i = idx / p, j = idx % p;
        double s = 0.0;
        for (int k = 0; k < p; ++k) s += (ta ? A[(int64_t)k * ld + i] : A[(int64_t)i * ld + k]) * B[(int64_t)k * ld + j];
        C[(int64_t)i * ld + j] = s;
    }
    __syncthreads();
}

// Rayleigh-Ritz on (A, S): eigs ascending, V (ld x ld) with V^T S V = I.
// scratch holds 5 ld x ld blocks.  The Jacobi sweep applies p/2 disjoint rotations at a time
// (round-robin pairing); each rotation zeroes a_ij with t = sign(th)/(|th| + sqrt(th^2+1)),
// th = (a_jj - a_ii)/(2 a_ij).
__global__ void __launch_bounds__(512) k_rayleigh_ritz(int p, int ld, const double *A, const double *S,
                                                       double *scratch, double *eigs, double *V, int *flag) {
    const int64_t L2 = (int64_t)ld * ld;
    double *R = scratch, *Ri = scratch + L2, *T = scratch + 2 * L2, *M = scratch + 3 * L2, *W = scratch + 4 * L2;
    chol_upper(p, ld, S, R, Ri, T, flag);
    small_gemm(p, ld, Ri, true, A, T);      // T = R^{-T} A
    small_gemm(p, ld, T, false, Ri, M);     // M = R^{-T} A R^{-1}
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
        const int i = idx / p, j = idx % p;
        const double v = 0.5 * (M[(int64_t)i * ld + j] + M[(int64_t)j * ld + i]);
        T[(int64_t)i * ld + j] = v;
        W[(int64_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ int pi[256], pj[256];
    __shared__ double pc[256], ps[256];
    __shared__ double red[16];
    __shared__ double offn, totn;
    const int m = (p % 2 == 0) ? p : p + 1, half = m / 2;
    for (int sweep = 0; sweep < 60 && p > 1; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
            const int i = idx / p, j = idx % p;
            const double v = T[(int64_t)i * ld + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (threadIdx.x == 0) { offn = off; totn = tot; }
        __syncthreads();
        if (!(offn > 1e-30 * totn) || offn == 0.0) break;
        for (int rnd = 0; rnd < m - 1; ++rnd) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                const int pa = k, pb = m - 1 - k;
                int a = pa == 0 ? 0 : 1 + (pa - 1 + rnd) % (m - 1);
                int b = pb == 0 ? 0 : 1 + (pb - 1 + rnd) % (m - 1);
                if (a > b) { int t = a; a = b; b = t; }
                double c = 1.0, s = 0.0;
                if (b < p) {
                    const double aij = T[(int64_t)a * ld + b];
                    if (aij != 0.0) {
                        const double th = (T[(int64_t)b * ld + b] - T[(int64_t)a * ld + a]) / (2.0 * aij);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + hypot(th, 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                } else {
                    a = b = -1;
                }
                pi[k] = a; pj[k] = b; pc[k] = c; ps[k] = s;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < half * p; idx += blockDim.x) {     // rows
                const int k = idx / p, col = idx % p;
                const int a = pi[k], b = pj[k];
                if (a < 0) continue;
                const double c = pc[k], s = ps[k];
                const double x = T[(int64_t)a * ld + col], y = T[(int64_t)b * ld + col];
                T[(int64_t)a * ld + col] = c * x - s * y;
                T[(int64_t)b * ld + col] = s * x + c * y;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < half * p; idx += blockDim.x) {     // columns
                const int k = idx / p, row = idx % p;
                const int a = pi[k], b = pj[k];
                if (a < 0) continue;
                const double c = pc[k], s = ps[k];
                double x = T[(int64_t)row * ld + a], y = T[(int64_t)row * ld + b];
                T[(int64_t)row * ld + a] = c * x - s * y;
                T[(int64_t)row * ld + b] = s * x + c * y;
                x = W[(int64_t)row * ld + a]; y = W[(int64_t)row * ld + b];
                W[(int64_t)row * ld + a] = c * x - s * y;
                W[(int64_t)row * ld + b] = s * x + c * y;
            }
            __syncthreads();
        }
    }
    // sort eigenvalues ascending (selection order) and permute W's columns into M
    __shared__ int order[256];
    if (threadIdx.x == 0) {
        for (int i = 0; i < p; ++i) order[i] = i;
        for (int i = 0; i < p; ++i) {
            int best = i;
            for (int j = i + 1; j < p; ++j)
                if (T[(int64_t)order[j] * ld + order[j]] < T[(int64_t)order[best] * ld + order[best]]) best = j;
            int t = order[i]; order[i] = order[best]; order[best] = t;
        }
        for (int i = 0; i < p; ++i) eigs[i] = T[(int64_t)order[i] * ld + order[i]];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
        const int i = idx / p, j = idx % p;
        M[(int64_t)i * ld + j] = W[(int64_t)i * ld + order[j]];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) V[idx] = 0.0;
    __syncthreads();
    small_gemm(p, ld, Ri, false, M, V);      // V = R^{-1} W
}

}  // namespace

void launch_small_update(ofks_ctx *c) { c->kernels += 1;
    ProfScope ps(c, PF_SMALL);
    k_small_update<<<1, 256, 0, c->stream>>>(c->p, c->ld, c->d_L0, c->d_S, c->prm.beta, c->prm.method,
                                             c->prm.precond != OFKS_PC_NONE ? 1 : 0, c->prm.occ, c->e_nuc,
                                             c->d_sc, c->d_Lam, c->d_C, c->d_colA, c->d_rec);
}

void launch_small_record(ofks_ctx *c) { c->kernels += 1; k_record_kkt<<<1, 1, 0, c->stream>>>(c->d_sc, c->d_rec); }

void launch_eta(ofks_ctx *c) { c->kernels += 1;
    k_eta<<<1, 1, 0, c->stream>>>(c->prm.eta_rule, c->k, c->have_prev ? 1 : 0, c->prm.eta_fixed, c->prm.eta_min,
                                  c->prm.eta_max, c->d_sc, c->d_rec);
}

void launch_pcg_alpha(ofks_ctx *c, int w, int pc, double *cb) {
    c->kernels += 1;
    k_pcg_alpha<<<w, 256, 0, c->stream>>>(w, pc, c->pq_units, c->d_cpart, cb);
}
void launch_pcg_beta(ofks_ctx *c, int w, int pc, double *cb) {
    c->kernels += 1;
    k_pcg_beta<<<w, 256, 0, c->stream>>>(w, pc, c->rz_units, c->d_cpart, cb);
}
void launch_pcg_compact_cols(ofks_ctx *c, int w, int nact, const int *cmap, double *colC) {
    c->kernels += 1;
    k_pcg_compact_cols<<<1, 256, 0, c->stream>>>(c->ld, w, nact, cmap, c->d_colA, colC);
}

void launch_cholesky_inv(ofks_ctx *c, const double *S, double *Rinv) { c->kernels += 1;
    k_cholesky_inv<<<1, 512, 0, c->stream>>>(c->p, c->ld, S, c->d_pp, Rinv, c->d_flag);
}

void launch_rayleigh_ritz(ofks_ctx *c, const double *A, const double *S, double *eigs, double *V) { c->kernels += 1;
    k_rayleigh_ritz<<<1, 512, 0, c->stream>>>(c->p, c->ld, A, S, c->d_pp, eigs, V, c->d_flag);
}
