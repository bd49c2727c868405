// Internal state and launcher prototypes of libofks (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ofks.h"

// Scalar accumulator slots in ctx->d_sc (float64, device).
enum {
    SC_MOM = 0,        // 10 multipole moments: Q, d(3), Qij (xx, yy, zz, xy, xz, yz)
    SC_EDC = 10,       // sum_q w (V_H/2 + V_xc - eps_xc) rho   (double-counting correction)
    SC_KKT2 = 11,      // ||H X - B X Lambda0||_F^2
    SC_BB = 12,        // <dX,dD>, <dD,dD>, <dX,dX>
    SC_ETA = 15,       // current eta
    SC_XNRM2 = 16,     // ||X||_F^2 (eta_0)
    SC_DNRM2 = 17,     // ||D||_F^2 (eta_0)
    SC_CG = 20,        // Poisson CG: rz[2] (ping-pong), pq[2], rr, rhs2, done flag, iters
    SC_COUNT = 32
};

// Kernel families timed by ofks_profile.
enum {
    PF_DENSITY = 0, PF_POISSON, PF_POTENTIAL, PF_SPMM_H, PF_GRAM, PF_SMALL, PF_GRAD,
    PF_PCG_SPMM, PF_PCG_UPDATE, PF_BB, PF_STEP, PF_SPMM_B, PF_OTHER, PF_POISSON_SPMV, PF_COUNT
};

// one level of the algebraic multigrid hierarchy of the Hartree Poisson operator (device CSR)
struct AmgMat {
    int64_t n = 0, m = 0;
    int *ptr = nullptr, *col = nullptr;
    double *val = nullptr;
};
struct AmgLevel {
    AmgMat A, P, R;                              // operator, prolongator, restriction = P^T
    double *dinv = nullptr;                      // inverse diagonal of A
    double omega = 0.0;                          // Jacobi damping 4 / (3 rho(D^-1 A))
    double *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
};

struct ofks_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    ofks_params prm{};

    // ---- mesh
    int64_t n_nodes = 0, n_tets = 0, n = 0;      // n: free DoFs
    int64_t nnz = 0;                             // stored entries of the free pattern
    int n_slices = 0;
    int64_t sell_len = 0;                        // padded SELL length
    int *d_slice_ptr = nullptr;                  // n_slices + 1 (entry offsets)
    int *d_slice_w = nullptr;                    // n_slices widths
    int *d_cols = nullptr;                       // sell_len free column ids
    int *d_perm = nullptr;                       // n_slices*32 -> free row id or -1
    double *d_valL = nullptr, *d_valB = nullptr, *d_valH = nullptr;
    double *d_dL = nullptr, *d_dB = nullptr;     // diagonals of L and B (free)
    // full-node stiffness for the Hartree Poisson problem (CSR)
    int64_t nnz_full = 0;
    int *d_fptr = nullptr, *d_fcol = nullptr;
    double *d_fval = nullptr, *d_minv = nullptr; // Jacobi inverse diagonal, 0 on the boundary
    // per tetrahedron
    int *d_tetf = nullptr;                       // T x 10 free ids (-1 on the boundary)
    int *d_tetn = nullptr;                       // T x 10 node ids
    int *d_emap = nullptr;                       // T x 100 SELL positions (-1 if not free)
    double *d_wq = nullptr;                      // T: |T|/4
    double *d_yq = nullptr;                      // T x 4 x 3 quadrature points minus centre
    double *d_vext = nullptr;                    // T x 4
    int n_bnd = 0;
    int *d_bnd = nullptr;                        // boundary node ids
    double *d_bxyz = nullptr;                    // n_bnd x 3 boundary node coords minus centre
    double center[3] = {0, 0, 0};
    std::vector<AmgLevel> amg;                   // Hartree preconditioner (empty: Jacobi)
    int *d_amg_idx = nullptr;                    // interior node ids (level 0 numbering)
    double *d_amg_chol = nullptr;                // dense inverse of the coarsest operator
    int64_t amg_ni = 0, amg_nc = 0;
    double e_nuc = 0.0;
    bool have_nuclei = false;

    // ---- quadrature and Hartree fields
    double *d_rho = nullptr, *d_vh = nullptr, *d_vxc = nullptr, *d_exc = nullptr;
    double *d_U = nullptr, *d_rhs = nullptr, *d_cr = nullptr, *d_cz = nullptr, *d_cp = nullptr,
           *d_cq = nullptr;

    // ---- blocks n x ld
    int p = 0, ld = 0;
    double *d_X[2] = {nullptr, nullptr};         // current / previous iterate (ping-pong)
    double *d_D[2] = {nullptr, nullptr};         // current / previous direction
    double *d_G[2] = {nullptr, nullptr};         // current / previous gradient
    double *d_HX = nullptr, *d_BX = nullptr;
    double *d_R = nullptr, *d_Z = nullptr, *d_P = nullptr, *d_Q = nullptr;   // PCG block
    double *d_W = nullptr;                       // PCG inverse Jacobi diagonal per column
    int cur = 0;                                 // index of the current X/D/G buffers
    // ---- small p x p (device)
    double *d_L0 = nullptr, *d_S = nullptr, *d_Lam = nullptr, *d_C = nullptr;
    double *d_colA = nullptr;                    // 4 x p column accumulators
    double *d_pp = nullptr;                      // p x p scratch (factorizations)
    double *d_sc = nullptr;                      // SC_COUNT scalars
    double *d_rec = nullptr;                     // iteration record (device)
    int *d_flag = nullptr;                       // error / status flags

    // ---- iteration state (host mirror)
    bool have_X = false, evaluated = false, have_prev = false;
    bool bx_valid = false;                       // d_BX holds B X for the current iterate
    int k = 0;
    int cg_last = 0;                             // CG iterations of the last Hartree solve
    int64_t cg_total = 0;                        // ... summed since the counter was cleared
    double kkt0 = 0.0, eta = 0.0;
    bool converged = false;
    double last_E = 0, last_kkt = 0, last_fea = 0;
    std::vector<double> history;                 // rows of 6
    double t_start = 0.0;
    double t_accum = 0.0;

    // ---- profiling
    int64_t kernels = 0;                         // kernel launches issued (all families)
    int64_t kernels_at_prof = 0;
    bool prof = false;
    int64_t prof_n[PF_COUNT] = {0};
    double prof_ms[PF_COUNT] = {0};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
};

// ---- helpers (api.cu)
int ofks_fail(ofks_ctx *c, int code, const char *fmt, ...);
int ofks_cuda_check(ofks_ctx *c, cudaError_t e, const char *what);
void prof_begin(ofks_ctx *c, int fam, cudaEvent_t *a, cudaEvent_t *b);
void prof_end(ofks_ctx *c, int fam, cudaEvent_t a, cudaEvent_t b);

struct ProfScope {
    ofks_ctx *c; int fam; cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(ofks_ctx *c_, int f) : c(c_), fam(f) { prof_begin(c, fam, &a, &b); }
    ~ProfScope() { prof_end(c, fam, a, b); }
};

// ---- setup.cu
int setup_mesh(ofks_ctx *c, int64_t n_nodes, const double *xyz, int64_t n_tets,
               const int64_t *tet10, const uint8_t *dirichlet);
int setup_nuclei(ofks_ctx *c, int M, const double *Z, const double *R);
int setup_nuclei_static(ofks_ctx *c, int M, const double *Z, const double *R);
void free_mesh(ofks_ctx *c);

// ---- fields.cu (density, potentials, Hamiltonian refresh, Poisson)
int launch_density(ofks_ctx *c, const double *X);
int run_hartree(ofks_ctx *c);
int launch_potential_refresh(ofks_ctx *c);

// ---- amg.cu (Hartree preconditioner)
int amg_setup(ofks_ctx *c, const int *tetn, int64_t T);
void amg_free(ofks_ctx *c);
void amg_apply(ofks_ctx *c, const double *r_full, double *z_full);

// ---- spmm.cu
void launch_sell_spmm(ofks_ctx *c, const double *val, const double *X, double *Y);
void launch_sell_spmm_colnorm(ofks_ctx *c, const double *val, const double *X, double *Y,
                              double *colsum);
void launch_pcg_apply(ofks_ctx *c, const double *Zin, double *P, double *Q, const double *beta_col,
                      const double *shift, double *pq, int first);

// ---- block.cu (tall-skinny products and vector updates)
void launch_gram2(ofks_ctx *c, const double *X, const double *A, const double *B, double *XA,
                  double *XB);
void launch_grad_update(ofks_ctx *c);
void launch_pcg_init(ofks_ctx *c);
void launch_pcg_update(ofks_ctx *c, int it);
void launch_direction_select(ofks_ctx *c);
void launch_bb_dots(ofks_ctx *c);
void launch_step_y(ofks_ctx *c, double *Y);
void launch_scale_cols(ofks_ctx *c, double *Y, double *BY, const double *colsum);
void launch_tri_solve_rows(ofks_ctx *c, const double *V, double *X, const double *Rinv);

// ---- small.cu (p x p work on one CTA)
void launch_small_update(ofks_ctx *c);
void launch_small_record(ofks_ctx *c);
void launch_eta(ofks_ctx *c);
void launch_cholesky_inv(ofks_ctx *c, const double *S, double *Rinv);
void launch_rayleigh_ritz(ofks_ctx *c, const double *A, const double *S, double *eigs,
                          double *V);
void launch_block_times_small(ofks_ctx *c, const double *X, const double *V, double *Y);
