/*
 * ofks.h - orthogonalization-free Kohn-Sham total-energy minimization (PCAL) on one GB300.
 *
 * C ABI of libofks.so.  The library solves the discretized Kohn-Sham problem
 *     min E_KS(X)  subject to  X^T B X = I_p,   X in R^{n x p}          (paper: Eq. prob:KS)
 * on a P2 tetrahedral mesh by the column-wise proximal linearized augmented Lagrangian
 * method PCAL (paper: Alg. 2) and post-processes with Rayleigh-Ritz (paper: Sec. 4.3).
 * Inputs follow the problem statement: mesh, nuclei, p and beta in; energy, orbitals and
 * eigenvalues out.  Every arithmetic step runs in CUDA kernels built for sm_103a; the host
 * side only builds index structures (sparsity patterns, element-to-entry maps) and drives
 * launches.  There is no CPU fallback: without a usable GPU every call fails.
 *
 * Conventions for every entry point
 *   - Return value: 0 on success, a negative OFKS_E* code on failure; the message is kept
 *     in the context and returned by ofks_last_error().  Nothing is thrown across the ABI.
 *   - Host arrays are owned by the caller and only read (inputs) or written (outputs)
 *     during the call; the library keeps its own device copies.
 *   - Blocks of orbitals are n_free x p, row-major, float64, where the free degrees of
 *     freedom are the non-Dirichlet nodes numbered in increasing global node id.
 *   - A context is bound to one device and is not thread-safe; calls on one context must
 *     be serialized by the caller.
 */
#ifndef OFKS_H
#define OFKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------- */
#define OFKS_OK            0
#define OFKS_EINVAL       -1   /* bad argument (size, range, pointer) */
#define OFKS_ECUDA        -2   /* a CUDA runtime call or kernel launch failed */
#define OFKS_ENOMEM       -3   /* device or host allocation failed */
#define OFKS_ESTATE       -4   /* call out of order (e.g. solve before set_mesh) */
#define OFKS_ENOTCONV     -5   /* iteration cap reached, or a Cholesky factor does not exist */
#define OFKS_ENONFINITE   -6   /* NaN/Inf met in energies or norms */
#define OFKS_ETIMEOUT     -7   /* an iterative inner solve hit its iteration limit */

/* ---- enumerations ------------------------------------------------------------------ */
#define OFKS_FP64          0   /* every step in float64 */
#define OFKS_MIXED         1   /* float32 iterations (float64 p x p, energies, tests), then a
                                  float64 refinement sweep once (kkt+fea)/kkt0 < mixed_tol, or once
                                  the float32 iterations have stalled below 1e-4 (no new best
                                  (kkt+fea)/kkt0 in 300 iterations) */

#define OFKS_PC_NONE       0   /* D = grad L_beta */
#define OFKS_PC_PCG        1   /* T_i^{-1} grad by Jacobi-PCG, fixed pcg_iters, zero start */
#define OFKS_PC_EXACT      2   /* the same PCG run to a 1e-12 relative residual */
#define OFKS_PC_LEARNED    3   /* graph network D = N(G), judged per column; PCG from D for rejects */

#define OFKS_ETA_BB2       0   /* eta = <dD,dD>/|<dX,dD>|, dD = difference of applied directions */
#define OFKS_ETA_BB1       1   /* eta = |<dX,dD>|/<dX,dX> */
#define OFKS_ETA_ABB1      2   /* BB1 on odd k, BB2 on even k */
#define OFKS_ETA_ABB2      3   /* BB2 on odd k, BB1 on even k */
#define OFKS_ETA_BB2_RAW   4   /* BB2 with differences of the raw gradients grad L_beta */
#define OFKS_ETA_FIXED     5   /* eta = eta_fixed every iteration */

/* the iteration (ofks_params.method) */
#define OFKS_METHOD_PCAL   0   /* Alg. 2: multipliers of Eq. (lambda2), column B-normalization
                                  (Eq. PCAL-main) */
#define OFKS_METHOD_PLAM   1   /* Alg. 1: multipliers of Eq. (multi), plain step X - D/eta
                                  (Eq. PLAM-main), no normalization */
#define OFKS_METHOD_MOPTQR 2   /* the manifold comparison method of Sec. 5: antigradient
                                  H X - B X X^T H X, the same preconditioner and step size, then the
                                  Cholesky-based Gram-Schmidt of Sec. 4.2 (Y^T B Y = R^T R,
                                  X <- Y R^{-1}): every iterate is B-orthonormal, at the cost of a
                                  p x p Cholesky factorization per iteration */

/* which fields ofks_get_field() copies out */
#define OFKS_F_RHO_Q       0   /* density at quadrature points, n_tets*4 */
#define OFKS_F_VH_Q        1   /* Hartree potential at quadrature points, n_tets*4 */
#define OFKS_F_VXC_Q       2   /* exchange-correlation potential at quadrature points */
#define OFKS_F_EXC_Q       3   /* exchange-correlation energy per particle at quadrature points */
#define OFKS_F_U           4   /* nodal Hartree potential, n_nodes (all nodes) */
#define OFKS_F_HX          5   /* H(X) X, n_free x p */
#define OFKS_F_BX          6   /* B X, n_free x p */
#define OFKS_F_G           7   /* grad_X L_beta(X, Lambda), n_free x p */
#define OFKS_F_D           8   /* preconditioned direction, n_free x p */
#define OFKS_F_LAMBDA0     9   /* X^T H X, p x p */
#define OFKS_F_S          10   /* X^T B X, p x p */
#define OFKS_F_LAMBDA     11   /* Eq. (lambda2) multipliers, p x p */
#define OFKS_F_VEXT_Q     12   /* external potential at quadrature points */

/* which matrix ofks_apply() multiplies with */
#define OFKS_M_L           0   /* stiffness on the free DoFs */
#define OFKS_M_B           1   /* mass on the free DoFs */
#define OFKS_M_H           2   /* current Hamiltonian L/2 + M_ext + M_Har + M_xc */

typedef struct ofks_ctx ofks_ctx;   /* opaque, owned by the library */

/* Preconditioners of the Hartree CG (ofks_params.poisson_pc). */
enum {
    OFKS_HPC_JACOBI = 0,     /* point Jacobi (inverse diagonal) */
    OFKS_HPC_MULTIGRID = 1,  /* V(2,2) cycle: P2 -> P1, then lattice coarsening (lattice meshes) or
                                smoothed aggregation (other meshes), damped Jacobi smoothing */
    OFKS_HPC_SEPARABLE = 2   /* lattice meshes: exact inverse of the separable Kronecker-sum operator
                                Kx(x)My(x)Mz + Mx(x)Ky(x)Mz + Mx(x)My(x)Kz (1-D linear stiffness K and
                                lumped mass M on the lattice coordinates) by fast diagonalization */
};

/* Preconditioner of the PCG that solves Eq. (precondition-T)'s systems T_k D = G (ofks_params.pcg_pc) */
enum {
    OFKS_PCGPC_JACOBI = 0,     /* the diagonal of T_k */
    OFKS_PCGPC_SEPARABLE = 1   /* lattice meshes, float32 PCG: the exact inverse of the separable
                                  A_sep / 2 - shift_k Mx (x) My (x) Mz (A_sep as for OFKS_HPC_SEPARABLE)
                                  by fast diagonalization on the tensor cores, all columns at once;
                                  elsewhere the diagonal */
};

typedef struct {
    int32_t p;              /* number of orbitals (columns of X) */
    double  beta;           /* penalty parameter of L_beta (paper Eq. ALM-sub) */
    double  occ;            /* electrons per orbital f: rho = f sum_l |psi_l|^2 */
    double  tol;            /* stop when (kkt + fea)/kkt_0 < tol (paper Sec. 4.1) */
    int32_t max_iter;       /* iteration cap of ofks_solve */
    int32_t precision;      /* OFKS_FP64 or OFKS_MIXED */
    int32_t precond;        /* OFKS_PC_* (paper Eq. precondition-T) */
    int32_t pcg_iters;      /* PCG iterations per preconditioner apply */
    int32_t eta_rule;       /* OFKS_ETA_* (paper Sec. 4.4) */
    double  eta_fixed;      /* used by OFKS_ETA_FIXED */
    double  eta_min, eta_max;   /* clamp of eta */
    int32_t hartree;        /* 1: Hartree term on; 0: off (fixed-potential problems) */
    int32_t xc;             /* 1: LDA (Slater + PZ81) on; 0: off */
    int32_t multipole_lmax; /* Hartree boundary data: multipoles up to l (0..2); -1: zero */
    double  poisson_tol;    /* relative residual of the Hartree CG solve */
    int32_t poisson_max_iter;
    int32_t poisson_pc;     /* Hartree CG preconditioner: OFKS_HPC_JACOBI, OFKS_HPC_MULTIGRID or
                               OFKS_HPC_SEPARABLE (falls back to Jacobi where the mesh has none) */
    double  mixed_tol;      /* OFKS_MIXED: hand over to float64 once (kkt+fea)/kkt0 < mixed_tol (or on a stall) */
    double  poisson_tol_mixed; /* Hartree CG tolerance during the float32 iterations (whose lattice
                                  SpMV, with the separable preconditioner, runs in float-float
                                  arithmetic: float32 pairs, ~48 bits) */
    double  judge_tau;      /* OFKS_PC_LEARNED: accept the network's column D if G.D > 0 and
                               |G - T D|_{M^-1} <= judge_tau |G|_{M^-1} (M the Jacobi diagonal of T,
                               |r|_{M^-1}^2 = r^T M^-1 r, the PCG's residual measure); a rejected column
                               runs the PCG, from D where that ratio is below 1, else from zero */
    int32_t learned_tc;     /* 1: width-64 hidden layer on the tensor cores (bf16 operands) at inference */
    int32_t poisson_adaptive; /* 1: Hartree CG tolerance max(poisson_tol, min(1e-4, 0.01 (kkt+fea)/kkt0))
                                 from the previous iterate (inexact potentials early, exact at the end) */
    int32_t poisson_csr;    /* 1: Hartree CG on the general CSR stiffness even when the mesh's node ids
                               follow a lattice (default 0: the lattice-stencil form when available) */
    int32_t gram_tc;        /* float32 dense contractions (mixed form): 1 (default) on the tensor cores --
                               the Grams with a bf16 hi/lo split (three products), the gradient
                               G = H X + B X C with a three-way split (six products), float32
                               accumulation (ld multiple of 4, ld <= 64); 0 float32 CUDA cores */
    int32_t spmm_f32_rows;  /* float32 block SpMMs (mixed form): 1 half a warp per row (lanes split the
                               columns), 0 (default) one lane per row and 4-column chunks */
    int32_t poisson_sep_tc; /* OFKS_HPC_SEPARABLE: 1 (default) the six axis contractions on the tensor
                               cores with bf16 operands, every intermediate tensor as a high and a low
                               bf16 part (axes up to 256 interior points), 0 float32 on the CUDA cores */
    int32_t pcg_compact;    /* OFKS_PC_PCG / OFKS_PC_EXACT: 1 (default) the PCG runs on the active
                               columns only (Lambda_ii < 0), gathered into a block of their count
                               rounded up to 4; the other columns take D = G (T = I) as always.
                               0: the PCG runs on all ld columns and discards the inactive ones */
    int32_t cuda_graphs;    /* 1 (default): fixed launch sequences (the fixed-count PCG loop, the Hartree
                               CG between residual checks) are captured once as CUDA graphs and
                               replayed; 0: every kernel is launched on its own.  Graphs are not
                               used while ofks_profile is on */
    int32_t pcg_staged;     /* float32 PCG at block widths 8..32 (multiples of 4): 1 row-major blocks and
                               an operator apply that stages the neighbour rows of each entry index
                               through shared memory; 0 (default, measured 3 % faster per PCG on the
                               chain with the vector updates included) the chunk-major blocks on the
                               type-grouped SELL (lattice meshes) */
    int32_t sweep_pc32;     /* OFKS_MIXED: 1 (default) the float64 sweep solves the preconditioner's systems
                               with the float32 PCG (the gradient rounded to float32, D widened back);
                               the gradient, Grams, energies and tests stay float64, so the fixed point
                               is unchanged.  0: float64 PCG in the sweep */
    int32_t method;         /* OFKS_METHOD_PCAL (default), OFKS_METHOD_PLAM or OFKS_METHOD_MOPTQR; the
                               stopping test (Sec. 4.1), the preconditioner (Eq. precondition-T, its
                               shifts from the method's multipliers) and eta are common to all three */
    int32_t learned_loss;   /* training loss of the learned preconditioner, per column c of negative shift:
                               1 (default) the energy-norm error (D - D*)^T T_c (D - D*) / G_c^T D*_c
                               (the norm the PCG reduces), averaged over those columns; 0 the relative
                               squared error |D - D*|^2 / |D*|^2 averaged over all columns */
    int32_t learned_retry;  /* OFKS_PC_LEARNED: after a call in which the judge took none of the network's
                               directions, the network sits out the next 1, 2, 4, ... calls (at most
                               learned_retry; reset once the judge takes one again), and those calls run
                               the PCG from zero; 0: the network runs on every call */
    int32_t pcg_pc;         /* OFKS_PCGPC_JACOBI (default) or OFKS_PCGPC_SEPARABLE: the preconditioner
                               inside the PCG (only the accuracy of D changes, never T or the fixed point) */
} ofks_params;

typedef struct {
    double  e_total;        /* E_KS at the last evaluated iterate (Hartree) */
    double  e_nuc;          /* nucleus-nucleus repulsion */
    double  kkt;            /* ||H X - B X X^T H X||_F */
    double  fea;            /* ||X^T B X - I||_F */
    double  kkt0;           /* kkt at iteration 0 */
    double  eta;            /* last step parameter */
    int32_t iters;          /* iterations taken so far (k) */
    int32_t converged;      /* 1 once (kkt + fea)/kkt0 < tol */
    double  seconds;        /* device time of the call, from CUDA events */
    int32_t hartree_iters;  /* CG iterations of the last Hartree solve */
    int32_t hartree_total;  /* CG iterations of all Hartree solves of the call */
    int32_t switch_iter;    /* OFKS_MIXED: iteration that started the float64 sweep, -1 before */
    int64_t judge_accept;   /* OFKS_PC_LEARNED: columns the judge accepted so far ... */
    int64_t judge_total;    /* ... out of this many judged */
    int32_t active_last;    /* columns with a negative multiplier (T != I) at the last direction */
    int64_t active_total;   /* ... summed over the directions computed so far */
    int64_t pcg_cols_total; /* block width of each PCG operator apply, summed over the applies so far
                               (the active count rounded up to 4 in the compact form, ld otherwise) */
    int64_t learned_calls;  /* OFKS_PC_LEARNED: network applications so far (calls outside a pause) */
    int64_t learned_warm;   /* ... columns the judge rejected whose PCG started from the network's D */
} ofks_result;

/* Fill *prm with the defaults: beta 10, occ 2, tol 1e-8, max_iter 1000, FP64, PCG with 8
 * iterations, BB2, eta in [1e-4, 1e8], Hartree and LDA on, multipole_lmax 2,
 * poisson_tol 1e-12, poisson_max_iter 20000, poisson_pc OFKS_HPC_SEPARABLE, mixed_tol 1e-6, poisson_tol_mixed
 * 1e-8, judge_tau 0.5, learned_tc 1, poisson_adaptive 0, poisson_csr 0, gram_tc 1, spmm_f32_rows 0,
 * poisson_sep_tc 1, pcg_compact 1, cuda_graphs 1, pcg_staged 0, sweep_pc32 1, method OFKS_METHOD_PCAL,
 * learned_loss 1, learned_retry 64, pcg_pc OFKS_PCGPC_JACOBI.  p is set to 1. */
void ofks_default_params(ofks_params *prm);

/* Create a context on CUDA device `device`.  *out receives the context (NULL on failure).
 * Errors: OFKS_ECUDA if the device cannot be used, OFKS_ENOMEM. */
int ofks_create(ofks_ctx **out, int device);

/* Release every device and host resource of the context.  Accepts NULL. */
void ofks_destroy(ofks_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  Valid until the next call. */
const char *ofks_last_error(const ofks_ctx *ctx);

/* Mesh (paper Sec. 2.2, discretization; Sec. 4.2 pre-processing).
 *   xyz       n_nodes x 3 node coordinates (bohr)
 *   tet10     n_tets x 10 node ids of P2 tetrahedra: vertices 0..3, then the midpoints of
 *             edges 01, 02, 03, 12, 13, 23 (straight-sided)
 *   dirichlet n_nodes flags, nonzero on the boundary (orbitals vanish there; the Hartree
 *             potential takes its multipole boundary values there)
 * Builds the sparsity patterns, assembles L and B on the device and resets orbitals,
 * nuclei-dependent data and history.  Errors: OFKS_EINVAL for ids out of range, a
 * degenerate tetrahedron or fewer than one free node; OFKS_ENOMEM. */
int ofks_set_mesh(ofks_ctx *ctx, int64_t n_nodes, const double *xyz,
                  int64_t n_tets, const int64_t *tet10, const uint8_t *dirichlet);

/* Nuclei (paper Eq. ext): M charges Z (> 0) at positions R (M x 3, bohr).  Evaluates V_ext
 * at the quadrature points and E_nuc.  Requires a mesh.  Errors: OFKS_EINVAL, OFKS_ESTATE. */
int ofks_set_nuclei(ofks_ctx *ctx, int32_t M, const double *Z, const double *R);

/* Largest number of nuclei ofks_set_nuclei_static accepts. */
#define OFKS_STATIC_NUCLEI_MAX 1024

/* ofks_set_nuclei without any device allocation (the paper has no counterpart: this is a
 * service of the library, not a step of the method).  For callers that cannot call cudaMalloc
 * -- code that moves the nuclei every step (relaxation, molecular dynamics) under a caching
 * allocator that owns the device memory, or in a loop where allocating is not allowed -- the
 * nuclear data is staged in a fixed array compiled into the library (OFKS_STATIC_NUCLEI_MAX
 * nuclei, 32 KiB per GPU that loads the library, held until the process exits) instead of
 * memory allocated per call.  Same arguments, results and errors as ofks_set_nuclei, plus
 * OFKS_EINVAL when M > OFKS_STATIC_NUCLEI_MAX.  ofks_create looks up the array's device address
 * on its device and keeps it in the context, so this call itself neither allocates nor looks
 * anything up.  All contexts share the array, which keeps the last call's contents: calls whose
 * work overlaps on the GPU (contexts driven concurrently) race. */
int ofks_set_nuclei_static(ofks_ctx *ctx, int32_t M, const double *Z, const double *R);

/* Parameters; p must satisfy 1 <= p <= n_free.  Changing p drops the orbitals.  A converged
 * context is reopened: the next ofks_step takes the stop test again under the new parameters
 * (and returns at once if it still holds).
 * Errors: OFKS_EINVAL for values out of range, OFKS_ESTATE without a mesh. */
int ofks_set_params(ofks_ctx *ctx, const ofks_params *prm);

/* Initial guess (paper Sec. 4.2): V (n_free x p, host) is B-orthonormalized by the
 * Cholesky-based Gram-Schmidt V = X0 R (R upper triangular) on the device, and the
 * iteration counter and history are reset.  Errors: OFKS_ENOTCONV if V^T B V is not
 * positive definite (V rank deficient), OFKS_ESTATE, OFKS_EINVAL. */
int ofks_init_orbitals(ofks_ctx *ctx, const double *V);

/* Set X directly (n_free x p, host, row-major; the caller keeps ownership), without
 * orthonormalization.  keep_history = 0 resets the iteration counter and the step-size history;
 * 1 keeps them (the caller re-uploads the block it read back).  The block travels as one
 * contiguous copy (page-locked host memory runs at the link's rate).  Errors: OFKS_ESTATE (no
 * mesh or params), OFKS_EINVAL (null pointer), OFKS_ECUDA. */
int ofks_set_orbitals(ofks_ctx *ctx, const double *X, int32_t keep_history);

/* Copy the current X (n_free x p, row-major) into the caller's host buffer X; returns after the
 * copy has landed.  Errors: OFKS_ESTATE (no orbitals yet), OFKS_EINVAL, OFKS_ECUDA. */
int ofks_get_orbitals(ofks_ctx *ctx, double *X);

/* Run up to k iterations of Alg. 2 from the current state; stops early once the stopping
 * test of Sec. 4.1 holds.  res (may be NULL) receives the record of the last evaluated
 * iterate and the device time of the call.  Errors: OFKS_ESTATE (no orbitals),
 * OFKS_ENONFINITE, OFKS_ETIMEOUT (the Hartree solve hit poisson_max_iter), OFKS_ECUDA. */
int ofks_step(ofks_ctx *ctx, int32_t k, ofks_result *res);

/* Iterate until the stopping test holds or max_iter iterations; OFKS_ENOTCONV at the cap
 * (res is still filled). */
int ofks_solve(ofks_ctx *ctx, ofks_result *res);

/* Evaluate the current iterate without updating it: density, Hartree and xc potentials,
 * H(X), H X, B X, the Grams, E, kkt, fea, the multipliers of Eq. (lambda2) and the
 * gradient; fields are then readable with ofks_get_field().  Errors: OFKS_ETIMEOUT when a
 * bounded wait of the tensor-core Gram or gradient gave up (the fields are then not valid; the
 * status is cleared, so the next call starts clean), OFKS_ENONFINITE, OFKS_ECUDA. */
int ofks_evaluate(ofks_ctx *ctx, ofks_result *res);

/* Post-processing (paper Sec. 4.3): the p x p generalized eigenproblem
 * (X^T H X) v = lambda (X^T B X) v in float64 on the device, X <- X V.  eigs (host, p)
 * receives the eigenvalues in ascending order. */
int ofks_rayleigh_ritz(ofks_ctx *ctx, double *eigs);

/* Copy a field (OFKS_F_*) of the last evaluation into out (host), which holds `count`
 * doubles; count must equal the field's size.  Errors: OFKS_EINVAL, OFKS_ESTATE. */
int ofks_get_field(ofks_ctx *ctx, int32_t which, double *out, int64_t count);

/* Y = A X for A = OFKS_M_L, OFKS_M_B or OFKS_M_H on host blocks (n_free x ncols) through
 * the device SpMM kernel.  ncols must equal p. */
int ofks_apply(ofks_ctx *ctx, int32_t which, const double *X, double *Y, int32_t ncols);

/* Sizes: free DoFs, all nodes, tetrahedra, stored nonzeros of the free matrices
 * (without padding) and of the all-node stiffness of the Hartree problem.  Any pointer may
 * be NULL. */
int ofks_get_sizes(ofks_ctx *ctx, int64_t *n_free, int64_t *n_nodes, int64_t *n_tets,
                   int64_t *nnz, int64_t *nnz_full);

/* Storage of the Hartree Poisson operator (the all-node stiffness of Sec. 2.2).  *format = 1 when
 * the node ids follow a lattice, id = (a Ly + b) Lz + c with every stiffness neighbour within two
 * lattice steps, and the CG SpMV runs on the lattice-stencil form: no column indices, the
 * symmetric half stored once per node type (8 parity classes); 0 for the general CSR.
 * *stored = float64 values of the form in use, *rows = rows its SpMV computes (non-Dirichlet),
 * lattice[3] = (Lx, Ly, Lz) or zeros, *precond = the OFKS_HPC_* preconditioner the next solve uses
 * (after the fallback to Jacobi on meshes without the requested one).  Any pointer may be NULL.
 * Errors: OFKS_EINVAL, OFKS_ESTATE. */
int ofks_poisson_info(ofks_ctx *ctx, int32_t *format, int64_t *stored, int64_t *rows, int32_t *lattice,
                      int32_t *precond);

/* Measured FMA rate of the context's device in TFLOP/s (2 flops per FMA): precision OFKS_FP64
 * for float64 or 32 for float32.  Eight independent FMA chains per thread on every SM, about
 * 0.4 s of device time.  Not part of the method: the denominator of the ALU roofline of the
 * float64 kernels.  Errors: OFKS_EINVAL, OFKS_ECUDA. */
int ofks_fma_peak(ofks_ctx *ctx, int32_t precision, double *tflops);

/* History of evaluated iterates: rows of 6 doubles (k, seconds since init, E, kkt, fea,
 * eta).  Copies min(cap, available) rows of the most recent ones into buf; *len = rows. */
int ofks_get_history(ofks_ctx *ctx, double *buf, int32_t cap, int32_t *len);

/* ---- learned preconditioner (not in the paper: a graph network in place of the PCG, with
 * the paper's Eq. precondition-T as its acceptance test and fallback) ------------------------
 * The network maps a gradient column G_c to an approximation of T_c^{-1} G_c on the free-DoF
 * graph of the mesh: input features [z/s, log diag - mean, -lam dB/diag, 1] with
 * z = G / diag, diag = dL/2 - lam dB, s = rms(z); layers Z = H W + (A H) U + b (A: mean over the
 * closed neighbourhood), widths 4 -> width -> width -> 1, relu on the hidden layers; output
 * D = s (z/s + y).  Parameters: float32 masters rounded to bfloat16 where used, flat layout
 * W0, U0, b0, W1, U1, b1, W2, U2, b2 (W and U row-major fan_in x fan_out). */

/* Random initialization (seeded; last layer zero, so the network starts as the Jacobi step).
 * width in {8, 16, 32, 64}.  Requires a mesh.  Resets the optimizer state. */
int ofks_precond_init(ofks_ctx *ctx, int32_t width, uint64_t seed);

/* Copy the parameters out (cap >= *count) or in (count must match the width's size). */
int ofks_precond_get_weights(ofks_ctx *ctx, float *w, int64_t cap, int64_t *count);
int ofks_precond_set_weights(ofks_ctx *ctx, const float *w, int64_t count);

/* D (n_free x p, host) = preconditioned directions of G (host) for per-column shifts (host, p;
 * columns with shift >= 0 take D = G, Eq. precondition-T): mode OFKS_PC_PCG, OFKS_PC_EXACT or
 * OFKS_PC_LEARNED (the network alone, no acceptance test).  The PCG modes solve the active
 * columns only when pcg_compact is set, as the iterations do.  Uses the context's scratch
 * blocks; iteration history is kept.  A mixed context (OFKS_MIXED, float32 blocks allocated)
 * runs OFKS_PC_PCG in float32 as its iterations do.  Errors: OFKS_EINVAL (null pointer, unknown
 * mode), OFKS_ESTATE (no mesh or params; OFKS_PC_LEARNED without a network), OFKS_ETIMEOUT (a
 * bounded device wait gave up), OFKS_ECUDA. */
int ofks_precondition(ofks_ctx *ctx, int32_t mode, const double *G, const double *shifts, double *D);

/* One Adam step (learning rate lr) of the network on the pair (G, Dstar) with per-column
 * shifts; *loss receives the loss before the step (mean over columns of |D - D*|^2/|D*|^2).
 * Errors: OFKS_ESTATE (no network: ofks_precond_init first), OFKS_EINVAL, OFKS_ECUDA. */
int ofks_train_precond_step(ofks_ctx *ctx, const double *G, const double *shifts, const double *Dstar,
                            double lr, double *loss);

/* Loss and parameter gradients (float64, same layout as the weights) without a step. */
int ofks_precond_grads(ofks_ctx *ctx, const double *G, const double *shifts, const double *Dstar,
                       double *grads, int64_t cap, double *loss);

/* Append one training pair generated by the method itself at the current iterate to the pairs
 * file at `path` (created with its header when absent): the gradient G = grad_X L_beta(X, Lambda)
 * (n_free x p), the shifts diag(Lambda) of Eq. (lambda2), and the target D* = T^{-1} G of
 * Eq. (precondition-T) solved to a 1e-12 relative residual (columns with a shift >= 0 take
 * D* = G).  File layout, all little-endian: magic "OFKSPR1\0" (8 bytes), int64 n_free, int32 p,
 * int32 zero; then per pair: float64 shifts[p], G[n_free x p], D*[n_free x p] (row-major).
 * *active (may be NULL) receives the number of columns with a negative shift.  The current
 * iterate is evaluated, not moved.  Errors: OFKS_ESTATE (no orbitals), OFKS_EINVAL (the file
 * exists with other sizes, or cannot be written), OFKS_ENOMEM, OFKS_ECUDA, OFKS_ETIMEOUT. */
int ofks_record_pair(ofks_ctx *ctx, const char *path, int32_t *active);

/* Train the network (ofks_precond_init or ofks_precond_set_weights first) on the pairs of the
 * file at `pairs_path`, which must have this context's n_free and p (pairs live on one mesh):
 * `epochs` passes over the pairs, each in an order shuffled by the SplitMix64 generator seeded
 * with (seed, epoch), one Adam step with learning rate 1e-3 per pair on the loss of
 * ofks_train_precond_step.  The Adam moments continue from earlier steps of this context.
 * The mean loss of the last epoch and the steps taken are read with ofks_train_info.
 * Errors: OFKS_ESTATE (no network), OFKS_EINVAL (missing, empty or mismatched file, epochs < 1),
 * OFKS_ENOMEM, OFKS_ECUDA. */
int ofks_train_precond(ofks_ctx *ctx, const char *pairs_path, int32_t epochs, uint64_t seed);

/* Mean loss over the last epoch of ofks_train_precond and the Adam steps it took (any pointer
 * may be NULL). */
int ofks_train_info(ofks_ctx *ctx, double *last_epoch_loss, int64_t *steps);

/* Checkpoint: X, X_prev, D_prev, G_prev, eta, k, kkt0 and the Hartree warm start U, restored
 * exactly on load, so a reloaded run continues from the same state (later iterates agree up to
 * the order of the device's floating-point atomics).  The mesh, nuclei and params must match
 * on load.  Errors: OFKS_EINVAL (path cannot be opened, or the file does not match the context's
 * sizes or its own header's history length), OFKS_ENOMEM (host buffers), OFKS_ESTATE (no
 * orbitals to save), OFKS_ECUDA. */
int ofks_save_state(ofks_ctx *ctx, const char *path);
int ofks_load_state(ofks_ctx *ctx, const char *path);

/* Per-kernel device time accumulated while profiling is on (CUDA events around each
 * launch of the named kernel family).  on = 1 starts (and clears), 0 stops.  While it is on
 * the CUDA graphs are not used (every launch runs on its own between its events). */
int ofks_profile(ofks_ctx *ctx, int32_t on);
/* kernel family id -> launches and total milliseconds since profiling was switched on;
 * name (may be NULL) receives a static string. */
int ofks_profile_get(ofks_ctx *ctx, int32_t id, int64_t *launches, double *ms,
                     const char **name);

#ifdef __cplusplus
}
#endif
#endif /* OFKS_H */
