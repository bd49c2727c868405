// Internal state and launcher prototypes of libofks (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
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

// Capacity (doubles) of the grid_accumulate partials: K block totals per block of a grid.
constexpr int64_t GACC_CAP = 1 << 20;
// Least capacity (doubles) of the per-column partials: the Grams' split tiles need up to
// (608 + 16) units x 2 x 64 x 64.
constexpr int64_t CPART_MIN = 6 << 20;

// Rows of the per-column scalar array ctx->d_colA (each ld float64 long).
enum { CB_SHIFT = 0, CB_ACTIVE = 1, CB_RZ = 2, CB_RZN = 3, CB_PQ = 4, CB_BETA = 5, CB_NORM = 6,
       CB_ALPHA = 7, CB_ACC = 8, CB_WARM = 9, CB_COUNT = 10 };

// Kernel families timed by ofks_profile.
enum {
    PF_DENSITY = 0, PF_POISSON, PF_POTENTIAL, PF_SPMM_H, PF_GRAM, PF_SMALL, PF_GRAD,
    PF_PCG_SPMM, PF_PCG_UPDATE, PF_BB, PF_STEP, PF_SPMM_B, PF_OTHER, PF_POISSON_SPMV, PF_GCN, PF_POISSON_VEC, PF_POISSON_PC,
    PF_PCG_SEP, PF_JUDGE, PF_COUNT
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

// n x ld blocks of one precision.  X, D and G are ping-pong pairs (current / previous iterate).
template <class T>
struct Blocks {
    T *X[2] = {nullptr, nullptr}, *D[2] = {nullptr, nullptr}, *G[2] = {nullptr, nullptr};
    T *HX = nullptr, *BX = nullptr;
    T *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *W = nullptr;   // PCG block, W = 1/diag
    T *Dc = nullptr;                                       // PCG result on the active columns only
    T *valL = nullptr, *valB = nullptr, *valH = nullptr;   // SELL values (float set only; the
                                                           // float64 values are d_valL/B/H)
};

// learned preconditioner (network parameters, optimizer moments, activations)
struct GcnState {
    int H = 0;                                   // hidden width (0: not initialized)
    float *w = nullptr, *m = nullptr, *v = nullptr;   // parameters and Adam moments (float32)
    double *grad = nullptr;                      // parameter gradients (float64 accumulation)
    float *valA = nullptr, *valAT = nullptr;     // mean aggregation A and A^T on the SELL pattern
    int64_t rows = 0;                            // n * p the activations are sized for
    float *F = nullptr, *H1 = nullptr, *H2 = nullptr, *Z1 = nullptr, *Z2 = nullptr, *AH = nullptr;
    float *y = nullptr, *scale = nullptr, *Dn = nullptr, *Ds = nullptr;
    float *dA = nullptr, *dB2 = nullptr, *G32 = nullptr;
    double *stats = nullptr, *lacc = nullptr;
    float *valL32 = nullptr, *valB32 = nullptr;  // float32 L and B on the SELL pattern (energy loss)
    float *colf = nullptr;                       // per-column scale, mean log-diagonal and shift (float32)
    int64_t t = 0;                               // Adam step count
    int cols = 0;                                // columns of the next application (0: all p)
};

// Lattice-stencil form of the full-node stiffness (stencil.cu).  Node type t = parity triple
// of the lattice coordinates; the type's values are nown arrays of n doubles from val + base.
constexpr int ST_MAXE = 125;                     // offsets in [-2, 2]^3
struct StencilType {
    int64_t base, n;                             // first stored value, nodes of the type
    int nx, ny, nz, px, py, pz;                  // sub-lattice extents and parities
    int nown, nent, blk0, pad;                   // stored slots, all entries, first SpMV block
};
struct StencilEntry {
    int lin;                                     // id offset of the neighbour
    int8_t oa, ob, oc, tp;                       // lattice offset; source type (-1: own slot)
    int slot;                                    // slot in the source type
};
struct Stencil {
    bool on = false;
    int Lx = 0, Ly = 0, Lz = 0, blocks = 0;
    int64_t len = 0, rows = 0;                   // stored values, rows the SpMV computes
    double *val = nullptr;
    float2 *valff = nullptr;                     // val as float32 pairs (float-float SpMV)
    StencilType *d_type = nullptr;
    StencilEntry *d_ent = nullptr;               // 8 x ST_MAXE
    int *d_slot = nullptr;                       // 8 x 125 offset code -> own slot or -1
};

// Separable (fast-diagonalization) preconditioner of the Hartree CG (separable.cu)
struct SepState {
    bool on = false;
    int n[3] = {0, 0, 0};                        // interior lattice extents
    float *S[3] = {nullptr, nullptr, nullptr};   // per-axis modes S[a][i] (n x n)
    float *St[3] = {nullptr, nullptr, nullptr};  // their transposes
    float *lx = nullptr, *lyz = nullptr;         // lam_x (nx), lam_y + lam_z (ny x nz)
    float *t0 = nullptr, *t1 = nullptr;          // interior tensors
    bool tc = false;                             // tensor-core form available (every axis <= 256)
    __nv_bfloat16 *hS[3] = {nullptr, nullptr, nullptr}, *hSt[3] = {nullptr, nullptr, nullptr};  // bf16, padded
    __nv_bfloat16 *hbuf = nullptr;               // six padded bf16 tensors (input, intermediates)
    __nv_bfloat16 *hlo = nullptr;                // their low parts: value = hbuf + hlo (same layout)
    int64_t hoff[6] = {0, 0, 0, 0, 0, 0};
    __nv_bfloat16 *pbuf = nullptr;               // the same six tensors for pw PCG columns
    int64_t poff[6] = {0, 0, 0, 0, 0, 0};
    int pw = 0;
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
    int max_slice_w = 0;                         // widest slice (entries per row)
    // type-grouped SELL of L and B (float32 values) for the float32 PCG on lattice meshes.  Its
    // rows, and the rows of the PCG's chunk-major blocks, are the free nodes in type order: node
    // type (parity triple of the lattice coordinates) first, then lattice order, so slice s is
    // rows 32 s .. 32 s + 31 of one type along the third axis and its neighbours at one offset
    // are consecutive rows of another type.  d_tmap: type-ordered row -> free row (-1 past n),
    // d_tinv: free row -> type-ordered row; d_tcols holds type-ordered column ids
    int n_tslices = 0;
    int64_t tsell_len = 0;
    int *d_tslice_ptr = nullptr, *d_tslice_w = nullptr, *d_tcols = nullptr;
    int *d_tmap = nullptr, *d_tinv = nullptr;
    // row stride of the float32 PCG's chunk-major blocks: n rounded up to 32 (= 32 n_tslices)
    int64_t n_slots = 0;
    float *d_tvalL = nullptr, *d_tvalB = nullptr;
    double *d_valL = nullptr, *d_valB = nullptr, *d_valH = nullptr;
    double *d_dL = nullptr, *d_dB = nullptr;     // diagonals of L and B (free)
    // full-node stiffness for the Hartree Poisson problem (CSR)
    int64_t nnz_full = 0;
    int *d_fptr = nullptr, *d_fcol = nullptr;
    double *d_fval = nullptr, *d_minv = nullptr; // Jacobi inverse diagonal, 0 on the boundary
    Stencil st;                                  // lattice form of the same operator (if the mesh has one)
    SepState sep;                                // separable preconditioner (lattice meshes)
    // per tetrahedron
    int *d_tetf = nullptr;                       // T x 10 free ids (-1 on the boundary)
    int *d_tetn = nullptr;                       // T x 10 node ids
    int *d_hptr = nullptr, *d_hlist = nullptr;   // per SELL position, its element entries t 100 + 10 a + b
    int *d_nptr = nullptr, *d_nlist = nullptr;   // per node, its element entries t 10 + a
    double *d_wq = nullptr;                      // T: |T|/4
    double *d_yq = nullptr;                      // T x 4 x 3 quadrature points minus centre
    double *d_vext = nullptr;                    // T x 4
    int n_bnd = 0;
    int *d_bnd = nullptr;                        // boundary node ids
    double *d_bxyz = nullptr;                    // n_bnd x 3 boundary node coords minus centre
    double *d_ynode = nullptr;                   // N x 3 node positions minus centre (edge nodes at the
                                                 // midpoints of their edges): the multipole moments
    double center[3] = {0, 0, 0};
    std::vector<AmgLevel> amg;                   // Hartree preconditioner (empty: Jacobi)
    int *d_amg_idx = nullptr;                    // interior node ids (level 0 numbering)
    double *d_amg_chol = nullptr;                // dense inverse of the coarsest operator
    int64_t amg_ni = 0, amg_nc = 0;
    bool amg_lat = false;                        // geometric lattice hierarchy, level 0 on the stencil form
    bool amg_tried = false;                      // the hierarchy was built (or failed) for this mesh
    std::vector<int> h_tetn;                     // host copies for building it on first use
    std::vector<double> h_xyz;
    double e_nuc = 0.0;
    bool have_nuclei = false;

    // ---- quadrature and Hartree fields
    double *d_rho = nullptr, *d_vh = nullptr, *d_vxc = nullptr, *d_exc = nullptr;
    double *d_ve = nullptr;                      // T x 4 weighted potentials w V_q (float32 or float64)
    double *d_U = nullptr, *d_rhs = nullptr, *d_cr = nullptr, *d_cz = nullptr, *d_cp = nullptr,
           *d_cq = nullptr;
    float2 *d_cpff = nullptr;                    // the CG direction p as float32 pairs

    // ---- blocks n x ld: float64 set (plain form, refinement sweep) and float32 set (mixed form)
    int p = 0, ld = 0;
    Blocks<double> b64;
    Blocks<float> b32;
    int phase = 64;                              // 64: float64 iterations, 32: float32 iterations
    bool mixed_alloc = false;                    // the float32 set is allocated
    int switch_k = -1;                           // iteration at which float32 handed over to float64
    int cur = 0;                                 // index of the current X/D/G buffers
    // ---- small p x p (device)
    double *d_L0 = nullptr, *d_S = nullptr, *d_Lam = nullptr, *d_C = nullptr;
    double *d_colA = nullptr;                    // 4 x p column accumulators
    double *d_pp = nullptr;                      // p x p scratch (factorizations)
    double *d_stage = nullptr;                   // n x p dense staging of host block copies (ld > p)
    double *d_colC = nullptr;                    // per-column PCG arrays of the compact form (stride w)
    int *d_cmap = nullptr;                       // compact form: active column ids [ld], compact index [ld]
    int *d_gmap = nullptr;                       // learned preconditioner: active column ids [ld]
    double *d_sc = nullptr;                      // SC_COUNT scalars
    double *d_rec = nullptr;                     // iteration record (device)
    int *d_flag = nullptr;                       // error / status flags
    // deterministic reductions (common.cuh): grid_accumulate partials (GACC_CAP doubles) and its
    // block counter; per-column partials [column][unit] of the block kernels (cpart_cap doubles)
    double *d_gpart = nullptr;
    unsigned *d_gcount = nullptr;
    double *d_cpart = nullptr;
    int64_t cpart_cap = 0;
    int64_t pq_units = 0, rz_units = 0;          // partial units of the last PCG apply / vector update
    double best_rel = 1.0;                       // float32 phase: best (kkt + fea)/kkt0 so far ...
    int best_k = 0;                              // ... and the iteration that reached it
    double train_loss = 0.0;                     // mean loss of the last epoch of ofks_train_precond
    int64_t train_steps = 0;                     // Adam steps taken by ofks_train_precond
    double *nuclei_stage = nullptr;              // device address of the no-allocation nuclei staging array

    // ---- iteration state (host mirror)
    bool have_X = false, evaluated = false, have_prev = false;
    bool bx_valid = false;                       // d_BX holds B X for the current iterate
    int k = 0;
    int cg_last = 0;                             // CG iterations of the last Hartree solve
    double cg_rate = 0.0;                        // per-iteration factor of the squared Hartree CG residual
                                                 // observed in the last solve (0: none yet)
    double hartree_tol = 0.0;                    // > 0: tolerance of the next Hartree solve (adaptive mode)
    bool hartree_ff = false;                     // this Hartree solve keeps p as float32 pairs (d_cpff) too
    int64_t cg_total = 0;                        // ... summed since the counter was cleared
    double kkt0 = 0.0, eta = 0.0;
    bool converged = false;
    double last_E = 0, last_kkt = 0, last_fea = 0;
    std::vector<double> history;                 // rows of 6
    // CUDA graphs of fixed launch sequences (the PCG loop, Hartree CG chunks), keyed by what
    // shapes the sequence: replayed instead of relaunching its kernels one by one
    struct GraphEntry { std::vector<int64_t> key; cudaGraphExec_t exec; int64_t kernels; };
    std::vector<GraphEntry> graphs;
    double t_start = 0.0;
    double t_accum = 0.0;

    GcnState gcn;
    std::vector<int> row_deg;                    // pattern row lengths of the free matrices
    double *d_shift_in = nullptr;                // p shifts for ofks_precondition / training calls
    int64_t judge_accept = 0, judge_total = 0;   // learned preconditioner: columns accepted / judged
    int64_t learned_calls = 0, learned_warm = 0; // network applications; rejected columns started from them
    int gcn_skip = 0, gcn_backoff = 0;           // calls the network still sits out; length of the last pause
    int last_active = 0;                         // columns with T != I at the last direction
    int64_t active_total = 0;
    int64_t pcg_cols_total = 0;                  // PCG block width summed over the operator applies

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

// Runs `body` (kernel launches on c->stream only, no host synchronisation) through the context's
// graph for `key`: captured on first use, replayed afterwards; the kernel count of the sequence is
// added each time.  Without graphs (profiling on, cuda_graphs = 0, or a capture that fails) body
// runs directly.  Defined in api.cu.
int run_graph(ofks_ctx *c, const std::vector<int64_t> &key, void (*body)(void *), void *arg);
void clear_graphs(ofks_ctx *c);

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
cudaError_t static_stage_lookup(ofks_ctx *c);
void free_mesh(ofks_ctx *c);


// ---- stencil.cu (lattice form of the Hartree stiffness)
int stencil_setup(ofks_ctx *c, int64_t N, const double *xyz, const int64_t *fptr, const int *fcol,
                  const uint8_t *dirichlet);
void stencil_fill(ofks_ctx *c);
void stencil_free(ofks_ctx *c);
void launch_stencil_spmv(ofks_ctx *c, const double *p, double *q, double *sc, int it);
// the same in float-float arithmetic from p as float32 pairs (pf); pq += p.q in float64
void launch_stencil_spmv_ff(ofks_ctx *c, const float2 *pf, const double *p, double *q, double *sc, int it);
void launch_stencil_residual(ofks_ctx *c, const double *x, const double *b, double *r);     // r = b - L x
void launch_stencil_jacobi(ofks_ctx *c, const double *x, const double *b, double w, double *y); // y = x + w minv (b - L x)

// ---- separable.cu (fast-diagonalization preconditioner of the Hartree CG)
int sep_setup(ofks_ctx *c, const double *xyz, const uint8_t *dirichlet);
void sep_cg_step(ofks_ctx *c, int it, int slot, int first);    // fused CG update + z = A_sep^-1 r + r.z
void sep_free(ofks_ctx *c);
bool sep_pcg_ready(ofks_ctx *c, int w);                        // separable PCG buffers for width w
void sep_pcg_passes(ofks_ctx *c, int w, const double *shift);  // z = T_sep^-1 r on the PCG tensor

// ---- fields.cu (density, potentials, Hamiltonian refresh, Poisson)
int hartree_pc(ofks_ctx *c);                    // OFKS_HPC_* the next Hartree solve uses (builds the
                                                // multigrid hierarchy on first request)
template <class T> int launch_density(ofks_ctx *c, const T *X);
int run_hartree(ofks_ctx *c);
template <class T> int launch_potential_refresh(ofks_ctx *c, T *valH, const T *valL);

// ---- amg.cu (Hartree preconditioner)
int amg_setup(ofks_ctx *c, const int *tetn, int64_t T, const double *xyz);
void amg_free(ofks_ctx *c);
void amg_apply(ofks_ctx *c, const double *r_full, double *z_full);

// ---- spmm.cu (T = double or float)
template <class T> void launch_sell_spmm(ofks_ctx *c, const T *val, const T *X, T *Y);
template <class T> void launch_sell_spmm_ld(ofks_ctx *c, const T *val, const T *X, T *Y, int ld);
template <class T> void launch_sell_spmm_colnorm(ofks_ctx *c, const T *val, const T *X, T *Y, double *colsum);
// the PCG operator apply on a block of width w with pc real columns (w = ld, pc = p: all columns)
template <class T>
void launch_pcg_apply(ofks_ctx *c, const T *valL, const T *valB, const T *Zin, int zc, T *P, T *Q, const double *beta_col,
                      const double *shift, double *pq, int first, int w, int pc);

// ---- block.cu (tall-skinny products and vector updates)
template <class T> void launch_gram2(ofks_ctx *c, const T *X, const T *A, const T *B, double *XA, double *XB);
// gram_tc.cu: the float32 Grams on the tensor cores (false: shapes not supported)
// partials of X^T A and X^T B per CTA into part (entry-major, *units CTAs), added by k_gram_fin
bool launch_gram_tc(ofks_ctx *c, const float *X, const float *A, const float *B, double *part, int64_t *units);
// grad_tc.cu: G = H X + B X C and |H X - B X Lambda0|^2 on the tensor cores (false: not supported)
bool launch_grad_tc(ofks_ctx *c, const float *HX, const float *BX, float *G, double *kkt2);
template <class T> void launch_grad_update(ofks_ctx *c, Blocks<T> &b);
// The PCG's working set: its block width w (row pitch of R, Z, P, Q, W and of the D it builds,
// and the stride of its per-column arrays cb) and its real column count pc.  In the compact
// form the columns are the active ones only: compact column k < pc is column cmap[k] of G, and
// cpos[j] is the compact index of column j (-1: inactive, D = G).
template <class T>
struct PcgView {
    int w = 0, pc = 0;
    double *cb = nullptr;
    const int *cmap = nullptr, *cpos = nullptr;
    T *D = nullptr;
};
// float32 PCG blocks (W, R, Z, P, Q and the D they build) chunk-major (4 columns per chunk, row
// stride n_slots) on lattice meshes with w a multiple of 4; the D of such a PCG is always
// v.D = Dc and comes back through launch_direction_expand
template <class T> bool pcg_zc(const ofks_ctx *c, int w);
// warm: the columns flagged in the view's CB_WARM row start from the natural-layout D (with
// T D in Q) instead of zero
template <class T> void launch_pcg_init(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v, bool warm = false);
// last: the final iteration, after which only D is read
template <class T> void launch_pcg_update(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v, bool last);
template <class T> void launch_judge(ofks_ctx *c, Blocks<T> &b);
// Z = T_sep^-1 R (separable preconditioner of the PCG, float32 chunk-major blocks on lattice
// meshes) with the rz partials; false when that form does not apply
template <class T> bool launch_pcg_sep(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v);
bool pcg_sep_active(ofks_ctx *c, int w);
template <class T> void launch_direction_select(ofks_ctx *c, Blocks<T> &b);
// D = the compact PCG result on the active columns, G on the others
template <class T> void launch_direction_expand(ofks_ctx *c, Blocks<T> &b, const PcgView<T> &v);
template <class T> void launch_bb_dots(ofks_ctx *c, Blocks<T> &b, bool raw);
template <class T> void launch_step_y(ofks_ctx *c, Blocks<T> &b, T *Y);
template <class T> void launch_scale_cols(ofks_ctx *c, T *Y, T *BY, const double *colsum);
template <class T> void launch_block_times_small(ofks_ctx *c, const T *X, const double *M, T *Y);
template <class S, class T> void launch_convert(ofks_ctx *c, const S *src, T *dst, int64_t count);
// dst[r dp + j] = src[r sp + j] for r < n, j < w (float64)
void launch_repack(ofks_ctx *c, const double *src, int64_t sp, double *dst, int64_t dp, int64_t n, int w);
// the float32 block (n x ld, padding columns zero) from a dense n x p float64 copy, and back
void launch_unpack_f32(ofks_ctx *c, const double *src, float *dst);
void launch_pack_f32(ofks_ctx *c, const float *src, double *dst);

// ---- small.cu (p x p work on one CTA)
void launch_small_update(ofks_ctx *c);
void launch_small_record(ofks_ctx *c);
void launch_eta(ofks_ctx *c);
void launch_pcg_alpha(ofks_ctx *c, int w, int pc, double *cb);
void launch_pcg_beta(ofks_ctx *c, int w, int pc, double *cb);
// out[j] (j < ktot) = fixed-order sum of part[j * units + u] over u for j < kact, else 0
void launch_col_fin(ofks_ctx *c, int kact, int ktot, int64_t units, const double *part, double *out);
// the compact form's per-column arrays: shift of the active columns, everything else zero
void launch_pcg_compact_cols(ofks_ctx *c, int w, int nact, const int *cmap, double *colC);
void launch_cholesky_inv(ofks_ctx *c, const double *S, double *Rinv);
void launch_rayleigh_ritz(ofks_ctx *c, const double *A, const double *S, double *eigs, double *V);

// ---- gcn.cu (learned preconditioner)
int64_t gcn_param_count(int H);
int gcn_setup(ofks_ctx *c, int H, uint64_t seed, const std::vector<int> &deg);
void gcn_free(ofks_ctx *c);
int gcn_forward_prepare(ofks_ctx *c);
int gcn_forward(ofks_ctx *c, const double *shift, bool keep);
int gcn_backward(ofks_ctx *c, const double *shift, double *loss);
int gcn_adam(ofks_ctx *c, double lr);
void launch_dense_tc(ofks_ctx *c, int64_t rows, const float *H, const float *AH, const float *W, const float *U,
                     const float *b, float *out, const float *w2 = nullptr, const float *u2 = nullptr,
                     float *a = nullptr, float *q = nullptr);
void launch_dense_tc_bf16(ofks_ctx *c, int64_t rows, const __nv_bfloat16 *H, const __nv_bfloat16 *AH, const float *W,
                          const float *U, const float *b, const float *w2, const float *u2, float *a, float *q);
// the network's block: column k is column cmap[k] of the n x ld block (cmap NULL: k), for the
// gcn.cols columns the next application works on (0: all p)
template <class E> void gcn_pack(ofks_ctx *c, const E *src, float *dst, const int *cmap = nullptr);
template <class E> void gcn_unpack(ofks_ctx *c, const float *src, E *dst, const int *cmap = nullptr);
inline int gcn_cols(const ofks_ctx *c);

// columns the learned preconditioner's network works on (its activations are sized for p)
inline int gcn_cols(const ofks_ctx *c) { return c->gcn.cols > 0 ? c->gcn.cols : c->p; }
