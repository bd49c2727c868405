// Multigrid preconditioner for the Hartree Poisson system L_II U_I = f_I (paper Sec. 2.2 solves
// this system by multigrid).  Level 0 -> 1 is the geometric P2 -> P1 interpolation on the same
// mesh (vertex values copied, an edge midpoint takes the mean of its two vertices), so level 1
// is the P1 stiffness.  Below that:
//   * lattice meshes (node ids on a lattice whose faces are the Dirichlet boundary): geometric
//     coarsening of the vertex lattice, every other coordinate per axis, with per-axis linear
//     interpolation in the actual (graded) coordinates and Galerkin operators A_c = P^T A P;
//     level 0 smooths and forms residuals with the lattice-stencil kernels on full-node vectors;
//   * other meshes: smoothed aggregation, P = (I - w D^-1 A) T.
// The hierarchy is built once per mesh on the host (Galerkin products, dense Cholesky inverse of
// the coarsest operator); every V-cycle runs in the kernels below and preconditions the CG.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int COARSE_MAX = 512;      // coarsest level solved densely
constexpr int MAX_LEVELS = 12;
constexpr double STRENGTH = 0.08;    // |a_ij| >= theta sqrt(|a_ii a_jj|) is a strong connection
constexpr int SWEEPS0 = 2;           // damped Jacobi sweeps before and after the coarse correction on level 0
constexpr int SWEEPS = 2;            // ... on the coarser levels

struct Csr {
    int64_t n = 0, m = 0;            // rows, columns
    std::vector<int64_t> ptr;
    std::vector<int> col;
    std::vector<double> val;
};

void par_for(int64_t n, const std::function<void(int64_t, int64_t)> &f) {
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    if (n < 50000) nt = 1;
    if (nt == 1) { f(0, n); return; }
    std::vector<std::thread> th;
    const int64_t ch = (n + nt - 1) / nt;
    for (unsigned i = 0; i < nt; ++i) {
        const int64_t a = i * ch, b = std::min<int64_t>(n, a + ch);
        if (a < b) th.emplace_back(f, a, b);
    }
    for (auto &t : th) t.join();
}

double diag_of(const Csr &A, int64_t i) {
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
        if (A.col[k] == i) return A.val[k];
    return 0.0;
}

// rho(D^-1 A) by power iteration from a fixed start vector
double spectral_radius(const Csr &A, const std::vector<double> &dinv) {
    std::vector<double> x(A.n), y(A.n);
    for (int64_t i = 0; i < A.n; ++i) x[i] = 1.0 + 0.5 * std::sin(0.37 * (double)i);
    double lam = 1.0;
    for (int it = 0; it < 20; ++it) {
        par_for(A.n, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; ++i) {
                double s = 0.0;
                for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
                y[i] = dinv[i] * s;
            }
        });
        double nx = 0.0, ny = 0.0;
        for (int64_t i = 0; i < A.n; ++i) { nx += x[i] * x[i]; ny += y[i] * y[i]; }
        lam = std::sqrt(ny / nx);
        const double s = 1.0 / std::sqrt(ny);
        for (int64_t i = 0; i < A.n; ++i) x[i] = y[i] * s;
    }
    return 1.1 * lam;
}

// standard three-pass aggregation on the strong-connection graph; returns #aggregates
int64_t aggregate(const Csr &A, std::vector<int> &agg) {
    const int64_t n = A.n;
    std::vector<double> d(n);
    for (int64_t i = 0; i < n; ++i) d[i] = std::fabs(diag_of(A, i));
    auto strong = [&](int64_t i, int64_t k) {
        const int j = A.col[k];
        return j != i && std::fabs(A.val[k]) >= STRENGTH * std::sqrt(d[i] * d[j]);
    };
    agg.assign(n, -1);
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {                      // pass 1: free neighbourhoods
        if (agg[i] >= 0) continue;
        bool ok = true;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1] && ok; ++k)
            if (strong(i, k) && agg[A.col[k]] >= 0) ok = false;
        if (!ok) continue;
        agg[i] = (int)na;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (strong(i, k)) agg[A.col[k]] = (int)na;
        ++na;
    }
    std::vector<int> pass1(agg);
    for (int64_t i = 0; i < n; ++i) {                      // pass 2: join a strong neighbour's aggregate
        if (agg[i] >= 0) continue;
        double best = -1.0;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (strong(i, k) && pass1[A.col[k]] >= 0 && std::fabs(A.val[k]) > best) {
                best = std::fabs(A.val[k]);
                agg[i] = pass1[A.col[k]];
            }
    }
    for (int64_t i = 0; i < n; ++i) {                      // pass 3: leftovers with their free neighbours
        if (agg[i] >= 0) continue;
        agg[i] = (int)na;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (strong(i, k) && agg[A.col[k]] < 0) agg[A.col[k]] = (int)na;
        ++na;
    }
    return na;
}

// row-wise sparse product C = A B with a dense marker per thread
Csr spgemm(const Csr &A, const Csr &B) {
    Csr C;
    C.n = A.n; C.m = B.m;
    C.ptr.assign(A.n + 1, 0);
    std::vector<std::vector<int>> cols(A.n);
    std::vector<std::vector<double>> vals(A.n);
    par_for(A.n, [&](int64_t a, int64_t b) {
        std::vector<int> mark(B.m, -1);
        std::vector<int> lst;
        std::vector<double> acc;
        for (int64_t i = a; i < b; ++i) {
            lst.clear(); acc.clear();
            for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                const int r = A.col[k];
                const double av = A.val[k];
                for (int64_t q = B.ptr[r]; q < B.ptr[r + 1]; ++q) {
                    const int c = B.col[q];
                    if (mark[c] < 0) { mark[c] = (int)lst.size(); lst.push_back(c); acc.push_back(0.0); }
                    acc[mark[c]] += av * B.val[q];
                }
            }
            std::vector<int> order(lst.size());
            for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
            std::sort(order.begin(), order.end(), [&](int x, int y) { return lst[x] < lst[y]; });
            cols[i].resize(lst.size());
            vals[i].resize(lst.size());
            for (size_t t = 0; t < order.size(); ++t) { cols[i][t] = lst[order[t]]; vals[i][t] = acc[order[t]]; }
            for (int c : lst) mark[c] = -1;
        }
    });
    for (int64_t i = 0; i < A.n; ++i) C.ptr[i + 1] = C.ptr[i] + (int64_t)cols[i].size();
    C.col.resize(C.ptr[A.n]);
    C.val.resize(C.ptr[A.n]);
    for (int64_t i = 0; i < A.n; ++i) {
        std::copy(cols[i].begin(), cols[i].end(), C.col.begin() + C.ptr[i]);
        std::copy(vals[i].begin(), vals[i].end(), C.val.begin() + C.ptr[i]);
    }
    return C;
}

Csr transpose(const Csr &A) {
    Csr T;
    T.n = A.m; T.m = A.n;
    T.ptr.assign(A.m + 1, 0);
    for (int64_t k = 0; k < A.ptr[A.n]; ++k) T.ptr[A.col[k] + 1]++;
    for (int64_t i = 0; i < A.m; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.ptr[A.n]);
    T.val.resize(A.ptr[A.n]);
    std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int64_t o = fill[A.col[k]]++;
            T.col[o] = (int)i;
            T.val[o] = A.val[k];
        }
    return T;
}

// ------------------------------------------------------------------------- device kernels
// y = A x (mode 0), y = b - A x (mode 1), y = x + w D^-1 (b - A x) (mode 2), y += A x (mode 3);
// 8 lanes per row
template <int MODE>
__global__ void __launch_bounds__(256) k_csr(int64_t n, const int *__restrict__ ptr, const int *__restrict__ col,
                                             const double *__restrict__ val, const double *__restrict__ x,
                                             const double *__restrict__ b, const double *__restrict__ dinv,
                                             double w, double *y) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
    const int lane = threadIdx.x & 7;
    double s = 0.0;
    if (row < n)
        for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 8) s = fma(val[k], x[col[k]], s);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 8);
    if (row >= n || lane != 0) return;
    if (MODE == 0) y[row] = s;
    else if (MODE == 1) y[row] = b[row] - s;
    else if (MODE == 2) y[row] = x[row] + w * dinv[row] * (b[row] - s);
    else y[row] += s;
}

__global__ void k_scaled(int64_t n, const double *__restrict__ b, const double *__restrict__ dinv, double w,
                         double *x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = w * dinv[i] * b[i];
}

__global__ void k_gather(int64_t n, const int *__restrict__ idx, const double *__restrict__ full, double *part) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) part[i] = full[idx[i]];
}

__global__ void k_scatter(int64_t n, const int *__restrict__ idx, const double *__restrict__ part, double *full) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) full[idx[i]] = part[i];
}

// x = Ainv b for the dense inverse of the coarsest operator (row-major n x n), a warp per row
__global__ void __launch_bounds__(256) k_coarse_solve(int n, const double *__restrict__ Ainv,
                                                       const double *__restrict__ b, double *x) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s = fma(Ainv[(int64_t)row * n + k], b[k], s);
    s = warp_sum(s);
    if (lane == 0) x[row] = s;
}

template <class T>
int up(ofks_ctx *c, T **d, const T *h, size_t cnt) {
    if (cudaMalloc((void **)d, sizeof(T) * std::max<size_t>(cnt, 1)) != cudaSuccess)
        return ofks_fail(c, OFKS_ENOMEM, "AMG: device allocation failed");
    if (cnt && cudaMemcpy(*d, h, sizeof(T) * cnt, cudaMemcpyHostToDevice) != cudaSuccess)
        return ofks_fail(c, OFKS_ECUDA, "AMG: upload failed");
    return OFKS_OK;
}

int up_csr(ofks_ctx *c, const Csr &A, AmgMat &M) {
    std::vector<int> p32(A.n + 1);
    for (int64_t i = 0; i <= A.n; ++i) p32[i] = (int)A.ptr[i];
    M.n = A.n; M.m = A.m;
    int rc;
    if ((rc = up(c, &M.ptr, p32.data(), p32.size())) || (rc = up(c, &M.col, A.col.data(), A.col.size())) ||
        (rc = up(c, &M.val, A.val.data(), A.val.size())))
        return rc;
    return OFKS_OK;
}

void free_csr(AmgMat &M) {
    if (M.ptr) cudaFree(M.ptr);
    if (M.col) cudaFree(M.col);
    if (M.val) cudaFree(M.val);
    M = AmgMat{};
}

inline unsigned g8(int64_t n) { return (unsigned)((n * 8 + 255) / 256); }
inline unsigned g1(int64_t n) { return (unsigned)((n + 255) / 256); }

// One axis of a lattice level: coordinates (boundary included) and the interpolation of every
// fine index from the coarse indices {0, 2, 4, ...} plus the last one; axes of 3 or fewer
// points are not coarsened.
struct AxisMap {
    std::vector<double> xc;                       // coarse coordinates
    std::vector<int> c0, c1;                      // coarse neighbours of fine index i (c1 = -1: copy)
    std::vector<double> w0, w1;
};

AxisMap coarsen_axis(const std::vector<double> &x) {
    const int n = (int)x.size();
    AxisMap M;
    M.c0.assign(n, -1); M.c1.assign(n, -1); M.w0.assign(n, 0.0); M.w1.assign(n, 0.0);
    std::vector<int> cidx(n, -1);
    if (n <= 3) {
        for (int i = 0; i < n; ++i) { cidx[i] = i; M.xc.push_back(x[i]); }
    } else {
        for (int i = 0; i < n; i += 2) { cidx[i] = (int)M.xc.size(); M.xc.push_back(x[i]); }
        if (cidx[n - 1] < 0) { cidx[n - 1] = (int)M.xc.size(); M.xc.push_back(x[n - 1]); }
    }
    for (int i = 0; i < n; ++i) {
        if (cidx[i] >= 0) { M.c0[i] = cidx[i]; M.w0[i] = 1.0; continue; }
        const double t = (x[i] - x[i - 1]) / (x[i + 1] - x[i - 1]);
        M.c0[i] = cidx[i - 1]; M.w0[i] = 1.0 - t;
        M.c1[i] = cidx[i + 1]; M.w1[i] = t;
    }
    return M;
}

// Tensor-product interpolation from the interior of the coarse lattice to the interior of the
// fine one (both numbered lexicographically over interior points; boundary values are zero).
Csr lattice_prolongator(const AxisMap ax[3], const int nf[3]) {
    int nc[3];
    for (int d = 0; d < 3; ++d) nc[d] = (int)ax[d].xc.size();
    const int64_t fi[3] = {nf[0] - 2, nf[1] - 2, nf[2] - 2}, ci[3] = {nc[0] - 2, nc[1] - 2, nc[2] - 2};
    Csr P;
    P.n = fi[0] * fi[1] * fi[2];
    P.m = ci[0] * ci[1] * ci[2];
    P.ptr.assign(P.n + 1, 0);
    auto terms = [&](int d, int i, int *cc, double *ww) {
        int k = 0;
        const int c0 = ax[d].c0[i], c1 = ax[d].c1[i];
        if (c0 > 0 && c0 < nc[d] - 1) { cc[k] = c0 - 1; ww[k++] = ax[d].w0[i]; }
        if (c1 > 0 && c1 < nc[d] - 1) { cc[k] = c1 - 1; ww[k++] = ax[d].w1[i]; }
        return k;
    };
    for (int a = 1; a < nf[0] - 1; ++a)
        for (int b = 1; b < nf[1] - 1; ++b)
            for (int cz = 1; cz < nf[2] - 1; ++cz) {
                int ca[2], cb[2], cc[2];
                double wa[2], wb[2], wc[2];
                const int na = terms(0, a, ca, wa), nb = terms(1, b, cb, wb), ncz = terms(2, cz, cc, wc);
                std::vector<std::pair<int, double>> row;
                for (int i = 0; i < na; ++i)
                    for (int j = 0; j < nb; ++j)
                        for (int k = 0; k < ncz; ++k)
                            row.push_back({(int)(((int64_t)ca[i] * ci[1] + cb[j]) * ci[2] + cc[k]), wa[i] * wb[j] * wc[k]});
                std::sort(row.begin(), row.end());
                for (auto &e : row) { P.col.push_back(e.first); P.val.push_back(e.second); }
                const int64_t r = ((int64_t)(a - 1) * fi[1] + (b - 1)) * fi[2] + (cz - 1);
                P.ptr[r + 1] = (int64_t)P.col.size();
            }
    return P;
}

}  // namespace

void amg_free(ofks_ctx *c) {
    for (auto &L : c->amg) {
        free_csr(L.A); free_csr(L.P); free_csr(L.R);
        for (double *p : {L.dinv, L.x, L.x2, L.b, L.r}) if (p) cudaFree(p);
    }
    c->amg.clear();
    if (c->d_amg_chol) cudaFree(c->d_amg_chol);
    if (c->d_amg_idx) cudaFree(c->d_amg_idx);
    c->d_amg_chol = nullptr;
    c->d_amg_idx = nullptr;
    c->amg_nc = 0;
    c->amg_lat = false;
}

namespace {

// rows of P restricted to the interior nodes -> rows over all nodes (Dirichlet rows empty)
Csr expand_rows(const Csr &P, const std::vector<int> &iid, int64_t N) {
    Csr F;
    F.n = N; F.m = P.m;
    F.ptr.assign(N + 1, 0);
    for (int64_t r = 0; r < P.n; ++r) F.ptr[iid[r] + 1] = P.ptr[r + 1] - P.ptr[r];
    for (int64_t i = 0; i < N; ++i) F.ptr[i + 1] += F.ptr[i];
    F.col.resize(P.col.size());
    F.val.resize(P.val.size());
    for (int64_t r = 0; r < P.n; ++r) {
        const int64_t o = F.ptr[iid[r]];
        for (int64_t k = P.ptr[r]; k < P.ptr[r + 1]; ++k) {
            F.col[o + k - P.ptr[r]] = P.col[k];
            F.val[o + k - P.ptr[r]] = P.val[k];
        }
    }
    return F;
}

}  // namespace

int amg_setup(ofks_ctx *c, const int *tetn, int64_t T, const double *xyz) {
    amg_free(c);
    const int64_t N = c->n_nodes;
    std::vector<int> fptr(N + 1), fcol(c->nnz_full), interior(N);
    std::vector<double> fval(c->nnz_full), minv(N);
    cudaError_t e = cudaMemcpy(fptr.data(), c->d_fptr, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fcol.data(), c->d_fcol, sizeof(int) * c->nnz_full, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fval.data(), c->d_fval, sizeof(double) * c->nnz_full, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(minv.data(), c->d_minv, sizeof(double) * N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "AMG: download of the stiffness");
    std::vector<int> iid, inum(N, -1);
    for (int64_t i = 0; i < N; ++i)
        if (minv[i] != 0.0) { inum[i] = (int)iid.size(); iid.push_back((int)i); }
    Csr A;
    A.n = A.m = (int64_t)iid.size();
    A.ptr.assign(A.n + 1, 0);
    for (int64_t r = 0; r < A.n; ++r) {
        const int i = iid[r];
        for (int k = fptr[i]; k < fptr[i + 1]; ++k)
            if (inum[fcol[k]] >= 0) { A.col.push_back(inum[fcol[k]]); A.val.push_back(fval[k]); }
        A.ptr[r + 1] = (int64_t)A.col.size();
    }
    int rc;
    if ((rc = up(c, &c->d_amg_idx, iid.data(), iid.size()))) return rc;
    c->amg_ni = A.n;

    // lattice hierarchy: odd lattice extents (2 N + 1 per axis, the cell vertices at even
    // coordinates) and Dirichlet nodes exactly on the lattice faces
    const int Lx = c->st.Lx, Ly = c->st.Ly, Lz = c->st.Lz;
    bool lat = c->st.on && (Lx & 1) && (Ly & 1) && (Lz & 1) && Lx >= 5 && Ly >= 5 && Lz >= 5;
    for (int64_t i = 0; i < N && lat; ++i) {
        const int64_t a = i / ((int64_t)Ly * Lz), b = (i / Lz) % Ly, cz = i % Lz;
        const bool face = a == 0 || a == Lx - 1 || b == 0 || b == Ly - 1 || cz == 0 || cz == Lz - 1;
        if (face != (minv[i] == 0.0)) lat = false;
    }
    const int V[3] = {(Lx + 1) / 2, (Ly + 1) / 2, (Lz + 1) / 2};   // vertex lattice (lattice mode)

    // P2 -> P1 interpolation restricted to interior nodes; vertex unknowns numbered in tet order,
    // or lexicographically over the interior of the vertex lattice in lattice mode
    std::vector<int> vnum(N, -1), ea(N, -1), eb(N, -1);
    int64_t nv = 0;
    if (lat) {
        for (int i = 1; i < V[0] - 1; ++i)
            for (int j = 1; j < V[1] - 1; ++j)
                for (int k = 1; k < V[2] - 1; ++k)
                    vnum[((int64_t)(2 * i) * Ly + 2 * j) * Lz + 2 * k] = (int)nv++;
    } else {
        for (int64_t t = 0; t < T; ++t)
            for (int a = 0; a < 4; ++a) {
                const int v = tetn[t * 10 + a];
                if (inum[v] >= 0 && vnum[v] < 0) vnum[v] = (int)nv++;
            }
    }
    for (int64_t t = 0; t < T; ++t)
        for (int e = 0; e < 6; ++e) {
            int a, b;
            p2_edge(e, a, b);
            const int m = tetn[t * 10 + 4 + e];
            ea[m] = tetn[t * 10 + a];
            eb[m] = tetn[t * 10 + b];
        }
    Csr P1;
    P1.n = A.n; P1.m = nv;
    P1.ptr.assign(A.n + 1, 0);
    for (int64_t r = 0; r < A.n; ++r) {
        const int i = iid[r];
        if (vnum[i] >= 0) { P1.col.push_back(vnum[i]); P1.val.push_back(1.0); }
        else if (ea[i] >= 0) {
            const int va = vnum[ea[i]], vb = vnum[eb[i]];
            if (va >= 0 && vb >= 0) {
                P1.col.push_back(std::min(va, vb)); P1.val.push_back(0.5);
                P1.col.push_back(std::max(va, vb)); P1.val.push_back(0.5);
            } else if (va >= 0 || vb >= 0) {
                P1.col.push_back(va >= 0 ? va : vb); P1.val.push_back(0.5);
            }
        }
        P1.ptr[r + 1] = (int64_t)P1.col.size();
    }
    const bool geometric = nv > 0 && nv < A.n;
    lat = lat && geometric;
    // lattice mode: per-axis coordinates of the vertex lattice
    int dims[3] = {V[0], V[1], V[2]};
    std::vector<double> coord[3];
    if (lat) {
        for (int i = 0; i < V[0]; ++i) coord[0].push_back(xyz[3 * ((int64_t)(2 * i) * Ly * Lz)]);
        for (int j = 0; j < V[1]; ++j) coord[1].push_back(xyz[3 * ((int64_t)(2 * j) * Lz) + 1]);
        for (int k = 0; k < V[2]; ++k) coord[2].push_back(xyz[3 * (int64_t)(2 * k) + 2]);
    }
    const bool verbose = std::getenv("OFKS_VERBOSE") != nullptr;
    for (int lev = 0; lev < MAX_LEVELS; ++lev) {
        AmgLevel L;
        std::vector<double> dinv(A.n);
        for (int64_t i = 0; i < A.n; ++i) dinv[i] = 1.0 / diag_of(A, i);
        const double rho = spectral_radius(A, dinv);
        L.omega = 4.0 / (3.0 * rho);
        const bool on_stencil = lat && lev == 0;          // level 0 runs on the lattice stencil
        if (!on_stencil && ((rc = up_csr(c, A, L.A)) || (rc = up(c, &L.dinv, dinv.data(), dinv.size())))) return rc;
        if (on_stencil) { L.A.n = N; L.A.m = N; }
        bool last = A.n <= COARSE_MAX || lev == MAX_LEVELS - 1;
        if (!last && lev == 0 && geometric) {
            Csr R = transpose(P1);
            Csr AP = spgemm(A, P1);
            Csr Ac = spgemm(R, AP);
            if (verbose)
                std::fprintf(stderr, "[ofks mg] level 0 (P2->P1%s): n=%lld nnz(A)=%lld coarse n=%lld omega=%.4f\n",
                             lat ? ", lattice" : "", (long long)A.n, (long long)A.ptr[A.n], (long long)nv, L.omega);
            if (on_stencil) {
                Csr PF = expand_rows(P1, iid, N);
                Csr RF = transpose(PF);
                if ((rc = up_csr(c, PF, L.P)) || (rc = up_csr(c, RF, L.R))) return rc;
            } else if ((rc = up_csr(c, P1, L.P)) || (rc = up_csr(c, R, L.R))) {
                return rc;
            }
            c->amg.push_back(L);
            A = std::move(Ac);
            continue;
        }
        if (!last && lat) {
            if (dims[0] <= 3 && dims[1] <= 3 && dims[2] <= 3) last = true;
            if (!last) {
                AxisMap ax[3] = {coarsen_axis(coord[0]), coarsen_axis(coord[1]), coarsen_axis(coord[2])};
                Csr P = lattice_prolongator(ax, dims);
                if (P.n != A.n) return ofks_fail(c, OFKS_EINVAL, "MG: lattice level size mismatch");
                Csr R = transpose(P);
                Csr AP = spgemm(A, P);
                Csr Ac = spgemm(R, AP);
                if (verbose)
                    std::fprintf(stderr, "[ofks mg] level %d (lattice %dx%dx%d): n=%lld nnz(A)=%lld coarse n=%lld omega=%.4f\n",
                                 lev, dims[0], dims[1], dims[2], (long long)A.n, (long long)A.ptr[A.n],
                                 (long long)P.m, L.omega);
                if ((rc = up_csr(c, P, L.P)) || (rc = up_csr(c, R, L.R))) return rc;
                c->amg.push_back(L);
                A = std::move(Ac);
                for (int d = 0; d < 3; ++d) { coord[d] = ax[d].xc; dims[d] = (int)coord[d].size(); }
                continue;
            }
        }
        if (!last) {
            std::vector<int> agg;
            const int64_t na = aggregate(A, agg);
            if (na >= A.n) {                               // no coarsening possible: stop here
                c->amg.push_back(L);
                break;
            }
            std::vector<double> tw(na, 0.0);
            for (int64_t i = 0; i < A.n; ++i) tw[agg[i]] += 1.0;
            for (auto &t : tw) t = 1.0 / std::sqrt(t);
            Csr Tt;                                         // tentative prolongator
            Tt.n = A.n; Tt.m = na;
            Tt.ptr.resize(A.n + 1);
            Tt.col.resize(A.n);
            Tt.val.resize(A.n);
            for (int64_t i = 0; i < A.n; ++i) { Tt.ptr[i] = i; Tt.col[i] = agg[i]; Tt.val[i] = tw[agg[i]]; }
            Tt.ptr[A.n] = A.n;
            Csr S = A;                                      // S = I - w D^-1 A
            for (int64_t i = 0; i < A.n; ++i)
                for (int64_t k = S.ptr[i]; k < S.ptr[i + 1]; ++k)
                    S.val[k] = (S.col[k] == i ? 1.0 : 0.0) - L.omega * dinv[i] * A.val[k];
            Csr P = spgemm(S, Tt);
            Csr R = transpose(P);
            Csr AP = spgemm(A, P);
            Csr Ac = spgemm(R, AP);
            if (verbose)
                std::fprintf(stderr, "[ofks mg] level %d: n=%lld nnz(A)=%lld nnz(P)=%lld aggregates=%lld omega=%.4f\n",
                             lev, (long long)A.n, (long long)A.ptr[A.n], (long long)P.ptr[P.n], (long long)na, L.omega);
            if ((rc = up_csr(c, P, L.P)) || (rc = up_csr(c, R, L.R))) return rc;
            c->amg.push_back(L);
            A = std::move(Ac);
            continue;
        }
        c->amg.push_back(L);
        break;
    }
    // dense inverse of the coarsest operator through its Cholesky factor
    const int64_t nc = A.n;
    if (nc > 4096) return ofks_fail(c, OFKS_ENOTCONV, "AMG: coarsening stalled at %lld unknowns", (long long)nc);
    if (verbose) std::fprintf(stderr, "[ofks mg] coarsest: n=%lld (dense)\n", (long long)nc);
    std::vector<double> Lf((size_t)nc * nc, 0.0), Dm((size_t)nc * nc, 0.0);
    for (int64_t i = 0; i < nc; ++i)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) Lf[(size_t)i * nc + A.col[k]] = A.val[k];
    for (int64_t j = 0; j < nc; ++j) {
        double d = Lf[(size_t)j * nc + j];
        for (int64_t k = 0; k < j; ++k) d -= Lf[(size_t)j * nc + k] * Lf[(size_t)j * nc + k];
        if (!(d > 0.0)) return ofks_fail(c, OFKS_ENOTCONV, "AMG: coarsest operator is not positive definite");
        d = std::sqrt(d);
        Lf[(size_t)j * nc + j] = d;
        for (int64_t i = j + 1; i < nc; ++i) {
            double s = Lf[(size_t)i * nc + j];
            for (int64_t k = 0; k < j; ++k) s -= Lf[(size_t)i * nc + k] * Lf[(size_t)j * nc + k];
            Lf[(size_t)i * nc + j] = s / d;
        }
    }
    std::vector<double> y(nc);
    for (int64_t col = 0; col < nc; ++col) {               // column col of A^-1: L L^T x = e_col
        for (int64_t i = 0; i < nc; ++i) {
            double s = (i == col) ? 1.0 : 0.0;
            for (int64_t k = 0; k < i; ++k) s -= Lf[(size_t)i * nc + k] * y[k];
            y[i] = s / Lf[(size_t)i * nc + i];
        }
        for (int64_t i = nc - 1; i >= 0; --i) {
            double s = y[i];
            for (int64_t k = i + 1; k < nc; ++k) s -= Lf[(size_t)k * nc + i] * Dm[(size_t)k * nc + col];
            Dm[(size_t)i * nc + col] = s / Lf[(size_t)i * nc + i];
        }
    }
    if ((rc = up(c, &c->d_amg_chol, Dm.data(), Dm.size()))) return rc;
    c->amg_nc = nc;
    for (auto &L : c->amg) {
        const size_t bytes = sizeof(double) * std::max<int64_t>(L.A.n, 1);
        if (cudaMalloc((void **)&L.x, bytes) != cudaSuccess || cudaMalloc((void **)&L.x2, bytes) != cudaSuccess ||
            cudaMalloc((void **)&L.b, bytes) != cudaSuccess || cudaMalloc((void **)&L.r, bytes) != cudaSuccess)
            return ofks_fail(c, OFKS_ENOMEM, "AMG: level vectors");
        // full-node level-0 vectors keep zero Dirichlet entries: the stencil kernels never write them
        if (cudaMemset(L.x, 0, bytes) != cudaSuccess || cudaMemset(L.x2, 0, bytes) != cudaSuccess ||
            cudaMemset(L.r, 0, bytes) != cudaSuccess)
            return ofks_fail(c, OFKS_ECUDA, "AMG: level vectors");
    }
    c->amg_lat = lat;
    return OFKS_OK;
}

// x = M^-1 b on level l by one symmetric V(nu,nu) cycle; level l's b holds the right side and
// its x receives the result.  In lattice mode level 0 works on full-node vectors through the
// stencil kernels (b and x are then the caller's vectors, Dirichlet entries zero).
static void vcycle(ofks_ctx *c, size_t l, const double *b0 = nullptr, double *x0 = nullptr) {
    AmgLevel &L = c->amg[l];
    cudaStream_t s = c->stream;
    if (l + 1 == c->amg.size()) {
        k_coarse_solve<<<(unsigned)((c->amg_nc * 32 + 255) / 256), 256, 0, s>>>((int)c->amg_nc, c->d_amg_chol,
                                                                               L.b, L.x);
        c->kernels += 1;
        return;
    }
    const int64_t n = L.A.n;
    const int nu = l == 0 ? SWEEPS0 : SWEEPS;
    AmgLevel &C = c->amg[l + 1];
    if (l == 0 && c->amg_lat) {
        const double *b = b0;
        double *x = x0, *y = L.x2;
        k_scaled<<<g1(n), 256, 0, s>>>(n, b, c->d_minv, L.omega, x);   // pre-smoothing from zero
        c->kernels += 1;
        for (int it = 1; it < nu; ++it) { launch_stencil_jacobi(c, x, b, L.omega, y); std::swap(x, y); }
        launch_stencil_residual(c, x, b, L.r);
        k_csr<0><<<g8(C.A.n), 256, 0, s>>>(C.A.n, L.R.ptr, L.R.col, L.R.val, L.r, nullptr, nullptr, 0.0, C.b);
        c->kernels += 1;
        vcycle(c, l + 1);
        k_csr<3><<<g8(n), 256, 0, s>>>(n, L.P.ptr, L.P.col, L.P.val, C.x, nullptr, nullptr, 0.0, x);
        c->kernels += 1;
        for (int it = 0; it < nu; ++it) { launch_stencil_jacobi(c, x, b, L.omega, y); std::swap(x, y); }
        if (x != x0) {
            cudaMemcpyAsync(x0, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
        }
        return;
    }
    // pre-smoothing from zero: x = w D^-1 b, then nu - 1 damped Jacobi sweeps
    k_scaled<<<g1(n), 256, 0, s>>>(n, L.b, L.dinv, L.omega, L.x);
    for (int it = 1; it < nu; ++it) {
        k_csr<2><<<g8(n), 256, 0, s>>>(n, L.A.ptr, L.A.col, L.A.val, L.x, L.b, L.dinv, L.omega, L.x2);
        std::swap(L.x, L.x2);
    }
    c->kernels += nu;
    k_csr<1><<<g8(n), 256, 0, s>>>(n, L.A.ptr, L.A.col, L.A.val, L.x, L.b, nullptr, 0.0, L.r);
    k_csr<0><<<g8(C.A.n), 256, 0, s>>>(C.A.n, L.R.ptr, L.R.col, L.R.val, L.r, nullptr, nullptr, 0.0, C.b);
    c->kernels += 2;
    vcycle(c, l + 1);
    k_csr<3><<<g8(n), 256, 0, s>>>(n, L.P.ptr, L.P.col, L.P.val, C.x, nullptr, nullptr, 0.0, L.x);
    for (int it = 0; it < nu; ++it) {
        k_csr<2><<<g8(n), 256, 0, s>>>(n, L.A.ptr, L.A.col, L.A.val, L.x, L.b, L.dinv, L.omega, L.x2);
        std::swap(L.x, L.x2);
    }
    c->kernels += 1 + nu;
}

void amg_apply(ofks_ctx *c, const double *r_full, double *z_full) {
    if (c->amg_lat) {   // full-node vectors throughout level 0
        vcycle(c, 0, r_full, z_full);
        return;
    }
    const int64_t ni = c->amg_ni;
    AmgLevel &L0 = c->amg[0];
    k_gather<<<g1(ni), 256, 0, c->stream>>>(ni, c->d_amg_idx, r_full, L0.b);
    vcycle(c, 0);
    k_scatter<<<g1(ni), 256, 0, c->stream>>>(ni, c->d_amg_idx, L0.x, z_full);
    c->kernels += 2;
}
