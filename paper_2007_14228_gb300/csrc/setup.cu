// Mesh set-up: sparsity patterns (host index work), SELL-C-sigma layout, element-to-entry
// maps, and device assembly of the stiffness L and mass B (paper Sec. 2.2) plus the
// quadrature geometry.  Only integer index structures are built on the host; every
// floating-point quantity is computed by the kernels below.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int SELL_SIGMA = 2048;   // rows sorted by length inside windows of this size

// Consistent mass matrix of the quadratic tetrahedron times 420/|T| (standard closed form),
// local order: vertices 0..3, edges 01, 02, 03, 12, 13, 23.
__constant__ int c_mass420[10][10] = {
    {6, 1, 1, 1, -4, -4, -4, -6, -6, -6},     {1, 6, 1, 1, -4, -6, -6, -4, -4, -6},
    {1, 1, 6, 1, -6, -4, -6, -4, -6, -4},     {1, 1, 1, 6, -6, -6, -4, -6, -4, -4},
    {-4, -4, -6, -6, 32, 16, 16, 16, 16, 8},  {-4, -6, -4, -6, 16, 32, 16, 16, 8, 16},
    {-4, -6, -6, -4, 16, 16, 32, 8, 16, 16},  {-6, -4, -4, -6, 16, 16, 8, 32, 16, 16},
    {-6, -4, -6, -4, 16, 8, 16, 16, 32, 16},  {-6, -6, -4, -4, 8, 16, 16, 16, 16, 32}};

// float32 values of the type-grouped SELL gathered from the float64 main SELL (-1: padding)
__global__ void k_tsell_values(int64_t len, const int *__restrict__ pos, const double *__restrict__ valL,
                               const double *__restrict__ valB, float *tL, float *tB) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    const int q = pos[e];
    tL[e] = q >= 0 ? (float)valL[q] : 0.f;
    tB[e] = q >= 0 ? (float)valB[q] : 0.f;
}

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)> &f) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 32u));
    if (n < 200000) nt = 1;
    if (nt == 1) { f(0, n); return; }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (unsigned i = 0; i < nt; ++i) {
        int64_t a = i * chunk, b = std::min<int64_t>(n, a + chunk);
        if (a >= b) break;
        th.emplace_back(f, a, b);
    }
    for (auto &t : th) t.join();
}

// Inverse of an element-to-entry map: for each target position, the element entries k (in
// increasing k) with map[k] == position; map values < 0 are skipped.  Counting sort.
template <class I>
void invert_map(const std::vector<I> &map, int64_t npos, std::vector<int> &ptr, std::vector<int> &list) {
    ptr.assign(npos + 1, 0);
    for (const I v : map)
        if (v >= 0) ptr[v + 1]++;
    for (int64_t i = 0; i < npos; ++i) ptr[i + 1] += ptr[i];
    list.resize(ptr[npos]);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t k = 0; k < (int64_t)map.size(); ++k)
        if (map[k] >= 0) list[fill[map[k]]++] = (int)k;
}

// index of (a, b), a <= b, in the upper triangle of a 10 x 10 local matrix stored row by row
__host__ __device__ inline int up10(int a, int b) {
    if (a > b) { const int t = a; a = b; b = t; }
    return a * 10 - a * (a - 1) / 2 + (b - a);
}

// One tetrahedron: geometry, the upper triangle of its local stiffness by the 4-point rule
// (exact for its degree-2 integrand), |T|/4 and the quadrature points.  The local matrices go
// to lloc (T x 55); k_gather_lb / k_gather_full add them into the global arrays.
__global__ void k_element(int64_t T, const int *__restrict__ tetn, const double *__restrict__ xyz, double *lloc,
                          double *wq, double *yq, double cx, double cy, double cz, int *flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int *tn = tetn + t * 10;
    double P[4][3];
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) P[a][d] = xyz[(int64_t)tn[a] * 3 + d];
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) { e1[d] = P[1][d] - P[0][d]; e2[d] = P[2][d] - P[0][d]; e3[d] = P[3][d] - P[0][d]; }
    double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
    double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double det = e1[0] * c23[0] + e1[1] * c23[1] + e1[2] * c23[2];
    if (!(fabs(det) > 0.0)) { atomicExch(flag, 1); return; }
    // gradients of the barycentric coordinates: rows of the inverse Jacobian
    double g[4][3];
    for (int d = 0; d < 3; ++d) {
        g[1][d] = c23[d] / det; g[2][d] = c31[d] / det; g[3][d] = c12[d] / det;
        g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    }
    const double vol = fabs(det) / 6.0, w = 0.25 * vol;
    double Lloc[55];
    for (int i = 0; i < 55; ++i) Lloc[i] = 0.0;
    for (int q = 0; q < 4; ++q) {
        double G[10][3];
        for (int a = 0; a < 4; ++a) {
            double s = 4.0 * p2_bary(q, a) - 1.0;
            for (int d = 0; d < 3; ++d) G[a][d] = s * g[a][d];
        }
        for (int e = 0; e < 6; ++e) {
            int a, b;
            p2_edge(e, a, b);
            double la = p2_bary(q, a), lb = p2_bary(q, b);
            for (int d = 0; d < 3; ++d) G[4 + e][d] = 4.0 * (la * g[b][d] + lb * g[a][d]);
        }
        for (int i = 0; i < 10; ++i)
            for (int j = i; j < 10; ++j)
                Lloc[up10(i, j)] += w * (G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2]);
    }
    for (int i = 0; i < 55; ++i) lloc[t * 55 + i] = Lloc[i];
    wq[t] = w;
    for (int q = 0; q < 4; ++q) {
        double x[3] = {0, 0, 0};
        for (int a = 0; a < 4; ++a)
            for (int d = 0; d < 3; ++d) x[d] += p2_bary(q, a) * P[a][d];
        yq[(t * 4 + q) * 3 + 0] = x[0] - cx;
        yq[(t * 4 + q) * 3 + 1] = x[1] - cy;
        yq[(t * 4 + q) * 3 + 2] = x[2] - cz;
    }
}

// Free-pattern values by gathering, in list order, the element entries that land on each SELL
// position (list entry t 100 + 10 a + b: entry (a, b) of tetrahedron t): L from the local
// stiffness, B = |T| m_ab / 420 from the closed-form P2 mass table.  Positions without entries
// (padding) get zero.  A gather adds in a fixed order, so the values are the same on every run.
__global__ void k_gather_lb(int64_t npos, const int *__restrict__ ptr, const int *__restrict__ list,
                            const double *__restrict__ lloc, const double *__restrict__ wq, double *valL,
                            double *valB) {
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    double l = 0.0, b = 0.0;
    for (int k = ptr[pos]; k < ptr[pos + 1]; ++k) {
        const int code = list[k], t = code / 100, ab = code - 100 * t, a = ab / 10, bb = ab - 10 * a;
        l += lloc[(int64_t)t * 55 + up10(a, bb)];
        b += 4.0 * wq[t] * (double)c_mass420[a][bb] / 420.0;
    }
    valL[pos] = l;
    valB[pos] = b;
}

// Full-node stiffness of the Hartree problem, gathered the same way
__global__ void k_gather_full(int64_t npos, const int *__restrict__ ptr, const int *__restrict__ list,
                              const double *__restrict__ lloc, double *fval) {
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    double l = 0.0;
    for (int k = ptr[pos]; k < ptr[pos + 1]; ++k) {
        const int code = list[k], t = code / 100, ab = code - 100 * t;
        l += lloc[(int64_t)t * 55 + up10(ab / 10, ab % 10)];
    }
    fval[pos] = l;
}

__global__ void k_diagonals(int64_t n, const int64_t *__restrict__ dpos, const double *valL,
                            const double *valB, double *dL, double *dB) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    dL[r] = valL[dpos[r]];
    dB[r] = valB[dpos[r]];
}

__global__ void k_jacobi_full(int64_t n, const int64_t *__restrict__ fdiag, const double *fval,
                              const int *__restrict__ interior, double *minv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    minv[i] = interior[i] ? 1.0 / fval[fdiag[i]] : 0.0;
}

// V_ext(x_q) = -sum_j Z_j / |x_q - R_j|   (paper Eq. ext)
__global__ void k_vext(int64_t nq, const double *__restrict__ yq, double cx, double cy, double cz,
                       int M, const double *__restrict__ ZR, double *vext) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double x = yq[q * 3] + cx, y = yq[q * 3 + 1] + cy, z = yq[q * 3 + 2] + cz;
    double v = 0.0;
    for (int j = 0; j < M; ++j) {
        double dx = x - ZR[4 * j + 1], dy = y - ZR[4 * j + 2], dz = z - ZR[4 * j + 3];
        v -= ZR[4 * j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    vext[q] = v;
}

// E_nuc = sum_{j<k} Z_j Z_k / |R_j - R_k|, one thread
__global__ void k_enuc(int M, const double *__restrict__ ZR, double *out) {
    double e = 0.0;
    for (int j = 0; j < M; ++j)
        for (int k = j + 1; k < M; ++k) {
            double dx = ZR[4 * j + 1] - ZR[4 * k + 1], dy = ZR[4 * j + 2] - ZR[4 * k + 2],
                   dz = ZR[4 * j + 3] - ZR[4 * k + 3];
            e += ZR[4 * j] * ZR[4 * k] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    *out = e;
}

template <class T>
int dev_upload(ofks_ctx *c, T **dst, const T *src, size_t count) {
    if (cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess)
        return ofks_fail(c, OFKS_ENOMEM, "device allocation of %zu bytes failed", sizeof(T) * count);
    if (count && cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess)
        return ofks_fail(c, OFKS_ECUDA, "host-to-device copy failed");
    return OFKS_OK;
}

template <class T>
int dev_zeros(ofks_ctx *c, T **dst, size_t count) {
    if (cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess)
        return ofks_fail(c, OFKS_ENOMEM, "device allocation of %zu bytes failed", sizeof(T) * count);
    if (cudaMemset(*dst, 0, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess)
        return ofks_fail(c, OFKS_ECUDA, "cudaMemset failed");
    return OFKS_OK;
}

template <class T>
void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace

void free_mesh(ofks_ctx *c) {
    clear_graphs(c);
    dev_free(c->d_slice_ptr); dev_free(c->d_slice_w); dev_free(c->d_cols); dev_free(c->d_perm);
    dev_free(c->d_valL); dev_free(c->d_valB); dev_free(c->d_valH); dev_free(c->d_dL); dev_free(c->d_dB);
    dev_free(c->d_fptr); dev_free(c->d_fcol); dev_free(c->d_fval); dev_free(c->d_minv);
    dev_free(c->d_tetf); dev_free(c->d_tetn); dev_free(c->d_hptr); dev_free(c->d_hlist); dev_free(c->d_nptr);
    dev_free(c->d_nlist); dev_free(c->d_wq); dev_free(c->d_yq);
    dev_free(c->d_vext); dev_free(c->d_bnd); dev_free(c->d_bxyz); dev_free(c->d_ynode);
    dev_free(c->d_rho); dev_free(c->d_vh); dev_free(c->d_vxc); dev_free(c->d_exc); dev_free(c->d_ve);
    dev_free(c->d_U); dev_free(c->d_rhs); dev_free(c->d_cr); dev_free(c->d_cz); dev_free(c->d_cp); dev_free(c->d_cpff);
    dev_free(c->d_cq);
    amg_free(c);
    gcn_free(c);
    stencil_free(c);
    sep_free(c);
    dev_free(c->d_tslice_ptr); dev_free(c->d_tslice_w); dev_free(c->d_tcols);
    dev_free(c->d_tmap); dev_free(c->d_tinv);
    dev_free(c->d_tvalL); dev_free(c->d_tvalB);
    c->n_tslices = 0; c->n_slots = 0; c->tsell_len = 0;
    c->amg_tried = false;
    std::vector<int>().swap(c->h_tetn);
    std::vector<double>().swap(c->h_xyz);
    c->n = c->n_nodes = c->n_tets = c->nnz = c->nnz_full = 0;
    c->have_nuclei = false;
}

int setup_mesh(ofks_ctx *c, int64_t n_nodes, const double *xyz, int64_t n_tets, const int64_t *tet10,
               const uint8_t *dirichlet) {
    if (n_nodes < 4 || n_tets < 1 || !xyz || !tet10 || !dirichlet)
        return ofks_fail(c, OFKS_EINVAL, "set_mesh: need n_nodes >= 4, n_tets >= 1 and non-null arrays");
    if (n_nodes >= (int64_t)1 << 31 || n_tets >= ((int64_t)1 << 31) / 100)
        return ofks_fail(c, OFKS_EINVAL, "set_mesh: mesh too large for 32-bit entry indices");
    for (int64_t i = 0; i < n_tets * 10; ++i)
        if (tet10[i] < 0 || tet10[i] >= n_nodes)
            return ofks_fail(c, OFKS_EINVAL, "set_mesh: tet10[%lld] = %lld out of range", (long long)i,
                             (long long)tet10[i]);
    free_mesh(c);
    const int64_t N = n_nodes, T = n_tets;
    std::vector<int> fidx(N);
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) fidx[i] = dirichlet[i] ? -1 : (int)n++;
    if (n < 1) return ofks_fail(c, OFKS_EINVAL, "set_mesh: no free node");
    std::vector<int> tetn(T * 10);
    for (int64_t i = 0; i < T * 10; ++i) tetn[i] = (int)tet10[i];

    // node -> tetrahedra adjacency
    std::vector<int64_t> aptr(N + 1, 0);
    for (int64_t i = 0; i < T * 10; ++i) aptr[tetn[i] + 1]++;
    for (int64_t i = 0; i < N; ++i) aptr[i + 1] += aptr[i];
    std::vector<int> adj(aptr[N]);
    {
        std::vector<int64_t> fill(aptr.begin(), aptr.end() - 1);
        for (int64_t t = 0; t < T; ++t)
            for (int a = 0; a < 10; ++a) adj[fill[tetn[t * 10 + a]]++] = (int)t;
    }
    // full-node pattern: row i = sorted unique nodes of the tetrahedra around i
    auto row_nodes = [&](int64_t i, std::vector<int> &buf) {
        buf.clear();
        for (int64_t k = aptr[i]; k < aptr[i + 1]; ++k)
            for (int a = 0; a < 10; ++a) buf.push_back(tetn[(int64_t)adj[k] * 10 + a]);
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    };
    std::vector<int64_t> fptr(N + 1, 0);
    parallel_for(N, [&](int64_t a, int64_t b) {
        std::vector<int> buf;
        for (int64_t i = a; i < b; ++i) { row_nodes(i, buf); fptr[i + 1] = (int64_t)buf.size(); }
    });
    for (int64_t i = 0; i < N; ++i) fptr[i + 1] += fptr[i];
    const int64_t nnz_full = fptr[N];
    std::vector<int> fcol(nnz_full);
    parallel_for(N, [&](int64_t a, int64_t b) {
        std::vector<int> buf;
        for (int64_t i = a; i < b; ++i) {
            row_nodes(i, buf);
            std::copy(buf.begin(), buf.end(), fcol.begin() + fptr[i]);
        }
    });
    // free pattern: restriction of the full rows to free nodes (fidx is monotone)
    std::vector<int64_t> rptr(n + 1, 0);
    std::vector<int> rowlen(n);
    std::vector<int64_t> node_of(n);
    for (int64_t i = 0; i < N; ++i)
        if (fidx[i] >= 0) node_of[fidx[i]] = i;
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t r = a; r < b; ++r) {
            int64_t i = node_of[r];
            int cnt = 0;
            for (int64_t k = fptr[i]; k < fptr[i + 1]; ++k) cnt += fidx[fcol[k]] >= 0;
            rowlen[r] = cnt;
        }
    });
    for (int64_t r = 0; r < n; ++r) rptr[r + 1] = rptr[r] + rowlen[r];
    c->row_deg = rowlen;
    const int64_t nnz = rptr[n];
    std::vector<int> rcol(nnz);
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t r = a; r < b; ++r) {
            int64_t i = node_of[r], o = rptr[r];
            for (int64_t k = fptr[i]; k < fptr[i + 1]; ++k)
                if (fidx[fcol[k]] >= 0) rcol[o++] = fidx[fcol[k]];
        }
    });
    // SELL-C-sigma: rows sorted by decreasing length inside windows of SELL_SIGMA rows
    std::vector<int> sorted(n), inv(n);
    std::iota(sorted.begin(), sorted.end(), 0);
    for (int64_t w0 = 0; w0 < n; w0 += SELL_SIGMA) {
        int64_t w1 = std::min<int64_t>(n, w0 + SELL_SIGMA);
        std::stable_sort(sorted.begin() + w0, sorted.begin() + w1,
                         [&](int x, int y) { return rowlen[x] > rowlen[y]; });
    }
    for (int64_t s = 0; s < n; ++s) inv[sorted[s]] = (int)s;
    const int n_slices = (int)((n + SELL_C - 1) / SELL_C);
    std::vector<int> slice_ptr(n_slices + 1, 0), slice_w(n_slices, 0), perm((int64_t)n_slices * SELL_C, -1);
    int64_t acc = 0;
    for (int s = 0; s < n_slices; ++s) {
        int w = 0;
        for (int l = 0; l < SELL_C; ++l) {
            int64_t sp = (int64_t)s * SELL_C + l;
            if (sp < n) { w = std::max(w, rowlen[sorted[sp]]); perm[sp] = sorted[sp]; }
        }
        slice_w[s] = w;
        if (acc >= ((int64_t)1 << 31)) return ofks_fail(c, OFKS_EINVAL, "set_mesh: SELL storage exceeds 2^31");
        slice_ptr[s] = (int)acc;
        acc += (int64_t)w * SELL_C;
    }
    if (acc >= ((int64_t)1 << 31)) return ofks_fail(c, OFKS_EINVAL, "set_mesh: SELL storage exceeds 2^31");
    slice_ptr[n_slices] = (int)acc;
    const int64_t sell_len = acc;
    std::vector<int> cols(sell_len, 0);
    parallel_for(n_slices, [&](int64_t a, int64_t b) {
        for (int64_t s = a; s < b; ++s)
            for (int l = 0; l < SELL_C; ++l) {
                int64_t sp = s * SELL_C + l;
                if (sp >= n) continue;
                int r = sorted[sp];
                int len = rowlen[r];
                for (int j = 0; j < slice_w[s]; ++j)
                    cols[slice_ptr[s] + (int64_t)j * SELL_C + l] = rcol[rptr[r] + std::min(j, len - 1)];
            }
    });
    auto sell_pos = [&](int r, int col) -> int64_t {
        const int *b = rcol.data() + rptr[r], *e = rcol.data() + rptr[r + 1];
        const int *f = std::lower_bound(b, e, col);
        int64_t sp = inv[r];
        return slice_ptr[sp / SELL_C] + (int64_t)(f - b) * SELL_C + (sp % SELL_C);
    };
    std::vector<int> emap(T * 100);
    std::vector<int64_t> fmap(T * 100);
    std::vector<int> tetf(T * 10);
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t t = a; t < b; ++t) {
            const int *tn = tetn.data() + t * 10;
            for (int i = 0; i < 10; ++i) {
                tetf[t * 10 + i] = fidx[tn[i]];
                for (int j = 0; j < 10; ++j) {
                    const int *rb = fcol.data() + fptr[tn[i]], *re = fcol.data() + fptr[tn[i] + 1];
                    fmap[t * 100 + i * 10 + j] = fptr[tn[i]] + (std::lower_bound(rb, re, tn[j]) - rb);
                    int fi = fidx[tn[i]], fj = fidx[tn[j]];
                    emap[t * 100 + i * 10 + j] = (fi >= 0 && fj >= 0) ? (int)sell_pos(fi, fj) : -1;
                }
            }
        }
    });
    std::vector<int64_t> dpos(n), fdiag(N);
    for (int64_t r = 0; r < n; ++r) dpos[r] = sell_pos((int)r, (int)r);
    for (int64_t i = 0; i < N; ++i) {
        const int *rb = fcol.data() + fptr[i], *re = fcol.data() + fptr[i + 1];
        fdiag[i] = fptr[i] + (std::lower_bound(rb, re, (int)i) - rb);
    }
    std::vector<int> interior(N), bnd;
    for (int64_t i = 0; i < N; ++i) {
        interior[i] = dirichlet[i] ? 0 : 1;
        if (dirichlet[i]) bnd.push_back((int)i);
    }
    // centre of the node bounding box (multipole origin)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], xyz[i * 3 + d]); hi[d] = std::max(hi[d], xyz[i * 3 + d]); }
    for (int d = 0; d < 3; ++d) c->center[d] = 0.5 * (lo[d] + hi[d]);
    std::vector<double> bxyz(bnd.size() * 3);
    for (size_t k = 0; k < bnd.size(); ++k)
        for (int d = 0; d < 3; ++d) bxyz[k * 3 + d] = xyz[(int64_t)bnd[k] * 3 + d] - c->center[d];
    // node positions for the moments: the affine (straight-sided) P2 node of each edge is its midpoint
    std::vector<double> ynode((size_t)N * 3);
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) ynode[i * 3 + d] = xyz[i * 3 + d] - c->center[d];
    for (int64_t t = 0; t < T; ++t)
        for (int e = 0; e < 6; ++e) {
            int a, b;
            p2_edge(e, a, b);
            const int64_t va = tetn[t * 10 + a], vb = tetn[t * 10 + b], m = tetn[t * 10 + 4 + e];
            for (int d = 0; d < 3; ++d) ynode[m * 3 + d] = 0.5 * (xyz[va * 3 + d] + xyz[vb * 3 + d]) - c->center[d];
        }

    // ---- device
    int rc;
    std::vector<int> fptr32(N + 1);
    if (nnz_full >= ((int64_t)1 << 31)) return ofks_fail(c, OFKS_EINVAL, "set_mesh: full pattern exceeds 2^31");
    for (int64_t i = 0; i <= N; ++i) fptr32[i] = (int)fptr[i];
    // inverse element-to-entry maps: the assembly and the Hamiltonian refresh gather each entry's
    // element contributions in a fixed order (no floating-point atomics)
    std::vector<int> hptr, hlist, gptr, glist, nptr, nlist;
    invert_map(emap, sell_len, hptr, hlist);
    invert_map(fmap, nnz_full, gptr, glist);
    invert_map(tetn, N, nptr, nlist);
    std::vector<int64_t>().swap(fmap);
    double *d_xyz = nullptr, *d_lloc = nullptr;
    int64_t *d_dpos = nullptr, *d_fdiag = nullptr;
    int *d_interior = nullptr, *d_flag = nullptr, *d_gptr = nullptr, *d_glist = nullptr;
    if ((rc = dev_upload(c, &c->d_slice_ptr, slice_ptr.data(), slice_ptr.size())) ||
        (rc = dev_upload(c, &c->d_slice_w, slice_w.data(), slice_w.size())) ||
        (rc = dev_upload(c, &c->d_cols, cols.data(), cols.size())) ||
        (rc = dev_upload(c, &c->d_perm, perm.data(), perm.size())) ||
        (rc = dev_zeros(c, &c->d_valL, sell_len)) || (rc = dev_zeros(c, &c->d_valB, sell_len)) ||
        (rc = dev_zeros(c, &c->d_valH, sell_len)) || (rc = dev_zeros(c, &c->d_dL, n)) ||
        (rc = dev_zeros(c, &c->d_dB, n)) ||
        (rc = dev_upload(c, &c->d_fptr, fptr32.data(), fptr32.size())) ||
        (rc = dev_upload(c, &c->d_fcol, fcol.data(), fcol.size())) ||
        (rc = dev_zeros(c, &c->d_fval, nnz_full)) || (rc = dev_zeros(c, &c->d_minv, N)) ||
        (rc = dev_upload(c, &c->d_tetf, tetf.data(), tetf.size())) ||
        (rc = dev_upload(c, &c->d_tetn, tetn.data(), tetn.size())) ||
        (rc = dev_upload(c, &c->d_hptr, hptr.data(), hptr.size())) ||
        (rc = dev_upload(c, &c->d_hlist, hlist.data(), hlist.size())) ||
        (rc = dev_upload(c, &c->d_nptr, nptr.data(), nptr.size())) ||
        (rc = dev_upload(c, &c->d_nlist, nlist.data(), nlist.size())) ||
        (rc = dev_upload(c, &d_gptr, gptr.data(), gptr.size())) ||
        (rc = dev_upload(c, &d_glist, glist.data(), glist.size())) ||
        (rc = dev_zeros(c, &d_lloc, T * 55)) ||
        (rc = dev_zeros(c, &c->d_wq, T)) || (rc = dev_zeros(c, &c->d_yq, T * 12)) ||
        (rc = dev_zeros(c, &c->d_vext, T * 4)) ||
        (rc = dev_upload(c, &c->d_bnd, bnd.data(), bnd.size())) ||
        (rc = dev_upload(c, &c->d_bxyz, bxyz.data(), bxyz.size())) ||
        (rc = dev_upload(c, &c->d_ynode, ynode.data(), ynode.size())) ||
        (rc = dev_zeros(c, &c->d_rho, T * 4)) || (rc = dev_zeros(c, &c->d_vh, T * 4)) ||
        (rc = dev_zeros(c, &c->d_ve, T * 4)) ||
        (rc = dev_zeros(c, &c->d_vxc, T * 4)) || (rc = dev_zeros(c, &c->d_exc, T * 4)) ||
        (rc = dev_zeros(c, &c->d_U, N)) || (rc = dev_zeros(c, &c->d_rhs, N)) ||
        (rc = dev_zeros(c, &c->d_cr, N)) || (rc = dev_zeros(c, &c->d_cz, N)) ||
        (rc = dev_zeros(c, &c->d_cp, N)) || (rc = dev_zeros(c, &c->d_cq, N)) || (rc = dev_zeros(c, &c->d_cpff, N)) ||
        (rc = dev_upload(c, &d_xyz, xyz, (size_t)N * 3)) ||
        (rc = dev_upload(c, &d_dpos, dpos.data(), dpos.size())) ||
        (rc = dev_upload(c, &d_fdiag, fdiag.data(), fdiag.size())) ||
        (rc = dev_upload(c, &d_interior, interior.data(), interior.size())) ||
        (rc = dev_zeros(c, &d_flag, 1))) {
        dev_free(d_xyz); dev_free(d_lloc); dev_free(d_gptr); dev_free(d_glist); dev_free(d_dpos); dev_free(d_fdiag); dev_free(d_interior);
        dev_free(d_flag);
        free_mesh(c);
        return rc;
    }
    const int B = 128;
    k_element<<<(unsigned)((T + B - 1) / B), B, 0, c->stream>>>(T, c->d_tetn, d_xyz, d_lloc, c->d_wq, c->d_yq,
                                                                 c->center[0], c->center[1], c->center[2], d_flag);
    k_gather_lb<<<(unsigned)((sell_len + 255) / 256), 256, 0, c->stream>>>(sell_len, c->d_hptr, c->d_hlist, d_lloc,
                                                                            c->d_wq, c->d_valL, c->d_valB);
    k_gather_full<<<(unsigned)((nnz_full + 255) / 256), 256, 0, c->stream>>>(nnz_full, d_gptr, d_glist, d_lloc,
                                                                              c->d_fval);
    k_diagonals<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, d_dpos, c->d_valL, c->d_valB,
                                                                     c->d_dL, c->d_dB);
    k_jacobi_full<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(N, d_fdiag, c->d_fval, d_interior,
                                                                       c->d_minv);
    if ((rc = stencil_setup(c, N, xyz, fptr.data(), fcol.data(), dirichlet)) != OFKS_OK ||
        (rc = sep_setup(c, xyz, dirichlet)) != OFKS_OK) {
        dev_free(d_xyz); dev_free(d_lloc); dev_free(d_gptr); dev_free(d_glist); dev_free(d_dpos); dev_free(d_fdiag); dev_free(d_interior);
        dev_free(d_flag);
        free_mesh(c);
        return rc;
    }
    c->n_nodes = N;
    stencil_fill(c);
    // type-grouped SELL for the float32 PCG (lattice meshes): the free rows in type order (the
    // lattice node types in turn, each in lattice order), which is also the row order of the
    // PCG's chunk-major blocks, so the 32 rows of a slice and their neighbours at one offset are
    // consecutive rows
    if (c->st.on) {
        const int Lx = c->st.Lx, Ly = c->st.Ly, Lz = c->st.Lz;
        std::vector<int> tp;
        tp.reserve(n);
        for (int t = 0; t < 8; ++t)
            for (int a = (t >> 2) & 1; a < Lx; a += 2)
                for (int b = (t >> 1) & 1; b < Ly; b += 2)
                    for (int cz = t & 1; cz < Lz; cz += 2) {
                        const int f = fidx[((int64_t)a * Ly + b) * Lz + cz];
                        if (f >= 0) tp.push_back(f);
                    }
        if ((int64_t)tp.size() == n) {
            const int nts = (int)((n + SELL_C - 1) / SELL_C);
            std::vector<int> tinv(n, -1), tmap((int64_t)nts * SELL_C, -1);
            for (int64_t k = 0; k < n; ++k) { tinv[tp[k]] = (int)k; tmap[k] = tp[k]; }
            std::vector<int> tptr(nts + 1, 0), tw(nts, 0);
            int64_t acc2 = 0;
            bool fits = true;
            for (int s = 0; s < nts; ++s) {
                int w = 0;
                for (int l = 0; l < SELL_C; ++l) {
                    const int64_t k = (int64_t)s * SELL_C + l;
                    if (k < n) w = std::max(w, rowlen[tp[k]]);
                }
                tw[s] = w;
                if (acc2 >= ((int64_t)1 << 31)) fits = false;
                tptr[s] = (int)acc2;
                acc2 += (int64_t)w * SELL_C;
            }
            fits = fits && acc2 < ((int64_t)1 << 31);
            if (fits) {
                tptr[nts] = (int)acc2;
                std::vector<int> tcol(acc2, 0), tpos(acc2, -1);
                parallel_for(nts, [&](int64_t a0, int64_t a1) {
                    for (int64_t s = a0; s < a1; ++s)
                        for (int l = 0; l < SELL_C; ++l) {
                            const int64_t k = s * SELL_C + l;
                            if (k >= n) continue;
                            const int r = tp[k], len = rowlen[r];
                            const int64_t sp = inv[r];
                            for (int j = 0; j < tw[s]; ++j) {
                                const int jj = std::min(j, len - 1);
                                const int64_t e = tptr[s] + (int64_t)j * SELL_C + l;
                                tcol[e] = tinv[rcol[rptr[r] + jj]];
                                if (j < len) tpos[e] = (int)(slice_ptr[sp / SELL_C] + (int64_t)j * SELL_C + sp % SELL_C);
                            }
                        }
                });
                int *d_tpos = nullptr;
                if ((rc = dev_upload(c, &c->d_tslice_ptr, tptr.data(), tptr.size())) ||
                    (rc = dev_upload(c, &c->d_tslice_w, tw.data(), tw.size())) ||
                    (rc = dev_upload(c, &c->d_tmap, tmap.data(), tmap.size())) ||
                    (rc = dev_upload(c, &c->d_tinv, tinv.data(), tinv.size())) ||
                    (rc = dev_upload(c, &c->d_tcols, tcol.data(), tcol.size())) ||
                    (rc = dev_upload(c, &d_tpos, tpos.data(), tpos.size())) ||
                    (rc = dev_zeros(c, &c->d_tvalL, acc2)) || (rc = dev_zeros(c, &c->d_tvalB, acc2))) {
                    dev_free(d_tpos);
                    dev_free(d_xyz); dev_free(d_lloc); dev_free(d_gptr); dev_free(d_glist); dev_free(d_dpos); dev_free(d_fdiag); dev_free(d_interior);
                    dev_free(d_flag);
                    free_mesh(c);
                    return rc;
                }
                k_tsell_values<<<(unsigned)((acc2 + 255) / 256), 256, 0, c->stream>>>(acc2, d_tpos, c->d_valL, c->d_valB,
                                                                                     c->d_tvalL, c->d_tvalB);
                cudaStreamSynchronize(c->stream);
                dev_free(d_tpos);
                c->n_tslices = nts;
                c->n_slots = (int64_t)nts * SELL_C;
                c->tsell_len = acc2;
                c->kernels += 1;
            }
        }
    }
    int hflag = 0;
    cudaError_t e = cudaMemcpyAsync(&hflag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(d_xyz); dev_free(d_lloc); dev_free(d_gptr); dev_free(d_glist); dev_free(d_dpos); dev_free(d_fdiag); dev_free(d_interior);
    dev_free(d_flag);
    if (e != cudaSuccess) { free_mesh(c); return ofks_cuda_check(c, e, "mesh assembly"); }
    if (hflag) { free_mesh(c); return ofks_fail(c, OFKS_EINVAL, "set_mesh: degenerate tetrahedron"); }
    c->n_nodes = N; c->n_tets = T; c->n = n; c->nnz = nnz; c->nnz_full = nnz_full;
    c->n_slices = n_slices; c->sell_len = sell_len; c->n_bnd = (int)bnd.size();
    c->max_slice_w = slice_w.empty() ? 0 : *std::max_element(slice_w.begin(), slice_w.end());
    // the multigrid hierarchy is built on the first Hartree solve that asks for it
    c->h_tetn.swap(tetn);
    c->h_xyz.assign(xyz, xyz + N * 3);
    return OFKS_OK;
}

int setup_nuclei(ofks_ctx *c, int M, const double *Z, const double *R) {
    std::vector<double> zr((size_t)M * 4);
    for (int j = 0; j < M; ++j) {
        zr[4 * j] = Z[j];
        for (int d = 0; d < 3; ++d) zr[4 * j + 1 + d] = R[3 * j + d];
    }
    double *d_zr = nullptr, *d_e = nullptr;
    int rc;
    if ((rc = dev_upload(c, &d_zr, zr.data(), zr.size())) || (rc = dev_zeros(c, &d_e, 1))) {
        dev_free(d_zr); dev_free(d_e);
        return rc;
    }
    int64_t nq = c->n_tets * 4;
    k_vext<<<(unsigned)((nq + 255) / 256), 256, 0, c->stream>>>(nq, c->d_yq, c->center[0], c->center[1],
                                                                  c->center[2], M, d_zr, c->d_vext);
    k_enuc<<<1, 1, 0, c->stream>>>(M, d_zr, d_e);
    cudaError_t e = cudaMemcpyAsync(&c->e_nuc, d_e, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(d_zr); dev_free(d_e);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "set_nuclei");
    c->have_nuclei = true;
    return OFKS_OK;
}

// ------------------------------------------------------------------------------------------
// No-allocation variant of setup_nuclei (ofks_set_nuclei_static).  The nuclear data that
// setup_nuclei stages in freshly allocated device memory lives here in a fixed file-scope
// array, so the call allocates nothing.  Every GPU that loads the library holds the array
// (32 KiB) until the process exits; all calls share it, so calls that overlap on the GPU
// (different contexts on different streams) race on its contents.
static __device__ __align__(256) double g_nuclei_stage[4 * OFKS_STATIC_NUCLEI_MAX + 1];

// Device address of the staging array on the context's device, looked up once per context by
// ofks_create with that device current (in host code the symbol is only a stand-in, never a
// device address).  Kept in the context, whose lifetime lies within one live CUDA context, so a
// later context after a device reset looks the address up again.
cudaError_t static_stage_lookup(ofks_ctx *c) {
    return cudaGetSymbolAddress((void **)&c->nuclei_stage, g_nuclei_stage);
}

int setup_nuclei_static(ofks_ctx *c, int M, const double *Z, const double *R) {
    double *stage = c->nuclei_stage;
    if (!stage) return ofks_fail(c, OFKS_ESTATE, "set_nuclei_static: no staging address (context not created)");
    double *e_slot = stage + 4 * OFKS_STATIC_NUCLEI_MAX;
    // Z[j] -> stage[4j], R[j] -> stage[4j+1 .. 4j+3]: strided copies, no host staging buffer
    cudaError_t e = cudaMemcpy2DAsync(stage, 4 * sizeof(double), Z, sizeof(double), sizeof(double), (size_t)M,
                                      cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(stage + 1, 4 * sizeof(double), R, 3 * sizeof(double), 3 * sizeof(double), (size_t)M,
                              cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(e_slot, 0, sizeof(double), c->stream);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "set_nuclei_static: staging copy");
    const int64_t nq = c->n_tets * 4;
    k_vext<<<(unsigned)((nq + 255) / 256), 256, 0, c->stream>>>(nq, c->d_yq, c->center[0], c->center[1],
                                                                  c->center[2], M, stage, c->d_vext);
    k_enuc<<<1, 1, 0, c->stream>>>(M, stage, e_slot);
    c->kernels += 2;
    e = cudaMemcpyAsync(&c->e_nuc, e_slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "set_nuclei_static");
    c->have_nuclei = true;
    return OFKS_OK;
}
