// Lattice-stencil form of the full-node stiffness L used by the Hartree CG (paper Sec. 2.2).
//
// The meshes of this library number their nodes on a lattice, id = (a Ly + b) Lz + c, and every
// hexahedral cell is split the same way, so the neighbours of a node sit at a fixed set of
// lattice offsets that depends only on the parities of (a, b, c): eight node types (cell
// vertices, three kinds of edge midpoints, face and body diagonals of the P2 lattice).  This
// form drops the column indices of the CSR and stores only the symmetric half: an entry
// L(i, j) with j > i lives with row i, at slot `offset` of i's type; row j reads it from there
// ("mirror" entries).  Each type's values are one array per slot over the type's sub-lattice,
// so a warp of consecutive nodes of one type reads 32 consecutive doubles per slot.  Bytes per
// row fall from 12 * 28.9 (CSR, P2 on the Kuhn split) to 8 * 15.
//
// Whether a mesh qualifies is decided from its index structure alone (the values come from the
// assembled CSR): lattice extents read off the coordinates, every CSR offset within [-2, 2]^3,
// every stencil neighbour of every non-Dirichlet row inside the lattice, and a symmetric
// pattern.  Otherwise the CG keeps the CSR.
#include <algorithm>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

inline int code_of(int oa, int ob, int oc) { return (oa + 2) * 25 + (ob + 2) * 5 + (oc + 2); }

// values of the stored half: row i of type t keeps L(i, j) for j >= i at its slot for j - i
__global__ void k_st_fill(int64_t N, int Ly, int Lz, const int *__restrict__ fptr, const int *__restrict__ fcol,
                          const double *__restrict__ fval, const StencilType *__restrict__ types,
                          const int *__restrict__ slot_lut, double *val) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t LyLz = (int64_t)Ly * Lz;
    const int a = (int)(i / LyLz), b = (int)((i / Lz) % Ly), c = (int)(i % Lz);
    const int t = ((a & 1) << 2) | ((b & 1) << 1) | (c & 1);
    const StencilType T = types[t];
    const int64_t idx = ((int64_t)(a >> 1) * T.ny + (b >> 1)) * T.nz + (c >> 1);
    for (int k = fptr[i]; k < fptr[i + 1]; ++k) {
        const int64_t j = fcol[k];
        if (j < i) continue;
        const int ja = (int)(j / LyLz), jb = (int)((j / Lz) % Ly), jc = (int)(j % Lz);
        const int s = slot_lut[t * 125 + (ja - a + 2) * 25 + (jb - b + 2) * 5 + (jc - c + 2)];
        val[T.base + (int64_t)s * T.n + idx] = fval[k];
    }
}

// Row sums s_i = (L x)_i over the non-Dirichlet rows, then by MODE
//   0: y = s and pq += x.s (slot it&1), zeroing the retired rz / rr slots (the CG protocol of
//      the CSR kernel)
//   1: y = b - s                  (multigrid residual)
//   2: y = x + w minv (b - s)     (damped Jacobi sweep)
// Blocks [blk0_t, blk0_{t+1}) cover the nodes of type t in sub-lattice order; one thread per
// row, and every lane of a warp runs the same stencil.  Dirichlet rows are not written.
template <int MODE>
__global__ void __launch_bounds__(256) k_st_apply(int Ly, int Lz, const StencilType *__restrict__ types,
                                                  const StencilEntry *__restrict__ ents,
                                                  const double *__restrict__ val, const double *__restrict__ minv,
                                                  const double *__restrict__ xv, const double *__restrict__ bv,
                                                  double w, double *yv, double *sc, int it, double *gpart,
                                                  unsigned *gcount) {
    __shared__ StencilType st[8];
    __shared__ StencilEntry se[ST_MAXE];
    __shared__ double sh[8];
    if (threadIdx.x < 8) st[threadIdx.x] = types[threadIdx.x];
    __syncthreads();
    int t = 0;
    while (t < 7 && (int)blockIdx.x >= st[t + 1].blk0) ++t;
    const StencilType T = st[t];
    for (int e = threadIdx.x; e < T.nent; e += blockDim.x) se[e] = ents[t * ST_MAXE + e];
    __syncthreads();
    const int64_t idx = (int64_t)((int)blockIdx.x - T.blk0) * blockDim.x + threadIdx.x;
    double pq = 0.0;
    if (idx < T.n) {
        const int64_t nyz = (int64_t)T.ny * T.nz;
        const int ia = (int)(idx / nyz);
        const int64_t rem = idx - (int64_t)ia * nyz;
        const int ib = (int)(rem / T.nz), ic = (int)(rem - (int64_t)ib * T.nz);
        const int a = 2 * ia + T.px, b = 2 * ib + T.py, c = 2 * ic + T.pz;
        const int64_t row = ((int64_t)a * Ly + b) * Lz + c;
        const double mi = minv[row];
        if (mi != 0.0) {
            double s = 0.0;
            int e = 0;
#pragma unroll 4
            for (; e < T.nown; ++e) {   // stored with this row
                const StencilEntry E = se[e];
                s = fma(val[T.base + (int64_t)E.slot * T.n + idx], xv[row + E.lin], s);
            }
#pragma unroll 4
            for (; e < T.nent; ++e) {   // stored with the neighbour (symmetric half)
                const StencilEntry E = se[e];
                const StencilType &S = st[E.tp];
                const int64_t j = ((int64_t)((a + E.oa) >> 1) * S.ny + ((b + E.ob) >> 1)) * S.nz + ((c + E.oc) >> 1);
                s = fma(val[S.base + (int64_t)E.slot * S.n + j], xv[row + E.lin], s);
            }
            if (MODE == 0) { yv[row] = s; pq = xv[row] * s; }
            else if (MODE == 1) yv[row] = bv[row] - s;
            else yv[row] = xv[row] + w * mi * (bv[row] - s);
        }
    }
    if (MODE == 0) {
        if (threadIdx.x == 0 && blockIdx.x == 0) {
            sc[0 + ((it + 1) & 1)] = 0.0;
            sc[4 + ((it + 1) & 1)] = 0.0;
        }
        const double tot[1] = {block_sum(pq, sh)};
        grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[2 + (it & 1)] += v; });
    }
}

// ---- float-float form of the MODE 0 apply (the Hartree CG during the float32 iterations)
//
// A value v is carried as the float32 pair (hi, lo) with v ~ hi + lo (hi = fl(v), lo = fl(v - hi):
// ~48 significant bits); a product a x adds hi_a hi_x exactly (its rounding error by an FMA,
// Dekker's product), plus hi_a lo_x + lo_a hi_x, to the row sum kept as a pair by Knuth's
// two-sum, on the FP32 pipes (the float64 form keeps the FP64 pipe ~77 % busy).  Intrinsics keep
// the compiler from contracting or reordering.  The loads of eight entries are issued before
// their products (the float64 form waits on its loads about as long as on the FP64 pipe).
__device__ __forceinline__ void ff_madd(float &sh, float &sl, const float2 a, const float2 x) {
    const float p = __fmul_rn(a.x, x.x);
    float e = __fmaf_rn(a.x, x.x, -p);
    e = __fmaf_rn(a.x, x.y, e);
    e = __fmaf_rn(a.y, x.x, e);
    const float t = __fadd_rn(sh, p);
    const float bv = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

constexpr int FF_B = 8;                           // entries whose loads are issued together

__global__ void __launch_bounds__(256) k_st_apply_ff(int Ly, int Lz, const StencilType *__restrict__ types,
                                                     const StencilEntry *__restrict__ ents,
                                                     const float2 *__restrict__ val, const double *__restrict__ minv,
                                                     const float2 *__restrict__ xf, const double *__restrict__ xv,
                                                     double *yv, double *sc, int it, double *gpart,
                                                     unsigned *gcount) {
    __shared__ StencilType st[8];
    __shared__ StencilEntry se[ST_MAXE];
    __shared__ double sh[8];
    if (threadIdx.x < 8) st[threadIdx.x] = types[threadIdx.x];
    __syncthreads();
    int t = 0;
    while (t < 7 && (int)blockIdx.x >= st[t + 1].blk0) ++t;
    const StencilType T = st[t];
    for (int e = threadIdx.x; e < T.nent; e += blockDim.x) se[e] = ents[t * ST_MAXE + e];
    __syncthreads();
    const int64_t idx = (int64_t)((int)blockIdx.x - T.blk0) * blockDim.x + threadIdx.x;
    double pq = 0.0;
    if (idx < T.n) {
        const int64_t nyz = (int64_t)T.ny * T.nz;
        const int ia = (int)(idx / nyz);
        const int64_t rem = idx - (int64_t)ia * nyz;
        const int ib = (int)(rem / T.nz), ic = (int)(rem - (int64_t)ib * T.nz);
        const int a = 2 * ia + T.px, b = 2 * ib + T.py, c = 2 * ic + T.pz;
        const int64_t row = ((int64_t)a * Ly + b) * Lz + c;
        if (minv[row] != 0.0) {
            float s_hi = 0.f, s_lo = 0.f;
            // entry e's value: own slots (e < nown) at this row's index, mirrored ones at the
            // neighbour's index in its type's arrays
            auto vaddr = [&](int e) -> const float2 * {
                const StencilEntry E = se[e];
                if (e < T.nown) return val + T.base + (int64_t)E.slot * T.n + idx;
                const StencilType &S = st[E.tp];
                const int64_t j = ((int64_t)((a + E.oa) >> 1) * S.ny + ((b + E.ob) >> 1)) * S.nz + ((c + E.oc) >> 1);
                return val + S.base + (int64_t)E.slot * S.n + j;
            };
            int e = 0;
            for (; e + FF_B <= T.nent; e += FF_B) {
                float2 v[FF_B], x[FF_B];
#pragma unroll
                for (int u = 0; u < FF_B; ++u) {
                    v[u] = __ldg(vaddr(e + u));
                    x[u] = __ldg(xf + row + se[e + u].lin);
                }
#pragma unroll
                for (int u = 0; u < FF_B; ++u) ff_madd(s_hi, s_lo, v[u], x[u]);
            }
            for (; e < T.nent; ++e) ff_madd(s_hi, s_lo, __ldg(vaddr(e)), __ldg(xf + row + se[e].lin));
            const double s = (double)s_hi + (double)s_lo;
            yv[row] = s;
            pq = xv[row] * s;
        }
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc[0 + ((it + 1) & 1)] = 0.0;
        sc[4 + ((it + 1) & 1)] = 0.0;
    }
    const double tot[1] = {block_sum(pq, sh)};
    grid_accumulate<1>(tot, gpart, gcount, [&](int, double v) { sc[2 + (it & 1)] += v; });
}

__global__ void k_st_split(int64_t len, const double *__restrict__ v, float2 *vf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < len) vf[i] = ff_split(v[i]);
}

}  // namespace

void stencil_free(ofks_ctx *c) {
    cudaFree(c->st.val); cudaFree(c->st.valff); cudaFree(c->st.d_type); cudaFree(c->st.d_ent); cudaFree(c->st.d_slot);
    c->st = Stencil{};
}

// Host detection and tables; returns OFKS_OK with c->st.on = false when the mesh does not
// qualify (the CG then runs on the CSR), an error code only for a failed allocation.
int stencil_setup(ofks_ctx *c, int64_t N, const double *xyz, const int64_t *fptr, const int *fcol,
                  const uint8_t *dirichlet) {
    stencil_free(c);
    if (N < 27) return OFKS_OK;
    // lattice extents: ids run fastest along the third axis, then the second
    int64_t Lz = 1;
    while (Lz < N && xyz[3 * Lz] == xyz[0] && xyz[3 * Lz + 1] == xyz[1]) ++Lz;
    int64_t LyLz = Lz;
    while (LyLz < N && xyz[3 * LyLz] == xyz[0]) ++LyLz;
    if (Lz < 3 || LyLz % Lz || N % LyLz) return OFKS_OK;
    const int64_t Ly = LyLz / Lz, Lx = N / LyLz;
    if (Ly < 3 || Lx < 3 || Lx > (1 << 30) || Ly > (1 << 30) || Lz > (1 << 30)) return OFKS_OK;

    // offsets present per type (a row's type is the parity triple of its lattice coordinates)
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    if (N < 200000) nt = 1;
    std::vector<std::vector<uint8_t>> seen(nt, std::vector<uint8_t>(8 * 125, 0));
    std::vector<int> bad(nt, 0);
    auto scan = [&](unsigned w, int64_t r0, int64_t r1) {
        uint8_t *sn = seen[w].data();
        for (int64_t i = r0; i < r1 && !bad[w]; ++i) {
            const int64_t a = i / LyLz, b = (i / Lz) % Ly, cc = i % Lz;
            const int t = (int)(((a & 1) << 2) | ((b & 1) << 1) | (cc & 1));
            for (int64_t k = fptr[i]; k < fptr[i + 1]; ++k) {
                const int64_t j = fcol[k];
                const int64_t oa = j / LyLz - a, ob = (j / Lz) % Ly - b, oc = j % Lz - cc;
                if (oa < -2 || oa > 2 || ob < -2 || ob > 2 || oc < -2 || oc > 2) { bad[w] = 1; break; }
                sn[t * 125 + code_of((int)oa, (int)ob, (int)oc)] = 1;
            }
        }
    };
    {
        std::vector<std::thread> th;
        const int64_t chunk = (N + nt - 1) / nt;
        for (unsigned w = 0; w < nt; ++w) {
            const int64_t r0 = w * chunk, r1 = std::min<int64_t>(N, r0 + chunk);
            if (r0 < r1) th.emplace_back(scan, w, r0, r1);
        }
        for (auto &x : th) x.join();
    }
    for (unsigned w = 0; w < nt; ++w)
        if (bad[w]) return OFKS_OK;
    std::vector<uint8_t> present(8 * 125, 0);
    for (unsigned w = 0; w < nt; ++w)
        for (int q = 0; q < 8 * 125; ++q) present[q] |= seen[w][q];

    // own slots (j - i >= 0, diagonal first), then the mirrored entries
    auto lin_of = [&](int oa, int ob, int oc) { return ((int64_t)oa * Ly + ob) * Lz + oc; };
    std::vector<int> slot(8 * 125, -1);
    StencilType types[8];
    std::vector<StencilEntry> ents(8 * ST_MAXE);
    int64_t len = 0;
    int blk = 0;
    for (int t = 0; t < 8; ++t) {
        StencilType &T = types[t];
        std::memset(&T, 0, sizeof(T));
        T.px = (t >> 2) & 1; T.py = (t >> 1) & 1; T.pz = t & 1;
        T.nx = (int)((Lx - T.px + 1) / 2); T.ny = (int)((Ly - T.py + 1) / 2); T.nz = (int)((Lz - T.pz + 1) / 2);
        T.n = (int64_t)T.nx * T.ny * T.nz;
        std::vector<int> own, mir;
        for (int q = 0; q < 125; ++q) {
            if (!present[t * 125 + q]) continue;
            const int oa = q / 25 - 2, ob = (q / 5) % 5 - 2, oc = q % 5 - 2;
            (lin_of(oa, ob, oc) >= 0 ? own : mir).push_back(q);
        }
        std::sort(own.begin(), own.end(), [&](int x, int y) {
            return lin_of(x / 25 - 2, (x / 5) % 5 - 2, x % 5 - 2) < lin_of(y / 25 - 2, (y / 5) % 5 - 2, y % 5 - 2);
        });
        for (size_t s = 0; s < own.size(); ++s) slot[t * 125 + own[s]] = (int)s;
        T.nown = (int)own.size();
        T.nent = (int)(own.size() + mir.size());
        T.base = len;
        len += (int64_t)T.nown * T.n;
        T.blk0 = blk;
        blk += (int)((T.n + 255) / 256);
        for (size_t s = 0; s < own.size(); ++s) {
            StencilEntry &E = ents[t * ST_MAXE + s];
            const int q = own[s];
            E.oa = (int8_t)(q / 25 - 2); E.ob = (int8_t)((q / 5) % 5 - 2); E.oc = (int8_t)(q % 5 - 2);
            E.lin = (int)lin_of(E.oa, E.ob, E.oc); E.tp = -1; E.slot = (int)s;
        }
        for (size_t s = 0; s < mir.size(); ++s) {   // slots filled in once every type is known
            StencilEntry &E = ents[t * ST_MAXE + T.nown + s];
            const int q = mir[s];
            E.oa = (int8_t)(q / 25 - 2); E.ob = (int8_t)((q / 5) % 5 - 2); E.oc = (int8_t)(q % 5 - 2);
            E.lin = (int)lin_of(E.oa, E.ob, E.oc);
            E.tp = (int8_t)(t ^ (((E.oa & 1) << 2) | ((E.ob & 1) << 1) | (E.oc & 1)));
            E.slot = -1;
        }
    }
    // mirrored entries read the neighbour type's own slot of the opposite offset
    for (int t = 0; t < 8; ++t)
        for (int e = types[t].nown; e < types[t].nent; ++e) {
            StencilEntry &E = ents[t * ST_MAXE + e];
            E.slot = slot[E.tp * 125 + code_of(-E.oa, -E.ob, -E.oc)];
            if (E.slot < 0) return OFKS_OK;   // pattern not symmetric
        }
    // every stencil neighbour of every computed row lies inside the lattice
    std::vector<int> out(nt, 0);
    auto check = [&](unsigned w, int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1 && !out[w]; ++i) {
            if (dirichlet[i]) continue;
            const int64_t a = i / LyLz, b = (i / Lz) % Ly, cc = i % Lz;
            const int t = (int)(((a & 1) << 2) | ((b & 1) << 1) | (cc & 1));
            for (int e = 0; e < types[t].nent; ++e) {
                const StencilEntry &E = ents[t * ST_MAXE + e];
                if (a + E.oa < 0 || a + E.oa >= Lx || b + E.ob < 0 || b + E.ob >= Ly || cc + E.oc < 0 ||
                    cc + E.oc >= Lz) { out[w] = 1; break; }
            }
        }
    };
    {
        std::vector<std::thread> th;
        const int64_t chunk = (N + nt - 1) / nt;
        for (unsigned w = 0; w < nt; ++w) {
            const int64_t r0 = w * chunk, r1 = std::min<int64_t>(N, r0 + chunk);
            if (r0 < r1) th.emplace_back(check, w, r0, r1);
        }
        for (auto &x : th) x.join();
    }
    for (unsigned w = 0; w < nt; ++w)
        if (out[w]) return OFKS_OK;

    Stencil &S = c->st;
    cudaError_t e = cudaMalloc(&S.val, sizeof(double) * std::max<int64_t>(len, 1));
    if (e == cudaSuccess) e = cudaMalloc(&S.valff, sizeof(float2) * std::max<int64_t>(len, 1));
    if (e == cudaSuccess) e = cudaMalloc(&S.d_type, sizeof(types));
    if (e == cudaSuccess) e = cudaMalloc(&S.d_ent, sizeof(StencilEntry) * ents.size());
    if (e == cudaSuccess) e = cudaMalloc(&S.d_slot, sizeof(int) * slot.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(S.val, 0, sizeof(double) * std::max<int64_t>(len, 1), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.d_type, types, sizeof(types), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.d_ent, ents.data(), sizeof(StencilEntry) * ents.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.d_slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        stencil_free(c);
        return ofks_fail(c, OFKS_ENOMEM, "set_mesh: lattice stencil: %s", cudaGetErrorString(e));
    }
    S.Lx = (int)Lx; S.Ly = (int)Ly; S.Lz = (int)Lz;
    S.blocks = blk;
    S.len = len;
    S.rows = 0;
    for (int64_t i = 0; i < N; ++i) S.rows += dirichlet[i] ? 0 : 1;
    S.on = true;
    return OFKS_OK;
}

// copy the stored half out of the assembled CSR values (after k_assemble)
void stencil_fill(ofks_ctx *c) {
    if (!c->st.on) return;
    const int64_t N = c->n_nodes;
    k_st_fill<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(N, c->st.Ly, c->st.Lz, c->d_fptr, c->d_fcol,
                                                                  c->d_fval, c->st.d_type, c->st.d_slot, c->st.val);
    c->kernels += 1;
    if (c->st.valff) {
        k_st_split<<<(unsigned)((c->st.len + 255) / 256), 256, 0, c->stream>>>(c->st.len, c->st.val, c->st.valff);
        c->kernels += 1;
    }
}

void launch_stencil_spmv(ofks_ctx *c, const double *p, double *q, double *sc, int it) {
    k_st_apply<0><<<(unsigned)c->st.blocks, 256, 0, c->stream>>>(c->st.Ly, c->st.Lz, c->st.d_type, c->st.d_ent,
                                                                c->st.val, c->d_minv, p, nullptr, 0.0, q, sc, it,
                                                                c->d_gpart, c->d_gcount);
    c->kernels += 1;
}

void launch_stencil_spmv_ff(ofks_ctx *c, const float2 *pf, const double *p, double *q, double *sc, int it) {
    k_st_apply_ff<<<(unsigned)c->st.blocks, 256, 0, c->stream>>>(c->st.Ly, c->st.Lz, c->st.d_type, c->st.d_ent,
                                                                c->st.valff, c->d_minv, pf, p, q, sc, it, c->d_gpart,
                                                                c->d_gcount);
    c->kernels += 1;
}

void launch_stencil_residual(ofks_ctx *c, const double *x, const double *b, double *r) {
    k_st_apply<1><<<(unsigned)c->st.blocks, 256, 0, c->stream>>>(c->st.Ly, c->st.Lz, c->st.d_type, c->st.d_ent,
                                                                c->st.val, c->d_minv, x, b, 0.0, r, nullptr, 0,
                                                                nullptr, nullptr);
    c->kernels += 1;
}

void launch_stencil_jacobi(ofks_ctx *c, const double *x, const double *b, double w, double *y) {
    k_st_apply<2><<<(unsigned)c->st.blocks, 256, 0, c->stream>>>(c->st.Ly, c->st.Lz, c->st.d_type, c->st.d_ent,
                                                                c->st.val, c->d_minv, x, b, w, y, nullptr, 0,
                                                                nullptr, nullptr);
    c->kernels += 1;
}
