// Stencil form of the float32 PCG operator apply (Eq. precondition-T: T_k Z = L Z / 2 -
// shift_k B Z) on lattice meshes whose Dirichlet nodes are the lattice's faces.
//
// On such a mesh the free node at lattice position (A, B, C) couples only to free nodes at
// offsets in [-2, 2]^3, and which offsets occur depends only on the node type t = the parity
// triple (A & 1, B & 1, C & 1) (the same Kuhn split in every cell).  So L and B are stored per
// type and offset as float32 arrays over the type's interior sub-lattice (zero where the
// neighbour is a Dirichlet node) and no column ids are read.  One CTA takes a tile of
// 4 x 4 x 64 lattice positions and up to PS_CG 4-column chunks of the PCG block: the chunks'
// rows of Z for the tile and its 2-wide halo go to shared memory once (coalesced along C), then
// each warp takes the 32 nodes of one type on one (A, B) line of the tile (C two apart) and
// multiplies its stencil against the staged rows.  The C axis of the staged tile is stored
// even positions first, odd ones after, so a warp's 32 neighbour reads at one offset are 32
// consecutive 16-byte pieces (no bank conflicts); the values of one offset are 32 consecutive
// floats of its array.  The own rows then update P <- Z + beta P and Q <- T Z + beta Q (so
// T P = Q) and the column sums P.Q go out as per-tile partials, added in tile order by the
// PCG's alpha kernel.  The operator is the same as the SELL apply's (k_pcg_apply_zc).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int PS_TA = 4, PS_TB = 4, PS_TC = 64;             // tile of lattice positions
constexpr int PS_HA = PS_TA + 4, PS_HB = PS_TB + 4, PS_HC = PS_TC + 4;   // with the halo
constexpr int PS_HC2 = PS_HC / 2;                           // per parity along C
constexpr int PS_CG = 3;                                    // 4-column chunks per CTA
constexpr int PS_THREADS = 1024;
constexpr int PS_WARPS = PS_THREADS / 32;

// values of the free-pattern SELL entries into the stencil arrays: dst[k] <- src[pos[k]]
__global__ void k_ps_values(int64_t m, const int64_t *__restrict__ dst, const int *__restrict__ src,
                            const double *__restrict__ valL, const double *__restrict__ valB, float *L, float *B) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= m) return;
    L[dst[k]] = (float)valL[src[k]];
    B[dst[k]] = (float)valB[src[k]];
}

struct PsArgs {
    int Lx, Ly, Lz, ny, nz;                  // full lattice; interior extents along B and C
    int64_t ns;                              // row stride of the chunk-major blocks
    int nchunks, ngroups, tiles, tA, tB, tC; // chunks of the block, CTA groups of chunks, tile grid
    int pc;
    int K[8], first[8][3], dims[8][3];
    int64_t base[8];
    const int *off;
    const float *L, *B;
    const float *Z;
    float *P, *Q;
    const double *beta, *shift;
    double *part;
    int first_it;
};

__device__ __forceinline__ int hidx(int a, int b, int cc) {      // staged tile index (C split by parity)
    return (a * PS_HB + b) * PS_HC + (cc & 1) * PS_HC2 + (cc >> 1);
}

}  // namespace

void pcg_stencil_free(ofks_ctx *c) {
    PcgStencil &S = c->ps;
    if (S.d_off) cudaFree(S.d_off);
    if (S.d_L) cudaFree(S.d_L);
    if (S.d_B) cudaFree(S.d_B);
    S = PcgStencil{};
}

// Host set-up: the free nodes must be the interior of the lattice in lexicographic order; the
// offsets of each type are the union over its rows; the values come from the SELL entries (row
// r's j-th stored entry is its j-th CSR entry, at slice_ptr[inv[r] / 32] + 32 j + inv[r] % 32).
int pcg_stencil_setup(ofks_ctx *c, const std::vector<int> &fidx, const std::vector<int64_t> &rptr,
                      const std::vector<int> &rcol, const std::vector<int> &inv, const std::vector<int> &slice_ptr) {
    pcg_stencil_free(c);
    if (!c->st.on) return OFKS_OK;
    const int Lx = c->st.Lx, Ly = c->st.Ly, Lz = c->st.Lz;
    const int nx = Lx - 2, ny = Ly - 2, nz = Lz - 2;
    const int64_t n = (int64_t)rptr.size() - 1;                  // free nodes
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz != n) return OFKS_OK;
    for (int A = 0; A < Lx; ++A)
        for (int B = 0; B < Ly; ++B)
            for (int C = 0; C < Lz; ++C) {
                const bool in = A > 0 && A < Lx - 1 && B > 0 && B < Ly - 1 && C > 0 && C < Lz - 1;
                const int f = fidx[((int64_t)A * Ly + B) * Lz + C];
                const int want = in ? (int)(((int64_t)(A - 1) * ny + (B - 1)) * nz + (C - 1)) : -1;
                if (f != want) return OFKS_OK;
            }
    PcgStencil S;
    S.Lx = Lx; S.Ly = Ly; S.Lz = Lz;
    auto coords = [&](int64_t r, int &A, int &B, int &C) {
        C = (int)(r % nz) + 1;
        B = (int)((r / nz) % ny) + 1;
        A = (int)(r / ((int64_t)ny * nz)) + 1;
    };
    auto type_of = [](int A, int B, int C) { return ((A & 1) << 2) | ((B & 1) << 1) | (C & 1); };
    // offsets per type
    std::vector<int> used(8 * 125, 0);
    for (int64_t r = 0; r < n; ++r) {
        int A, B, C;
        coords(r, A, B, C);
        const int t = type_of(A, B, C);
        for (int64_t k = rptr[r]; k < rptr[r + 1]; ++k) {
            int A2, B2, C2;
            coords(rcol[k], A2, B2, C2);
            const int da = A2 - A, db = B2 - B, dc = C2 - C;
            if (da < -2 || da > 2 || db < -2 || db > 2 || dc < -2 || dc > 2) return OFKS_OK;
            used[t * 125 + (da + 2) * 25 + (db + 2) * 5 + dc + 2] = 1;
        }
    }
    std::vector<int> slot(8 * 125, -1), off(8 * PS_KMAX, 0);
    int64_t tot = 0;
    for (int t = 0; t < 8; ++t) {
        int k = 0;
        for (int o = 0; o < 125; ++o)
            if (used[t * 125 + o]) {
                if (k >= PS_KMAX) return OFKS_OK;
                slot[t * 125 + o] = k;
                off[t * PS_KMAX + k] = o;
                ++k;
            }
        S.K[t] = k;
        const int par[3] = {(t >> 2) & 1, (t >> 1) & 1, t & 1}, L3[3] = {Lx, Ly, Lz};
        for (int d = 0; d < 3; ++d) {
            const int f0 = (par[d] == 1) ? 1 : 2;             // first interior coordinate of that parity
            S.first[t][d] = f0;
            S.dims[t][d] = f0 <= L3[d] - 2 ? (L3[d] - 2 - f0) / 2 + 1 : 0;
        }
        S.base[t] = tot;
        tot += (int64_t)k * S.dims[t][0] * S.dims[t][1] * S.dims[t][2];
    }
    // destination of every stored entry, and its SELL position
    std::vector<int64_t> dst(rptr[n]);
    std::vector<int> src(rptr[n]);
    for (int64_t r = 0; r < n; ++r) {
        int A, B, C;
        coords(r, A, B, C);
        const int t = type_of(A, B, C);
        const int64_t nt = (int64_t)S.dims[t][0] * S.dims[t][1] * S.dims[t][2];
        const int64_t it = ((int64_t)((A - S.first[t][0]) / 2) * S.dims[t][1] + (B - S.first[t][1]) / 2) * S.dims[t][2] +
                           (C - S.first[t][2]) / 2;
        const int sp = inv[r];
        for (int64_t k = rptr[r]; k < rptr[r + 1]; ++k) {
            int A2, B2, C2;
            coords(rcol[k], A2, B2, C2);
            const int o = (A2 - A + 2) * 25 + (B2 - B + 2) * 5 + (C2 - C + 2);
            dst[k] = S.base[t] + (int64_t)slot[t * 125 + o] * nt + it;
            src[k] = slice_ptr[sp / SELL_C] + (int)(k - rptr[r]) * SELL_C + sp % SELL_C;
        }
    }
    int64_t *d_dst = nullptr;
    int *d_src = nullptr;
    cudaError_t e = cudaMalloc((void **)&S.d_off, sizeof(int) * off.size());
    if (e == cudaSuccess) e = cudaMemcpy(S.d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.d_L, sizeof(float) * std::max<int64_t>(tot, 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.d_B, sizeof(float) * std::max<int64_t>(tot, 1));
    if (e == cudaSuccess) e = cudaMemset(S.d_L, 0, sizeof(float) * std::max<int64_t>(tot, 1));
    if (e == cudaSuccess) e = cudaMemset(S.d_B, 0, sizeof(float) * std::max<int64_t>(tot, 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_dst, sizeof(int64_t) * std::max<size_t>(dst.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_src, sizeof(int) * std::max<size_t>(src.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_dst, dst.data(), sizeof(int64_t) * dst.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_src, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int64_t m = (int64_t)dst.size();
        k_ps_values<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(m, d_dst, d_src, c->d_valL, c->d_valB, S.d_L,
                                                                          S.d_B);
        e = cudaStreamSynchronize(c->stream);
    }
    if (d_dst) cudaFree(d_dst);
    if (d_src) cudaFree(d_src);
    if (e != cudaSuccess) {
        if (S.d_off) cudaFree(S.d_off);
        if (S.d_L) cudaFree(S.d_L);
        if (S.d_B) cudaFree(S.d_B);
        return ofks_fail(c, OFKS_ENOMEM, "set_mesh: stencil form of the PCG operator: %s", cudaGetErrorString(e));
    }
    S.len = tot;
    S.on = true;
    c->ps = S;
    return OFKS_OK;
}

namespace {

// One CTA: tile blockIdx.x % tiles, chunk group blockIdx.x / tiles.
__global__ void __launch_bounds__(PS_THREADS, 1) k_pcg_apply_st(const PsArgs a) {
    extern __shared__ __align__(16) unsigned char psm[];
    float4 *Zs = reinterpret_cast<float4 *>(psm);                       // PS_CG x PS_HA x PS_HB x PS_HC
    __shared__ int soff[8 * PS_KMAX];
    __shared__ float csum[PS_WARPS][PS_CG * 4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x % a.tiles, grp = blockIdx.x / a.tiles;
    const int q0 = grp * PS_CG, nq = min(PS_CG, a.nchunks - q0);
    const int ta = tile / (a.tB * a.tC), tb = (tile / a.tC) % a.tB, tc = tile % a.tC;
    const int A0 = 1 + ta * PS_TA, B0 = 1 + tb * PS_TB, C0 = 1 + tc * PS_TC;   // tile origin (full coordinates)
    for (int i = tid; i < 8 * PS_KMAX; i += blockDim.x) soff[i] = a.off[i];
    for (int i = tid; i < PS_WARPS * PS_CG * 4; i += blockDim.x) (&csum[0][0])[i] = 0.f;
    // stage Z (the group's chunks) for the tile and its halo; positions off the interior are 0
    // (rows of PS_HC positions along C; each thread takes every blockDim.x-th item, four at a
    // time with all four loads issued before the stores)
    const int hsz = PS_HA * PS_HB * PS_HC;
    const int items = nq * hsz;
    for (int i0 = tid; i0 < items; i0 += 4 * (int)blockDim.x) {
        float4 v[4];
        int dsti[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            dsti[u] = -1;
            if (i < items) {
                const int q = i / hsz, rem = i - q * hsz;
                const int hab = rem / PS_HC, hc = rem - hab * PS_HC;
                const int ha = hab / PS_HB, hb = hab - ha * PS_HB;
                const int A = A0 - 2 + ha, B = B0 - 2 + hb, C = C0 - 2 + hc;
                dsti[u] = q * hsz + hidx(ha, hb, hc);
                if (A >= 1 && A <= a.Lx - 2 && B >= 1 && B <= a.Ly - 2 && C >= 1 && C <= a.Lz - 2) {
                    const int64_t r = ((int64_t)(A - 1) * a.ny + (B - 1)) * a.nz + (C - 1);
                    v[u] = __ldg(reinterpret_cast<const float4 *>(a.Z) + ((int64_t)(q0 + q) * a.ns + r));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (dsti[u] >= 0) Zs[dsti[u]] = v[u];
    }
    __syncthreads();
    // work items: (type, A line, B line) of the tile, 32 nodes of the type along C each
    for (int item = warp; item < 8 * 4; item += PS_WARPS) {
        const int t = item >> 2, la = (item >> 1) & 1, lb = item & 1;
        const int pa = (t >> 2) & 1, pb = (t >> 1) & 1, pcp = t & 1;
        const int A = A0 + ((pa - A0) & 1) + 2 * la, B = B0 + ((pb - B0) & 1) + 2 * lb;
        const int e0 = (pcp - C0) & 1, C = C0 + e0 + 2 * lane;
        const bool real = A <= a.Lx - 2 && B <= a.Ly - 2 && C <= a.Lz - 2;
        const int64_t nt = (int64_t)a.dims[t][0] * a.dims[t][1] * a.dims[t][2];
        const int64_t it = real ? ((int64_t)((A - a.first[t][0]) / 2) * a.dims[t][1] + (B - a.first[t][1]) / 2) *
                                          a.dims[t][2] + (C - a.first[t][2]) / 2
                                : 0;
        const float *Lt = a.L + a.base[t] + it, *Bt = a.B + a.base[t] + it;
        const int ha = A - A0 + 2, hb = B - B0 + 2, hc = C - C0 + 2;
        float aL[PS_CG][4], aB[PS_CG][4];
#pragma unroll
        for (int q = 0; q < PS_CG; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i) { aL[q][i] = 0.f; aB[q][i] = 0.f; }
        if (real) {
            const int K = a.K[t];
            // the values of four offsets are loaded before their products, so four pairs of
            // global loads are in flight per lane; the offsets' products keep the slot order
            for (int k0 = 0; k0 < K; k0 += 4) {
                float vl[4], vb[4];
                int h[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + u < K ? k0 + u : K - 1;
                    vl[u] = __ldg(Lt + (int64_t)k * nt);
                    vb[u] = __ldg(Bt + (int64_t)k * nt);
                    const int o = soff[t * PS_KMAX + k];
                    h[u] = hidx(ha + o / 25 - 2, hb + (o / 5) % 5 - 2, hc + o % 5 - 2);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (k0 + u >= K) break;
#pragma unroll
                    for (int q = 0; q < PS_CG; ++q) {
                        if (q >= nq) break;
                        const float4 x = Zs[q * hsz + h[u]];
                        aL[q][0] = fmaf(vl[u], x.x, aL[q][0]); aL[q][1] = fmaf(vl[u], x.y, aL[q][1]);
                        aL[q][2] = fmaf(vl[u], x.z, aL[q][2]); aL[q][3] = fmaf(vl[u], x.w, aL[q][3]);
                        aB[q][0] = fmaf(vb[u], x.x, aB[q][0]); aB[q][1] = fmaf(vb[u], x.y, aB[q][1]);
                        aB[q][2] = fmaf(vb[u], x.z, aB[q][2]); aB[q][3] = fmaf(vb[u], x.w, aB[q][3]);
                    }
                }
            }
        }
        // own rows: P <- Z + beta P, Q <- (L/2 - shift B) Z + beta Q; column sums P.Q
        const int64_t r = real ? ((int64_t)(A - 1) * a.ny + (B - 1)) * a.nz + (C - 1) : 0;
        const int h0 = hidx(ha, hb, hc);
#pragma unroll
        for (int q = 0; q < PS_CG; ++q) {
            if (q >= nq) break;
            const int c0 = (q0 + q) * 4;
            float contrib[4] = {0.f, 0.f, 0.f, 0.f};
            if (real) {
                const float4 z4 = Zs[q * hsz + h0];
                const float zr[4] = {z4.x, z4.y, z4.z, z4.w};
                const int64_t o = ((int64_t)(q0 + q) * a.ns + r) << 2;
                float pr[4] = {0.f, 0.f, 0.f, 0.f}, qr[4] = {0.f, 0.f, 0.f, 0.f};
                if (!a.first_it) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(a.P + o);
                    const float4 q4 = *reinterpret_cast<const float4 *>(a.Q + o);
                    pr[0] = p4.x; pr[1] = p4.y; pr[2] = p4.z; pr[3] = p4.w;
                    qr[0] = q4.x; qr[1] = q4.y; qr[2] = q4.z; qr[3] = q4.w;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sh = (float)a.shift[c0 + i];
                    const float bt = a.first_it ? 0.f : (float)a.beta[c0 + i];
                    const float tz = 0.5f * aL[q][i] - sh * aB[q][i];
                    pr[i] = a.first_it ? zr[i] : fmaf(bt, pr[i], zr[i]);
                    qr[i] = a.first_it ? tz : fmaf(bt, qr[i], tz);
                    contrib[i] = pr[i] * qr[i];
                }
                *reinterpret_cast<float4 *>(a.P + o) = make_float4(pr[0], pr[1], pr[2], pr[3]);
                *reinterpret_cast<float4 *>(a.Q + o) = make_float4(qr[0], qr[1], qr[2], qr[3]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float s = warp_sum_f(contrib[i]);
                if (lane == 0) csum[warp][q * 4 + i] += s;     // this warp's items in order
            }
        }
    }
    __syncthreads();
    // the tile's partial per column: the warps' sums added in warp order
    for (int j = tid; j < nq * 4; j += blockDim.x) {
        float s = 0.f;
        for (int wp = 0; wp < PS_WARPS; ++wp) s += csum[wp][j];
        a.part[(int64_t)(q0 * 4 + j) * a.tiles + tile] = (double)s;
    }
}

}  // namespace

bool launch_pcg_apply_st(ofks_ctx *c, int w, int pc, const float *Zc, float *P, float *Q, const double *beta_col,
                         const double *shift, int first) {
    const PcgStencil &S = c->ps;
    if (!S.on || !c->prm.pcg_stencil || w % 4) return false;
    PsArgs a;
    a.Lx = S.Lx; a.Ly = S.Ly; a.Lz = S.Lz; a.ny = S.Ly - 2; a.nz = S.Lz - 2;
    a.ns = c->n_slots;
    a.nchunks = w / 4;
    a.ngroups = (a.nchunks + PS_CG - 1) / PS_CG;
    a.tA = (S.Lx - 2 + PS_TA - 1) / PS_TA;
    a.tB = (S.Ly - 2 + PS_TB - 1) / PS_TB;
    a.tC = (S.Lz - 2 + PS_TC - 1) / PS_TC;
    a.tiles = a.tA * a.tB * a.tC;
    if ((int64_t)a.tiles * w > c->cpart_cap) return false;
    a.pc = pc;
    for (int t = 0; t < 8; ++t) {
        a.K[t] = S.K[t];
        a.base[t] = S.base[t];
        for (int d = 0; d < 3; ++d) { a.first[t][d] = S.first[t][d]; a.dims[t][d] = S.dims[t][d]; }
    }
    a.off = S.d_off; a.L = S.d_L; a.B = S.d_B;
    a.Z = Zc; a.P = P; a.Q = Q; a.beta = beta_col; a.shift = shift; a.part = c->d_cpart;
    a.first_it = first;
    const int smem = PS_CG * PS_HA * PS_HB * PS_HC * (int)sizeof(float4);
    cudaFuncSetAttribute(k_pcg_apply_st, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_pcg_apply_st<<<(unsigned)(a.tiles * a.ngroups), PS_THREADS, smem, c->stream>>>(a);
    c->kernels += 1;
    c->pq_units = a.tiles;
    return true;
}
