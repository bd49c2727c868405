// C ABI of libofks: context, parameters, orbitals and the PCAL driver (paper Alg. 2).
//
// One iteration at X^k (all on the context's stream, no host arithmetic):
//   density rho(X) -> Hartree CG -> potentials + H refresh          (Sec. 2.2, Eq. hamiltonian)
//   H X (SELL SpMM); Lambda0 = X^T H X, S = X^T B X                  (Eq. multi)
//   Lambda (Eq. lambda2), C = beta (S - I) - Lambda, E, fea
//   G = H X + B X C, kkt = ||H X - B X Lambda0||_F                   (Eq. PLAM-main, Sec. 4.1)
//   stopping test (kkt + fea)/kkt0 < tol                             (Sec. 4.1)
//   D = T^{-1} G by Jacobi-PCG per column (Eq. precondition-T)
//   eta by BB (Sec. 4.4); Y = X - D/eta; B Y with column norms; X <- Y/||Y||_B (Eq. PCAL-main)
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

static const char *kPfNames[PF_COUNT] = {"density", "poisson", "potential", "spmm_h", "gram", "small",
                                         "grad", "pcg_spmm", "pcg_update", "bb", "step", "spmm_b", "other",
                                         "poisson_spmv", "gcn", "poisson_vec", "poisson_pc", "pcg_sep",
                                         "judge"};

int ofks_fail(ofks_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int ofks_cuda_check(ofks_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return OFKS_OK;
    return ofks_fail(c, OFKS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static cudaEvent_t ev_get(ofks_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(ofks_ctx *c, int, cudaEvent_t *a, cudaEvent_t *b) {
    if (!c->prof) return;
    *a = ev_get(c);
    *b = ev_get(c);
    cudaEventRecord(*a, c->stream);
}

void prof_end(ofks_ctx *c, int fam, cudaEvent_t a, cudaEvent_t b) {
    if (!c->prof || !a) return;
    cudaEventRecord(b, c->stream);
    c->prof_pending.push_back({fam, {a, b}});
}

static void prof_resolve(ofks_ctx *c) {
    if (c->prof_pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &pe : c->prof_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
        c->prof_n[pe.first]++;
        c->prof_ms[pe.first] += ms;
        c->ev_pool.push_back(pe.second.first);
        c->ev_pool.push_back(pe.second.second);
    }
    c->prof_pending.clear();
}

template <class T>
static void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

template <class T>
static void free_set(Blocks<T> &b) {
    for (int i = 0; i < 2; ++i) { dfree(b.X[i]); dfree(b.D[i]); dfree(b.G[i]); }
    dfree(b.HX); dfree(b.BX); dfree(b.R); dfree(b.Z); dfree(b.P); dfree(b.Q); dfree(b.W); dfree(b.Dc);
    dfree(b.valL); dfree(b.valB); dfree(b.valH);
}

void clear_graphs(ofks_ctx *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

int run_graph(ofks_ctx *c, const std::vector<int64_t> &key, void (*body)(void *), void *arg) {
    if (c->prof || !c->prm.cuda_graphs) {
        body(arg);
        return OFKS_OK;
    }
    for (auto &g : c->graphs)
        if (g.key == key) {
            c->kernels += g.kernels;
            return ofks_cuda_check(c, cudaGraphLaunch(g.exec, c->stream), "graph launch");
        }
    const int64_t k0 = c->kernels;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        body(arg);
        return OFKS_OK;
    }
    body(arg);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    const int64_t nk = c->kernels - k0;
    c->kernels = k0;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {                       // nothing of the capture ran: launch directly
        cudaGetLastError();
        body(arg);
        return OFKS_OK;
    }
    c->graphs.push_back({key, exec, nk});
    c->kernels += nk;
    return ofks_cuda_check(c, cudaGraphLaunch(exec, c->stream), "graph launch");
}

static void free_blocks(ofks_ctx *c) {
    clear_graphs(c);
    free_set(c->b64);
    free_set(c->b32);
    dfree(c->d_L0); dfree(c->d_S); dfree(c->d_Lam); dfree(c->d_C); dfree(c->d_colA); dfree(c->d_pp); dfree(c->d_stage);
    dfree(c->d_cpart);
    dfree(c->d_gmap);
    c->cpart_cap = 0;
    dfree(c->d_colC); dfree(c->d_cmap);
    c->p = c->ld = 0;
    c->have_X = c->evaluated = c->have_prev = false;
    c->phase = 64;
}

template <class T>
static int alloc_set(ofks_ctx *c, Blocks<T> &b, int ld, bool values) {
    // rows: n, or the float32 PCG's row stride (n rounded up to 32) when larger
    const size_t blk = sizeof(T) * (size_t)std::max<int64_t>(c->n, c->n_slots) * ld;
    T **bl[] = {&b.X[0], &b.X[1], &b.D[0], &b.D[1], &b.G[0], &b.G[1], &b.HX, &b.BX, &b.R, &b.Z, &b.P, &b.Q, &b.W,
                &b.Dc};
    for (T **q : bl) {
        if (cudaMalloc((void **)q, blk) != cudaSuccess)
            return ofks_fail(c, OFKS_ENOMEM, "cannot allocate %zu bytes for an n x p block", blk);
        cudaMemsetAsync(*q, 0, blk, c->stream);
    }
    if (values) {
        const size_t vb = sizeof(T) * (size_t)std::max<int64_t>(c->sell_len, 1);
        if (cudaMalloc((void **)&b.valL, vb) != cudaSuccess || cudaMalloc((void **)&b.valB, vb) != cudaSuccess ||
            cudaMalloc((void **)&b.valH, vb) != cudaSuccess)
            return ofks_fail(c, OFKS_ENOMEM, "cannot allocate the float32 matrix values");
        launch_convert(c, c->d_valL, b.valL, c->sell_len);
        launch_convert(c, c->d_valB, b.valB, c->sell_len);
        launch_convert(c, c->d_valH, b.valH, c->sell_len);
    }
    return OFKS_OK;
}

static int alloc_blocks(ofks_ctx *c, int p, bool mixed) {
    free_blocks(c);
    const int ld = (p <= 2) ? p : (p + 3) / 4 * 4;
    const size_t sm = sizeof(double) * (size_t)ld * ld;
    int rc = alloc_set(c, c->b64, ld, false);
    if (!rc && mixed) rc = alloc_set(c, c->b32, ld, true);
    if (rc) { free_blocks(c); return rc; }
    double **sl[] = {&c->d_L0, &c->d_S, &c->d_Lam, &c->d_C};
    for (double **b : sl) {
        if (cudaMalloc((void **)b, sm) != cudaSuccess) { free_blocks(c); return ofks_fail(c, OFKS_ENOMEM, "p x p"); }
        cudaMemsetAsync(*b, 0, sm, c->stream);
    }
    if (cudaMalloc((void **)&c->d_colA, sizeof(double) * CB_COUNT * ld) != cudaSuccess ||
        cudaMalloc((void **)&c->d_colC, sizeof(double) * CB_COUNT * ld) != cudaSuccess ||
        cudaMalloc((void **)&c->d_cmap, sizeof(int) * 2 * ld) != cudaSuccess ||
        cudaMalloc((void **)&c->d_gmap, sizeof(int) * ld) != cudaSuccess ||
        cudaMalloc((void **)&c->d_pp, sm * 8 + sizeof(double) * ld) != cudaSuccess) {
        free_blocks(c);
        return ofks_fail(c, OFKS_ENOMEM, "p x p scratch");
    }
    cudaMemsetAsync(c->d_colA, 0, sizeof(double) * CB_COUNT * ld, c->stream);
    if (ld != p && cudaMalloc((void **)&c->d_stage, sizeof(double) * (size_t)c->n * p) != cudaSuccess) {
        free_blocks(c);
        return ofks_fail(c, OFKS_ENOMEM, "host-copy staging block");
    }
    // per-column partials: one per (column, slice group) for the SELL kernels (at most one group
    // per slice), and room for the Grams' per-split tiles
    c->cpart_cap = std::max<int64_t>((int64_t)ld * (std::max<int64_t>(c->n_slices, c->n_tslices) + 64),
                                     CPART_MIN);
    if (cudaMalloc((void **)&c->d_cpart, sizeof(double) * (size_t)c->cpart_cap) != cudaSuccess) {
        free_blocks(c);
        return ofks_fail(c, OFKS_ENOMEM, "reduction partials");
    }
    c->p = p;
    c->ld = ld;
    c->mixed_alloc = mixed;
    return ofks_cuda_check(c, cudaStreamSynchronize(c->stream), "block allocation");
}

// copy the iteration state between the float32 and float64 sets (X, previous X, D, G, B X)
template <class S, class T>
static void copy_state(ofks_ctx *c, Blocks<S> &a, Blocks<T> &b) {
    const int64_t cnt = c->n * (int64_t)c->ld;
    for (int i = 0; i < 2; ++i) {
        launch_convert(c, a.X[i], b.X[i], cnt);
        launch_convert(c, a.D[i], b.D[i], cnt);
        launch_convert(c, a.G[i], b.G[i], cnt);
    }
    launch_convert(c, a.BX, b.BX, cnt);
    launch_convert(c, a.HX, b.HX, cnt);
}

// the float64 set holds the current state (after float32 iterations it is stale)
static void state_to64(ofks_ctx *c) {
    if (c->phase == 32) copy_state(c, c->b32, c->b64);
}

// entering float32 iterations from the float64 set
static void state_to32(ofks_ctx *c) {
    if (c->phase == 32) copy_state(c, c->b64, c->b32);
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Host blocks are dense n x p; device blocks have row pitch ld.  With ld > p the copy goes as
// one contiguous transfer through the staging block and a repacking kernel: a pitched copy of
// n rows of p doubles runs far below the link's bandwidth.
static int upload_block(ofks_ctx *c, const double *h, double *d) {
    const size_t bytes = sizeof(double) * (size_t)c->n * c->p;
    if (c->ld == c->p)
        return ofks_cuda_check(c, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream), "block upload");
    cudaError_t e = cudaMemcpyAsync(c->d_stage, h, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) launch_repack(c, c->d_stage, c->p, d, c->ld, c->n, c->p);
    return ofks_cuda_check(c, e, "block upload");
}

static int download_block(ofks_ctx *c, const double *d, double *h) {
    const size_t bytes = sizeof(double) * (size_t)c->n * c->p;
    const double *src = d;
    if (c->ld != c->p) {
        launch_repack(c, d, c->ld, c->d_stage, c->p, c->n, c->p);
        src = c->d_stage;
    }
    cudaError_t e = cudaMemcpyAsync(h, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return ofks_cuda_check(c, e, "block download");
}

static int read_flag(ofks_ctx *c, int *h) {
    cudaError_t e = cudaMemcpyAsync(h, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
    return ofks_cuda_check(c, e, "status flag");
}

// ------------------------------------------------------------------------------ iteration
struct Rec { double E, fea, kkt, eta; };

template <class T> static const T *vals_L(ofks_ctx *c);
template <> const double *vals_L<double>(ofks_ctx *c) { return c->d_valL; }
template <> const float *vals_L<float>(ofks_ctx *c) { return c->b32.valL; }
template <class T> static const T *vals_B(ofks_ctx *c);
template <> const double *vals_B<double>(ofks_ctx *c) { return c->d_valB; }
template <> const float *vals_B<float>(ofks_ctx *c) { return c->b32.valB; }
template <class T> static T *vals_H(ofks_ctx *c);
template <> double *vals_H<double>(ofks_ctx *c) { return c->d_valH; }
template <> float *vals_H<float>(ofks_ctx *c) { return c->b32.valH; }
template <class T> static Blocks<T> &blocks(ofks_ctx *c);
template <> Blocks<double> &blocks<double>(ofks_ctx *c) { return c->b64; }
template <> Blocks<float> &blocks<float>(ofks_ctx *c) { return c->b32; }

template <class T>
static int evaluate_t(ofks_ctx *c, bool need_bx, Rec *out) {
    Blocks<T> &b = blocks<T>(c);
    T *X = b.X[c->cur];
    int rc;
    if ((rc = launch_density(c, X))) return rc;
    if ((rc = run_hartree(c))) return rc;
    if ((rc = launch_potential_refresh(c, vals_H<T>(c), vals_L<T>(c)))) return rc;
    {
        ProfScope ps(c, PF_SPMM_H);
        launch_sell_spmm(c, (const T *)vals_H<T>(c), (const T *)X, b.HX);
    }
    if (need_bx) {
        ProfScope ps(c, PF_SPMM_B);
        launch_sell_spmm(c, vals_B<T>(c), (const T *)X, b.BX);
    }
    launch_gram2(c, (const T *)X, (const T *)b.HX, (const T *)b.BX, c->d_L0, c->d_S);
    launch_small_update(c);
    launch_grad_update(c, b);
    launch_small_record(c);
    double h[4];
    int tc_flag = 0;                             // a tensor-core Gram or gradient whose bounded wait gave up
    cudaError_t e = cudaMemcpyAsync(h, c->d_rec, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tc_flag, c->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if ((rc = ofks_cuda_check(c, e, "evaluate"))) return rc;
    if (tc_flag) {
        e = cudaMemsetAsync(c->d_flag + 2, 0, sizeof(int), c->stream);
        if ((rc = ofks_cuda_check(c, e, "evaluate"))) return rc;
        c->evaluated = false;
        return ofks_fail(c, OFKS_ETIMEOUT, "tensor-core Gram or gradient: a bounded wait timed out");
    }
    out->E = h[0]; out->fea = h[1]; out->kkt = h[2];
    c->evaluated = true;
    c->last_E = h[0]; c->last_fea = h[1]; c->last_kkt = h[2];
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !std::isfinite(h[2]))
        return ofks_fail(c, OFKS_ENONFINITE, "non-finite iterate record: E=%g fea=%g kkt=%g", h[0], h[1], h[2]);
    return OFKS_OK;
}

static int evaluate(ofks_ctx *c, bool need_bx, Rec *out) {
    return c->phase == 32 ? evaluate_t<float>(c, need_bx, out) : evaluate_t<double>(c, need_bx, out);
}

template <class T>
static int precondition_t(ofks_ctx *c) {
    Blocks<T> &b = blocks<T>(c);
    const int ld = c->ld;
    T *D = b.D[c->cur], *G = b.G[c->cur];
    if (c->prm.precond == OFKS_PC_NONE) {
        return ofks_cuda_check(c, cudaMemcpyAsync(D, G, sizeof(T) * c->n * ld, cudaMemcpyDeviceToDevice, c->stream),
                               "direction copy");
    }
    const bool learned = c->prm.precond == OFKS_PC_LEARNED;
    // the network runs unless it sits out a pause after calls in which the judge took none of its
    // directions (the PCG then does all the work, and the network's cost is not repaid)
    if (c->prm.learned_retry == 0) c->gcn_skip = 0;
    const bool net = learned && c->gcn_skip == 0;
    if (learned && !net) c->gcn_skip--;
    PcgView<T> v;
    v.w = ld; v.pc = c->p; v.cb = c->d_colA; v.D = D;
    std::vector<double> act0(ld), sh0(ld);
    cudaMemcpyAsync(act0.data(), c->d_colA + CB_ACTIVE * ld, sizeof(double) * ld, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(sh0.data(), c->d_colA + CB_SHIFT * ld, sizeof(double) * ld, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e0 = cudaStreamSynchronize(c->stream);
    if (e0 != cudaSuccess) return ofks_cuda_check(c, e0, "preconditioner");
    int nact = 0;
    for (int j = 0; j < c->p; ++j) nact += act0[j] != 0.0;
    c->last_active = nact;
    c->active_total += nact;
    if (nact == 0) {                 // every T is I (Eq. precondition-T): D = G, no system is solved
        ProfScope ps(c, PF_PCG_UPDATE);
        launch_direction_select(c, b);
        return ofks_cuda_check(c, cudaGetLastError(), "preconditioner");
    }
    // the PCG runs on a compact block of the columns that need it, of width w: the active columns
    // (the columns are independent systems, so the others' work would only be discarded), or in
    // the learned mode those the judge did not accept
    auto compact_view = [&](const std::vector<int> &cols, const std::vector<int> &cpos) -> int {
        const int m = (int)cols.size();
        const int w = m <= 2 ? m : (m + 3) / 4 * 4;
        std::vector<int> h(2 * (size_t)ld, -1);                // cmap | cpos
        for (int k = 0; k < m; ++k) h[k] = cols[k];
        for (int j = 0; j < ld; ++j) h[ld + j] = cpos[j];
        cudaError_t e = cudaMemcpyAsync(c->d_cmap, h.data(), sizeof(int) * 2 * ld, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // h leaves scope
        if (e != cudaSuccess) return ofks_cuda_check(c, e, "preconditioner");
        launch_pcg_compact_cols(c, w, m, c->d_cmap, c->d_colC);
        v.w = w; v.pc = m; v.cb = c->d_colC;
        v.cmap = c->d_cmap; v.cpos = c->d_cmap + ld; v.D = b.Dc;
        return OFKS_OK;
    };
    bool run_pcg = true, warm = false;
    if (!net) {
        const int w = nact <= 2 ? nact : (nact + 3) / 4 * 4;
        if (c->prm.pcg_compact && w < ld) {
            std::vector<int> cols, cpos(ld, -1);
            for (int j = 0; j < c->p; ++j)
                if (act0[j] != 0.0) { cpos[j] = (int)cols.size(); cols.push_back(j); }
            if (int rc = compact_view(cols, cpos)) return rc;
        } else if (pcg_zc<T>(c, ld)) {                        // float32 blocks chunk-major
            std::vector<int> h(2 * (size_t)ld, -1);            // all columns; inactive ones take G
            for (int j = 0; j < ld; ++j) h[j] = j;
            for (int j = 0; j < c->p; ++j) h[ld + j] = act0[j] != 0.0 ? j : -1;
            cudaError_t e = cudaMemcpyAsync(c->d_cmap, h.data(), sizeof(int) * 2 * ld, cudaMemcpyHostToDevice,
                                            c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return ofks_cuda_check(c, e, "preconditioner");
            v.cmap = c->d_cmap; v.cpos = c->d_cmap + ld; v.D = b.Dc;
        }
    } else {
        // D = network(G) on the active columns; each is judged by its residual against the PCG's
        // own measure, |G - T D|_{M^-1} / |G|_{M^-1} (M the Jacobi diagonal of T), and by the sign
        // of G.D: accepted columns keep the network's D; the others run the PCG, started from the
        // network's D where that residual is below 1 (a better start than zero), else from zero
        if (!c->gcn.H) return ofks_fail(c, OFKS_ESTATE, "learned preconditioner: no network (ofks_precond_init)");
        int rc;
        if ((rc = gcn_forward_prepare(c))) return rc;
        std::vector<int> gmap;
        std::vector<double> gsh;
        for (int j = 0; j < c->p; ++j)
            if (act0[j] != 0.0) { gmap.push_back(j); gsh.push_back(sh0[j]); }
        if (!c->d_shift_in && cudaMalloc((void **)&c->d_shift_in, sizeof(double) * 256) != cudaSuccess)
            return ofks_fail(c, OFKS_ENOMEM, "shift buffer");
        cudaError_t eg = cudaMemcpyAsync(c->d_gmap, gmap.data(), sizeof(int) * gmap.size(), cudaMemcpyHostToDevice,
                                         c->stream);
        if (eg == cudaSuccess)
            eg = cudaMemcpyAsync(c->d_shift_in, gsh.data(), sizeof(double) * gsh.size(), cudaMemcpyHostToDevice,
                                 c->stream);
        if (eg == cudaSuccess) eg = cudaStreamSynchronize(c->stream);      // gmap, gsh leave scope
        if (eg != cudaSuccess) return ofks_cuda_check(c, eg, "learned preconditioner columns");
        c->gcn.cols = (int)gmap.size();
        gcn_pack<T>(c, G, c->gcn.G32, c->d_gmap);
        rc = gcn_forward(c, c->d_shift_in, false);
        if (!rc) gcn_unpack<T>(c, c->gcn.Dn, D, c->d_gmap);
        c->gcn.cols = 0;
        if (rc) return rc;
        c->learned_calls++;
        {
            // the network's directions judged: T D on every column, then the residual sums
            ProfScope ps(c, PF_JUDGE);
            launch_pcg_apply(c, vals_L<T>(c), vals_B<T>(c), (const T *)D, 0, b.P, b.Q, c->d_colA + CB_BETA * ld,
                             c->d_colA + CB_SHIFT * ld, c->d_colA + CB_PQ * ld, 1, ld, c->p);
            launch_judge(c, b);
        }
        std::vector<double> h(3 * (size_t)ld);
        cudaMemcpyAsync(h.data(), c->d_colA + CB_RZ * ld, sizeof(double) * 3 * ld, cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ofks_cuda_check(c, e, "learned preconditioner judge");
        std::vector<int> cols, cpos(ld, -1);
        std::vector<double> warmv(ld, 0.0);
        int accepted = 0, nwarm = 0;
        for (int j = 0; j < c->p; ++j) {
            if (act0[j] == 0.0) continue;                  // T = I column: D = G
            const double rr = h[j], gg = h[ld + j], gd = h[2 * ld + j];
            const double ratio = gg > 0.0 ? std::sqrt(rr / gg) : 1e300;
            const bool ok = gd > 0.0 && ratio <= c->prm.judge_tau;
            c->judge_total++;
            if (ok) {
                cpos[j] = -2;
                ++accepted;
                continue;
            }
            cpos[j] = (int)cols.size();
            cols.push_back(j);
            if (ratio < 1.0) { warmv[j] = 1.0; ++nwarm; }
        }
        c->judge_accept += accepted;
        c->learned_warm += nwarm;
        if (accepted == 0) {              // the PCG does all the work: pause the network
            if (c->prm.learned_retry > 0) {
                c->gcn_backoff = std::min(c->prm.learned_retry, std::max(1, 2 * c->gcn_backoff));
                c->gcn_skip = c->gcn_backoff;
            }
        } else {
            c->gcn_backoff = 0;
        }
        run_pcg = !cols.empty();
        if (run_pcg) {
            cudaMemcpyAsync(c->d_colA + CB_WARM * ld, warmv.data(), sizeof(double) * ld, cudaMemcpyHostToDevice,
                            c->stream);
            if ((rc = compact_view(cols, cpos))) return rc;   // synchronizes: warmv may leave scope
            warm = nwarm > 0;
        }
    }
    const bool sep = c->prm.pcg_pc == OFKS_PCGPC_SEPARABLE;
    if (run_pcg) {
        {
            ProfScope ps(c, PF_PCG_UPDATE);
            launch_pcg_init(c, b, v, warm);
            cudaMemsetAsync(v.cb + CB_PQ * v.w, 0, sizeof(double) * v.w, c->stream);
        }
        if (sep) {     // Z = T_sep^-1 R replaces the Jacobi start's Z and r.z
            ProfScope ps(c, PF_PCG_SEP);
            if (launch_pcg_sep(c, b, v)) launch_col_fin(c, v.pc, v.w, c->rz_units, c->d_cpart, v.cb + CB_RZ * v.w);
        }
    }
    const bool exact = c->prm.precond == OFKS_PC_EXACT;
    const int max_it = !run_pcg ? 0 : exact ? 5000 : c->prm.pcg_iters;
    const int w = v.w;
    std::vector<double> rz0, rz(w), act(w);
    if (exact) {
        rz0.resize(w);
        cudaMemcpyAsync(rz0.data(), v.cb + CB_RZ * w, sizeof(double) * w, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(act.data(), v.cb + CB_ACTIVE * w, sizeof(double) * w, cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
    }
    // one PCG iteration: T P (with the P, Q updates), alpha, D/R/Z update, beta
    struct Loop { ofks_ctx *c; Blocks<T> *b; PcgView<T> v; int it0, it1, max_it; bool exact; };
    auto iterate_pcg = [](void *a) {
        Loop &L = *static_cast<Loop *>(a);
        ofks_ctx *c = L.c;
        Blocks<T> &b = *L.b;
        const PcgView<T> &v = L.v;
        const int w = v.w;
        for (int it = L.it0; it < L.it1; ++it) {
            {
                ProfScope ps(c, PF_PCG_SPMM);
                launch_pcg_apply(c, vals_L<T>(c), vals_B<T>(c), (const T *)b.Z, pcg_zc<T>(c, w) ? 1 : 0, b.P, b.Q,
                                 v.cb + CB_BETA * w, v.cb + CB_SHIFT * w, v.cb + CB_PQ * w, it == 0 ? 1 : 0, w, v.pc);
            }
            const bool last = !L.exact && it + 1 == L.max_it;
            {
                ProfScope ps(c, PF_PCG_UPDATE);
                launch_pcg_alpha(c, w, v.pc, v.cb);
                launch_pcg_update(c, b, v, last);
            }
            if (!last && c->prm.pcg_pc == OFKS_PCGPC_SEPARABLE) {
                ProfScope ps(c, PF_PCG_SEP);
                launch_pcg_sep(c, b, v);          // Z and r.z of the separable preconditioner
            }
            {
                ProfScope ps(c, PF_PCG_UPDATE);
                launch_pcg_beta(c, w, v.pc, v.cb);
            }
        }
    };
    if (!exact && max_it > 0) {                  // the fixed-count loop: one graph per shape
        Loop L{c, &b, v, 0, max_it, max_it, false};
        const std::vector<int64_t> key = {1, (int64_t)sizeof(T), w, v.pc, max_it, (int64_t)(uintptr_t)v.cb,
                                          (int64_t)(uintptr_t)v.D, (int64_t)(uintptr_t)b.Z, c->prm.pcg_pc,
                                          (int64_t)(uintptr_t)c->sep.pbuf};
        int rc;
        if ((rc = run_graph(c, key, iterate_pcg, &L))) return rc;
        c->pcg_cols_total += (int64_t)w * max_it;
    }
    for (int it = 0; exact && it < max_it; ++it) {
        Loop L{c, &b, v, it, it + 1, max_it, true};
        iterate_pcg(&L);
        c->pcg_cols_total += w;
        if ((it + 1) % 25 == 0) {
            cudaMemcpyAsync(rz.data(), v.cb + CB_RZ * w, sizeof(double) * w, cudaMemcpyDeviceToHost, c->stream);
            cudaStreamSynchronize(c->stream);
            bool done = true;
            for (int j = 0; j < v.pc; ++j)
                if (act[j] != 0.0 && rz[j] > 1e-24 * rz0[j]) done = false;
            if (done) break;
        }
    }
    {
        ProfScope ps(c, PF_PCG_UPDATE);
        // a PCG that ran into Dc comes back through the column map; without a PCG (every column
        // of the learned mode accepted) D holds the network's directions and the T = I columns take G
        if (v.cpos && run_pcg) launch_direction_expand(c, b, v);
        else launch_direction_select(c, b);
    }
    return ofks_cuda_check(c, cudaGetLastError(), "preconditioner");
}

// The direction D = T^{-1} G of Eq. (precondition-T).  In the float64 sweep of the mixed form
// (sweep_pc32) the linear systems are solved by the float32 PCG on the float64 gradient rounded
// to float32, and D is widened back: the preconditioner only shapes the path (any approximate
// T^{-1} leaves the fixed point G = 0 and the float64 stopping test unchanged), and the float64
// PCG is the largest cost of a float64 iteration.
template <class T>
static int direction_t(ofks_ctx *c) {
    if constexpr (sizeof(T) == 8) {
        if (c->prm.precision == OFKS_MIXED && c->mixed_alloc && c->prm.sweep_pc32 &&
            c->prm.precond != OFKS_PC_NONE) {
            const int64_t cnt = c->n * (int64_t)c->ld;
            launch_convert(c, (const double *)c->b64.G[c->cur], c->b32.G[c->cur], cnt);
            c->phase = 32;
            const int rc = precondition_t<float>(c);
            c->phase = 64;
            if (rc) return rc;
            launch_convert(c, (const float *)c->b32.D[c->cur], c->b64.D[c->cur], cnt);
            return ofks_cuda_check(c, cudaGetLastError(), "float32 preconditioner of the float64 sweep");
        }
    }
    return precondition_t<T>(c);
}

template <class T>
static int update_step_t(ofks_ctx *c) {
    Blocks<T> &b = blocks<T>(c);
    const int prv = c->cur ^ 1, ld = c->ld;
    int rc;
    if ((rc = direction_t<T>(c))) return rc;
    launch_bb_dots(c, b, c->prm.eta_rule == OFKS_ETA_BB2_RAW);
    launch_eta(c);
    const int method = c->prm.method;
    // the new iterate goes to the other slot (the current one stays as X^{k-1} for the BB step);
    // MOptQR forms Y and B Y in scratch blocks and writes Y R^{-1}, B Y R^{-1} into place
    T *Y = method == OFKS_METHOD_MOPTQR ? b.W : b.X[prv];
    T *BY = method == OFKS_METHOD_MOPTQR ? b.Q : b.BX;
    {
        ProfScope ps(c, PF_STEP);
        launch_step_y(c, b, Y);
    }
    if (method == OFKS_METHOD_PCAL) {
        // Eq. (PCAL-main): B Y with the column B-norms, then X = Y / ||Y||_B column by column
        cudaMemsetAsync(c->d_colA + CB_NORM * ld, 0, sizeof(double) * ld, c->stream);
        {
            ProfScope ps(c, PF_SPMM_B);
            launch_sell_spmm_colnorm(c, vals_B<T>(c), (const T *)Y, b.BX, c->d_colA + CB_NORM * ld);
        }
        ProfScope ps(c, PF_STEP);
        launch_scale_cols(c, Y, b.BX, c->d_colA + CB_NORM * ld);
    } else {
        {
            ProfScope ps(c, PF_SPMM_B);
            launch_sell_spmm(c, vals_B<T>(c), (const T *)Y, BY);
        }
        if (method == OFKS_METHOD_MOPTQR) {
            // Cholesky-based Gram-Schmidt (Sec. 4.2): Y^T B Y = R^T R, X = Y R^{-1}, B X = B Y R^{-1}
            double *Rinv = c->d_pp + 6 * (size_t)ld * ld, *SY = c->d_pp + 2 * (size_t)ld * ld;
            launch_gram2(c, (const T *)Y, (const T *)BY, (const T *)BY, SY, SY + (size_t)ld * ld);
            launch_cholesky_inv(c, SY, Rinv);
            ProfScope ps(c, PF_STEP);
            launch_block_times_small(c, (const T *)Y, Rinv, b.X[prv]);
            launch_block_times_small(c, (const T *)BY, Rinv, b.BX);
        }
    }
    if ((rc = ofks_cuda_check(c, cudaGetLastError(), "update step"))) return rc;
    if (method == OFKS_METHOD_MOPTQR) {
        int flag = 0;
        if ((rc = read_flag(c, &flag))) return rc;
        if (flag) return ofks_fail(c, OFKS_ENOTCONV, "MOptQR: Y^T B Y is not positive definite");
    }
    double eta;
    cudaError_t e = cudaMemcpyAsync(&eta, c->d_sc + SC_ETA, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if ((rc = ofks_cuda_check(c, e, "update step"))) return rc;
    c->eta = eta;
    c->cur = prv;
    c->have_prev = true;
    c->k++;
    return OFKS_OK;
}

static int update_step(ofks_ctx *c) { return c->phase == 32 ? update_step_t<float>(c) : update_step_t<double>(c); }

static int run_iterations(ofks_ctx *c, int kmax, ofks_result *res) {
    if (!c->have_X) return ofks_fail(c, OFKS_ESTATE, "no orbitals: call ofks_init_orbitals first");
    cudaEvent_t e0 = ev_get(c), e1 = ev_get(c);
    c->cg_total = 0;
    cudaEventRecord(e0, c->stream);
    int rc = OFKS_OK;
    for (int it = 0; it < kmax && !c->converged; ++it) {
        Rec r{};
        // inexact Hartree potentials while far from stationarity (tightens to poisson_tol)
        c->hartree_tol = 0.0;
        if (c->prm.poisson_adaptive)
            c->hartree_tol = (c->k == 0 || !(c->kkt0 > 0)) ? 1e-4
                             : std::min(1e-4, 1e-2 * (c->last_kkt + c->last_fea) / c->kkt0);
        if ((rc = evaluate(c, !c->bx_valid, &r))) break;
        c->bx_valid = true;
        if (c->k == 0) c->kkt0 = r.kkt;
        c->history.insert(c->history.end(), {(double)c->k, now_s() - c->t_start, r.E, r.kkt, r.fea, c->eta});
        // float32 iterations hand over at mixed_tol, or once they have stalled below 1e-4: no new
        // best (kkt + fea)/kkt0 within the last 300 iterations (their rounding floor is above
        // mixed_tol on this system)
        const double rel = c->kkt0 > 0 ? (r.kkt + r.fea) / c->kkt0 : 1.0;
        if (c->phase == 32 && (c->k == 0 || rel < c->best_rel)) { c->best_rel = rel; c->best_k = c->k; }
        const bool stalled = c->phase == 32 && c->best_rel < 1e-4 && c->k - c->best_k >= 300;
        if (c->phase == 32 && c->kkt0 > 0 && (rel < c->prm.mixed_tol || stalled)) {
            // float32 iterations have reached their floor: continue with the float64 sweep
            state_to64(c);
            c->phase = 64;
            c->bx_valid = false;
            c->switch_k = c->k;
            c->history.resize(c->history.size() - 6);   // the float64 evaluation replaces this record
            --it;
            continue;
        }
        if (c->kkt0 > 0 && (r.kkt + r.fea) / c->kkt0 < c->prm.tol) { c->converged = true; break; }
        if ((rc = update_step(c))) break;
    }
    c->hartree_tol = 0.0;
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    if (!rc) {   // a tensor-core Gram whose bounded wait gave up
        int hf = 0;
        cudaMemcpy(&hf, c->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost);
        if (hf) {
            cudaMemset(c->d_flag + 2, 0, sizeof(int));
            rc = ofks_fail(c, OFKS_ETIMEOUT, "tensor-core Gram: wait timed out");
        }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->ev_pool.push_back(e0);
    c->ev_pool.push_back(e1);
    if (res) {
        res->e_total = c->last_E; res->e_nuc = c->e_nuc; res->kkt = c->last_kkt; res->fea = c->last_fea;
        res->kkt0 = c->kkt0; res->eta = c->eta; res->iters = c->k; res->converged = c->converged ? 1 : 0;
        res->seconds = ms * 1e-3;
        res->hartree_iters = c->cg_last;
        res->hartree_total = (int32_t)c->cg_total;
        res->switch_iter = c->switch_k;
        res->judge_accept = c->judge_accept;
        res->judge_total = c->judge_total;
        res->active_last = c->last_active;
        res->active_total = c->active_total;
        res->pcg_cols_total = c->pcg_cols_total;
        res->learned_calls = c->learned_calls;
        res->learned_warm = c->learned_warm;
    }
    return rc;
}

// ------------------------------------------------------------------------------ ABI
extern "C" {

void ofks_default_params(ofks_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->p = 1; p->beta = 10.0; p->occ = 2.0; p->tol = 1e-8; p->max_iter = 1000;
    p->precision = OFKS_FP64; p->precond = OFKS_PC_PCG; p->pcg_iters = 8; p->eta_rule = OFKS_ETA_BB2;
    p->eta_fixed = 0.0; p->eta_min = 1e-4; p->eta_max = 1e8; p->hartree = 1; p->xc = 1;
    p->multipole_lmax = 2; p->poisson_tol = 1e-12; p->poisson_max_iter = 20000;
    p->poisson_pc = OFKS_HPC_SEPARABLE;
    p->mixed_tol = 1e-6; p->poisson_tol_mixed = 1e-8;
    p->judge_tau = 0.5; p->learned_tc = 1; p->poisson_adaptive = 0; p->poisson_csr = 0; p->gram_tc = 1;
    p->poisson_sep_tc = 1; p->spmm_f32_rows = 0; p->pcg_compact = 1; p->cuda_graphs = 1;
    p->pcg_staged = 0;
    p->sweep_pc32 = 1;
    p->method = OFKS_METHOD_PCAL;
    p->learned_loss = 1; p->learned_retry = 64; p->pcg_pc = OFKS_PCGPC_JACOBI;
}

int ofks_create(ofks_ctx **out, int device) {
    if (!out) return OFKS_EINVAL;
    *out = nullptr;
    ofks_ctx *c = new (std::nothrow) ofks_ctx();
    if (!c) return OFKS_ENOMEM;
    ofks_default_params(&c->prm);
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_sc, sizeof(double) * SC_COUNT);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_rec, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_flag, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_sc, 0, sizeof(double) * SC_COUNT);
    if (e == cudaSuccess) e = cudaMemset(c->d_rec, 0, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMemset(c->d_flag, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_gpart, sizeof(double) * GACC_CAP);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_gcount, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_gcount, 0, sizeof(unsigned) * 4);
    // device address of the no-allocation staging array, looked up with this device current
    if (e == cudaSuccess) e = static_stage_lookup(c);
    if (e != cudaSuccess) {
        ofks_destroy(c);
        return OFKS_ECUDA;
    }
    *out = c;
    return OFKS_OK;
}

void ofks_destroy(ofks_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_blocks(c);
    free_mesh(c);
    clear_graphs(c);
    dfree(c->d_sc); dfree(c->d_rec); dfree(c->d_flag); dfree(c->d_shift_in); dfree(c->d_gpart); dfree(c->d_gcount);
    for (auto &pe : c->prof_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *ofks_last_error(const ofks_ctx *c) { return c ? c->err.c_str() : "null context"; }

int ofks_set_mesh(ofks_ctx *c, int64_t n_nodes, const double *xyz, int64_t n_tets, const int64_t *tet10,
                  const uint8_t *dirichlet) {
    if (!c) return OFKS_EINVAL;
    cudaSetDevice(c->device);
    free_blocks(c);
    int rc = setup_mesh(c, n_nodes, xyz, n_tets, tet10, dirichlet);
    if (rc) return rc;
    if (c->prm.p > c->n) c->prm.p = 1;
    c->bx_valid = false;
    return alloc_blocks(c, c->prm.p, c->prm.precision == OFKS_MIXED);
}

int ofks_set_nuclei(ofks_ctx *c, int32_t M, const double *Z, const double *R) {
    if (!c) return OFKS_EINVAL;
    if (!c->n) return ofks_fail(c, OFKS_ESTATE, "set_nuclei: no mesh");
    if (M < 1 || !Z || !R) return ofks_fail(c, OFKS_EINVAL, "set_nuclei: need M >= 1 and arrays");
    for (int j = 0; j < M; ++j)
        if (!(Z[j] > 0)) return ofks_fail(c, OFKS_EINVAL, "set_nuclei: Z[%d] must be > 0", j);
    cudaSetDevice(c->device);
    c->evaluated = false;
    return setup_nuclei(c, M, Z, R);
}

int ofks_set_nuclei_static(ofks_ctx *c, int32_t M, const double *Z, const double *R) {
    if (!c) return OFKS_EINVAL;
    if (!c->n) return ofks_fail(c, OFKS_ESTATE, "set_nuclei_static: no mesh");
    if (M < 1 || !Z || !R) return ofks_fail(c, OFKS_EINVAL, "set_nuclei_static: need M >= 1 and arrays");
    if (M > OFKS_STATIC_NUCLEI_MAX)
        return ofks_fail(c, OFKS_EINVAL, "set_nuclei_static: %d nuclei exceed the fixed maximum of %d", M,
                         OFKS_STATIC_NUCLEI_MAX);
    for (int j = 0; j < M; ++j)
        if (!(Z[j] > 0)) return ofks_fail(c, OFKS_EINVAL, "set_nuclei_static: Z[%d] must be > 0", j);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return ofks_cuda_check(c, e, "set_nuclei_static");
    c->evaluated = false;
    return setup_nuclei_static(c, M, Z, R);
}

int ofks_set_params(ofks_ctx *c, const ofks_params *prm) {
    if (!c || !prm) return OFKS_EINVAL;
    if (!c->n) return ofks_fail(c, OFKS_ESTATE, "set_params: no mesh");
    if (prm->p < 1 || prm->p > c->n) return ofks_fail(c, OFKS_EINVAL, "set_params: p=%d outside [1, %lld]", prm->p, (long long)c->n);
    if (prm->p > 256) return ofks_fail(c, OFKS_EINVAL, "set_params: p=%d above the supported 256", prm->p);
    if (!(prm->beta >= 0) || !(prm->occ > 0) || !(prm->tol > 0) || prm->max_iter < 0 || prm->pcg_iters < 0 ||
        prm->eta_rule < 0 || prm->eta_rule > OFKS_ETA_FIXED || prm->precond < 0 || prm->precond > OFKS_PC_LEARNED ||
        !(prm->judge_tau > 0) || prm->learned_tc < 0 || prm->learned_tc > 1 ||
        prm->poisson_adaptive < 0 || prm->poisson_adaptive > 1 ||
        prm->poisson_csr < 0 || prm->poisson_csr > 1 || prm->poisson_sep_tc < 0 || prm->poisson_sep_tc > 1 ||
        prm->spmm_f32_rows < 0 || prm->spmm_f32_rows > 1 || prm->gram_tc < 0 || prm->gram_tc > 1 ||
        prm->pcg_compact < 0 || prm->pcg_compact > 1 || prm->cuda_graphs < 0 || prm->cuda_graphs > 1 ||
        (prm->precision != OFKS_FP64 && prm->precision != OFKS_MIXED) || !(prm->mixed_tol > 0) ||
        !(prm->poisson_tol_mixed > 0) || !(prm->eta_min > 0) || !(prm->eta_max >= prm->eta_min) ||
        prm->multipole_lmax < -1 || prm->multipole_lmax > 2 || !(prm->poisson_tol > 0) ||
        prm->poisson_max_iter < 1 || prm->poisson_pc < 0 || prm->poisson_pc > OFKS_HPC_SEPARABLE || (prm->eta_rule == OFKS_ETA_FIXED && !(prm->eta_fixed > 0)) ||
        prm->method < OFKS_METHOD_PCAL || prm->method > OFKS_METHOD_MOPTQR ||
        prm->learned_loss < 0 || prm->learned_loss > 1 || prm->learned_retry < 0 ||
        prm->pcg_pc < OFKS_PCGPC_JACOBI || prm->pcg_pc > OFKS_PCGPC_SEPARABLE)
        return ofks_fail(c, OFKS_EINVAL, "set_params: a parameter is out of range");
    cudaSetDevice(c->device);
    const bool mixed = prm->precision == OFKS_MIXED;
    const bool realloc = prm->p != c->p || mixed != c->mixed_alloc;
    c->prm = *prm;
    c->converged = false;     // the stop test is taken again, under these parameters, at the next iterate
    clear_graphs(c);                              // captured sequences depend on the parameters
    c->evaluated = false;
    if (realloc) {
        int rc = alloc_blocks(c, prm->p, mixed);
        if (rc) return rc;
        c->bx_valid = false;
    }
    if (!mixed) c->phase = 64;
    return OFKS_OK;
}

int ofks_init_orbitals(ofks_ctx *c, const double *V) {
    if (!c || !V) return OFKS_EINVAL;
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "init_orbitals: no mesh/params");
    cudaSetDevice(c->device);
    int rc;
    Blocks<double> &b = c->b64;
    double *Vd = b.X[c->cur ^ 1], *BV = b.Q;
    if ((rc = upload_block(c, V, Vd))) return rc;
    launch_sell_spmm(c, (const double *)c->d_valB, (const double *)Vd, BV);
    launch_gram2(c, (const double *)Vd, (const double *)BV, (const double *)BV, c->d_S, c->d_L0);
    double *Rinv = c->d_pp + 6 * (size_t)c->ld * c->ld;
    launch_cholesky_inv(c, c->d_S, Rinv);
    launch_block_times_small(c, (const double *)Vd, Rinv, b.X[c->cur]);
    launch_block_times_small(c, (const double *)BV, Rinv, b.BX);
    int flag = 0;
    if ((rc = read_flag(c, &flag))) return rc;
    if (flag) return ofks_fail(c, OFKS_ENOTCONV, "init_orbitals: V^T B V is not positive definite");
    c->bx_valid = true;
    c->phase = c->prm.precision == OFKS_MIXED ? 32 : 64;
    state_to32(c);
    c->switch_k = -1;
    c->have_X = true; c->have_prev = false; c->converged = false; c->evaluated = false;
    c->gcn_skip = 0; c->gcn_backoff = 0;     // the learned preconditioner's pauses restart
    c->k = 0; c->kkt0 = 0; c->eta = 0;
    c->history.clear();
    c->t_start = now_s();
    return OFKS_OK;
}

int ofks_set_orbitals(ofks_ctx *c, const double *X, int32_t keep) {
    if (!c || !X) return OFKS_EINVAL;
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "set_orbitals: no mesh/params");
    cudaSetDevice(c->device);
    if (!keep) c->phase = c->prm.precision == OFKS_MIXED ? 32 : 64;
    if (c->phase == 32 && c->ld != c->p) {
        // float32 iterations read only the float32 block (the float64 set is refilled from it
        // before any float64 use): one pass from the staging copy straight into it
        const size_t bytes = sizeof(double) * (size_t)c->n * c->p;
        cudaError_t e = cudaMemcpyAsync(c->d_stage, X, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) launch_unpack_f32(c, c->d_stage, c->b32.X[c->cur]);
        int rc = ofks_cuda_check(c, e, "block upload");
        if (rc) return rc;
    } else {
        int rc = upload_block(c, X, c->b64.X[c->cur]);
        if (rc) return rc;
        if (c->phase == 32)
            launch_convert(c, (const double *)c->b64.X[c->cur], c->b32.X[c->cur], c->n * (int64_t)c->ld);
    }
    c->bx_valid = false;
    c->have_X = true;
    c->evaluated = false;
    if (!keep) {
        c->have_prev = false; c->converged = false; c->k = 0; c->kkt0 = 0; c->eta = 0;
        c->gcn_skip = 0; c->gcn_backoff = 0;     // the learned preconditioner's pauses restart
        c->history.clear();
        c->t_start = now_s();
    }
    return OFKS_OK;
}

int ofks_get_orbitals(ofks_ctx *c, double *X) {
    if (!c || !X) return OFKS_EINVAL;
    if (!c->have_X) return ofks_fail(c, OFKS_ESTATE, "get_orbitals: no orbitals");
    cudaSetDevice(c->device);
    if (c->phase == 32 && c->ld != c->p) {          // one pass from the float32 block into the staging copy
        launch_pack_f32(c, c->b32.X[c->cur], c->d_stage);
        cudaError_t e = cudaMemcpyAsync(X, c->d_stage, sizeof(double) * (size_t)c->n * c->p, cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        return ofks_cuda_check(c, e, "block download");
    }
    if (c->phase == 32) launch_convert(c, (const float *)c->b32.X[c->cur], c->b64.X[c->cur], c->n * (int64_t)c->ld);
    return download_block(c, c->b64.X[c->cur], X);
}

int ofks_step(ofks_ctx *c, int32_t k, ofks_result *res) {
    if (!c || k < 0) return OFKS_EINVAL;
    if (!c->have_nuclei) return ofks_fail(c, OFKS_ESTATE, "step: no nuclei");
    cudaSetDevice(c->device);
    return run_iterations(c, k, res);
}

int ofks_solve(ofks_ctx *c, ofks_result *res) {
    if (!c) return OFKS_EINVAL;
    if (!c->have_nuclei) return ofks_fail(c, OFKS_ESTATE, "solve: no nuclei");
    cudaSetDevice(c->device);
    int rc = run_iterations(c, c->prm.max_iter - c->k, res);
    if (rc) return rc;
    if (!c->converged) return ofks_fail(c, OFKS_ENOTCONV, "solve: not converged after %d iterations", c->k);
    return OFKS_OK;
}

int ofks_evaluate(ofks_ctx *c, ofks_result *res) {
    if (!c) return OFKS_EINVAL;
    if (!c->have_X || !c->have_nuclei) return ofks_fail(c, OFKS_ESTATE, "evaluate: need orbitals and nuclei");
    cudaSetDevice(c->device);
    Rec r{};
    int rc = evaluate(c, !c->bx_valid, &r);
    if (rc) return rc;
    c->bx_valid = true;
    if (res) {
        res->e_total = r.E; res->e_nuc = c->e_nuc; res->kkt = r.kkt; res->fea = r.fea; res->kkt0 = c->kkt0;
        res->eta = c->eta; res->iters = c->k; res->converged = c->converged; res->seconds = 0;
        res->hartree_iters = c->cg_last; res->hartree_total = c->cg_last;
    }
    return OFKS_OK;
}

int ofks_rayleigh_ritz(ofks_ctx *c, double *eigs) {
    if (!c || !eigs) return OFKS_EINVAL;
    if (!c->have_X || !c->have_nuclei) return ofks_fail(c, OFKS_ESTATE, "rayleigh_ritz: need orbitals and nuclei");
    cudaSetDevice(c->device);
    if (c->phase == 32) {            // Rayleigh-Ritz runs on the float64 state
        state_to64(c);
        c->phase = 64;
        c->bx_valid = false;
    }
    Rec r{};
    int rc = evaluate(c, !c->bx_valid, &r);
    if (rc) return rc;
    const size_t L2 = (size_t)c->ld * c->ld;
    double *V = c->d_pp + 5 * L2, *de = c->d_pp + 7 * L2;
    launch_rayleigh_ritz(c, c->d_L0, c->d_S, de, V);
    launch_block_times_small(c, (const double *)c->b64.X[c->cur], V, c->b64.X[c->cur ^ 1]);
    int flag = 0;
    if ((rc = read_flag(c, &flag))) return rc;
    if (flag) return ofks_fail(c, OFKS_ENOTCONV, "rayleigh_ritz: X^T B X is not positive definite");
    cudaError_t e = cudaMemcpyAsync(eigs, de, sizeof(double) * c->p, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if ((rc = ofks_cuda_check(c, e, "rayleigh_ritz"))) return rc;
    c->cur ^= 1;
    c->bx_valid = false;
    c->have_prev = false;
    c->evaluated = false;
    return OFKS_OK;
}

int ofks_get_field(ofks_ctx *c, int32_t which, double *out, int64_t count) {
    if (!c || !out) return OFKS_EINVAL;
    if (!c->evaluated) return ofks_fail(c, OFKS_ESTATE, "get_field: evaluate first");
    cudaSetDevice(c->device);
    const int64_t nq = c->n_tets * 4, nb = c->n * (int64_t)c->p, pp = (int64_t)c->p * c->p;
    const double *src = nullptr;
    int64_t need = 0;
    int kind = 0;   // 0 flat, 1 block n x p, 2 small p x p
    switch (which) {
        case OFKS_F_RHO_Q: src = c->d_rho; need = nq; break;
        case OFKS_F_VH_Q: src = c->d_vh; need = nq; break;
        case OFKS_F_VXC_Q: src = c->d_vxc; need = nq; break;
        case OFKS_F_EXC_Q: src = c->d_exc; need = nq; break;
        case OFKS_F_VEXT_Q: src = c->d_vext; need = nq; break;
        case OFKS_F_U: src = c->d_U; need = c->n_nodes; break;
        case OFKS_F_HX: case OFKS_F_BX: case OFKS_F_G: case OFKS_F_D: {
            const int dcur = c->cur ^ (c->have_prev ? 1 : 0);
            need = nb; kind = 1;
            if (c->phase == 32) {       // float32 state: widen into a float64 scratch block
                const float *f = which == OFKS_F_HX ? c->b32.HX : which == OFKS_F_BX ? c->b32.BX
                               : which == OFKS_F_G ? c->b32.G[c->cur] : c->b32.D[dcur];
                launch_convert(c, f, c->b64.R, c->n * (int64_t)c->ld);
                src = c->b64.R;
            } else {
                src = which == OFKS_F_HX ? c->b64.HX : which == OFKS_F_BX ? c->b64.BX
                    : which == OFKS_F_G ? c->b64.G[c->cur] : c->b64.D[dcur];
            }
            break;
        }
        case OFKS_F_LAMBDA0: src = c->d_L0; need = pp; kind = 2; break;
        case OFKS_F_S: src = c->d_S; need = pp; kind = 2; break;
        case OFKS_F_LAMBDA: src = c->d_Lam; need = pp; kind = 2; break;
        default: return ofks_fail(c, OFKS_EINVAL, "get_field: unknown field %d", which);
    }
    if (count != need) return ofks_fail(c, OFKS_EINVAL, "get_field: field %d has %lld values, got %lld", which,
                                        (long long)need, (long long)count);
    if (kind == 1) return download_block(c, src, out);
    cudaError_t e;
    if (kind == 2)
        e = cudaMemcpy2DAsync(out, sizeof(double) * c->p, src, sizeof(double) * c->ld, sizeof(double) * c->p, c->p,
                              cudaMemcpyDeviceToHost, c->stream);
    else
        e = cudaMemcpyAsync(out, src, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return ofks_cuda_check(c, e, "get_field");
}

int ofks_apply(ofks_ctx *c, int32_t which, const double *X, double *Y, int32_t ncols) {
    if (!c || !X || !Y) return OFKS_EINVAL;
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "apply: no mesh/params");
    if (ncols != c->p) return ofks_fail(c, OFKS_EINVAL, "apply: ncols must equal p");
    const double *val = which == OFKS_M_L ? c->d_valL : which == OFKS_M_B ? c->d_valB : which == OFKS_M_H ? c->d_valH : nullptr;
    if (!val) return ofks_fail(c, OFKS_EINVAL, "apply: unknown matrix %d", which);
    if (which == OFKS_M_H && !c->evaluated) return ofks_fail(c, OFKS_ESTATE, "apply: H needs an evaluation");
    cudaSetDevice(c->device);
    int rc = upload_block(c, X, c->b64.Z);
    if (rc) return rc;
    launch_sell_spmm(c, val, (const double *)c->b64.Z, c->b64.Q);
    if ((rc = ofks_cuda_check(c, cudaGetLastError(), "apply"))) return rc;
    return download_block(c, c->b64.Q, Y);
}

int ofks_get_sizes(ofks_ctx *c, int64_t *n_free, int64_t *n_nodes, int64_t *n_tets, int64_t *nnz,
                   int64_t *nnz_full) {
    if (!c) return OFKS_EINVAL;
    if (n_free) *n_free = c->n;
    if (n_nodes) *n_nodes = c->n_nodes;
    if (n_tets) *n_tets = c->n_tets;
    if (nnz) *nnz = c->nnz;
    if (nnz_full) *nnz_full = c->nnz_full;
    return OFKS_OK;
}

int ofks_poisson_info(ofks_ctx *c, int32_t *format, int64_t *stored, int64_t *rows, int32_t *lattice,
                      int32_t *precond) {
    if (!c) return OFKS_EINVAL;
    if (c->n_nodes == 0) return ofks_fail(c, OFKS_ESTATE, "poisson_info: no mesh");
    const bool lat = c->st.on && !c->prm.poisson_csr;
    int64_t nr = 0;
    if (lat) nr = c->st.rows;
    else nr = c->n_nodes - c->n_bnd;
    if (format) *format = lat ? 1 : 0;
    if (stored) *stored = lat ? c->st.len : c->nnz_full;
    if (rows) *rows = nr;
    if (precond) *precond = hartree_pc(c);
    if (lattice) {
        lattice[0] = c->st.on ? c->st.Lx : 0;
        lattice[1] = c->st.on ? c->st.Ly : 0;
        lattice[2] = c->st.on ? c->st.Lz : 0;
    }
    return OFKS_OK;
}

int ofks_get_history(ofks_ctx *c, double *buf, int32_t cap, int32_t *len) {
    if (!c || !len || cap < 0 || (cap > 0 && !buf)) return OFKS_EINVAL;
    const int rows = (int)(c->history.size() / 6);
    const int m = rows < cap ? rows : cap;
    if (m > 0) memcpy(buf, c->history.data() + (size_t)(rows - m) * 6, sizeof(double) * 6 * m);
    *len = m;
    return OFKS_OK;
}

struct StateHeader {
    char magic[8];
    int64_t n, n_nodes;
    int32_t p, ld, k, phase, have_prev, converged;
    double kkt0, eta, eta_dev;
    int64_t hist_rows;
};

int ofks_save_state(ofks_ctx *c, const char *path) {
    if (!c || !path) return OFKS_EINVAL;
    if (!c->have_X) return ofks_fail(c, OFKS_ESTATE, "save_state: no orbitals");
    cudaSetDevice(c->device);
    state_to64(c);
    if (!c->bx_valid)
        launch_sell_spmm(c, (const double *)c->d_valB, (const double *)c->b64.X[c->cur], c->b64.BX);
    StateHeader h{};
    memcpy(h.magic, "OFKSST1", 8);
    h.n = c->n; h.n_nodes = c->n_nodes; h.p = c->p; h.ld = c->ld; h.k = c->k; h.have_prev = c->have_prev;
    h.converged = c->converged; h.kkt0 = c->kkt0; h.eta = c->eta; h.hist_rows = (int64_t)c->history.size() / 6;
    h.phase = c->phase;
    cudaMemcpyAsync(&h.eta_dev, c->d_sc + SC_ETA, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    const size_t blk = (size_t)c->n * c->ld;
    std::vector<double> buf(blk * 5 + c->n_nodes);
    const double *srcs[5] = {c->b64.X[c->cur], c->b64.X[c->cur ^ 1], c->b64.D[c->cur ^ 1], c->b64.G[c->cur ^ 1],
                             c->b64.BX};
    for (int i = 0; i < 5; ++i)
        cudaMemcpyAsync(buf.data() + i * blk, srcs[i], sizeof(double) * blk, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(buf.data() + 5 * blk, c->d_U, sizeof(double) * c->n_nodes, cudaMemcpyDeviceToHost, c->stream);
    int rc = ofks_cuda_check(c, cudaStreamSynchronize(c->stream), "save_state");
    if (rc) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return ofks_fail(c, OFKS_EINVAL, "save_state: cannot open %s", path);
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size() &&
              fwrite(c->history.data(), sizeof(double), c->history.size(), f) == c->history.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? OFKS_OK : ofks_fail(c, OFKS_EINVAL, "save_state: write to %s failed", path);
}

int ofks_load_state(ofks_ctx *c, const char *path) {
    if (!c || !path) return OFKS_EINVAL;
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "load_state: set mesh and params first");
    FILE *f = fopen(path, "rb");
    if (!f) return ofks_fail(c, OFKS_EINVAL, "load_state: cannot open %s", path);
    StateHeader h{};
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "OFKSST1", 8) != 0) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "load_state: %s is not a state file", path);
    }
    if (h.n != c->n || h.n_nodes != c->n_nodes || h.p != c->p || h.ld != c->ld) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "load_state: sizes differ from the current mesh/params");
    }
    const size_t blk = (size_t)c->n * c->ld;
    // the history length must be what the file's size leaves after the header and the blocks
    const int64_t body = (int64_t)sizeof(double) * (int64_t)(blk * 5 + c->n_nodes);
    int64_t fsize = -1;
    if (fseek(f, 0, SEEK_END) == 0) fsize = (int64_t)ftell(f);
    if (fsize < 0 || fseek(f, (long)sizeof(h), SEEK_SET) != 0) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "load_state: cannot size %s", path);
    }
    if (h.hist_rows < 0 || (int64_t)sizeof(h) + body + h.hist_rows * 6 * (int64_t)sizeof(double) != fsize) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "load_state: %s has %lld bytes, not what its header describes", path,
                         (long long)fsize);
    }
    std::vector<double> buf, hist;
    try {
        buf.resize(blk * 5 + c->n_nodes);
        hist.resize((size_t)h.hist_rows * 6);
    } catch (const std::bad_alloc &) {
        fclose(f);
        return ofks_fail(c, OFKS_ENOMEM, "load_state: host buffers");
    }
    bool ok = fread(buf.data(), sizeof(double), buf.size(), f) == buf.size() &&
              fread(hist.data(), sizeof(double), hist.size(), f) == hist.size();
    fclose(f);
    if (!ok) return ofks_fail(c, OFKS_EINVAL, "load_state: %s is truncated", path);
    cudaSetDevice(c->device);
    c->cur = 0;
    double *dsts[5] = {c->b64.X[0], c->b64.X[1], c->b64.D[1], c->b64.G[1], c->b64.BX};
    for (int i = 0; i < 5; ++i)
        cudaMemcpyAsync(dsts[i], buf.data() + i * blk, sizeof(double) * blk, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_U, buf.data() + 5 * blk, sizeof(double) * c->n_nodes, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_sc + SC_ETA, &h.eta_dev, sizeof(double), cudaMemcpyHostToDevice, c->stream);
    int rc = ofks_cuda_check(c, cudaStreamSynchronize(c->stream), "load_state");
    if (rc) return rc;
    c->bx_valid = true;
    c->phase = (h.phase == 32 && c->mixed_alloc) ? 32 : 64;
    state_to32(c);
    c->have_X = true; c->k = h.k; c->have_prev = h.have_prev; c->converged = h.converged; c->kkt0 = h.kkt0;
    c->gcn_skip = 0; c->gcn_backoff = 0;     // the learned preconditioner's pauses restart
    c->best_rel = 1.0; c->best_k = h.k;            // the float32 stall test restarts from here
    c->eta = h.eta; c->evaluated = false;
    c->history = hist;
    c->t_start = now_s() - (hist.empty() ? 0.0 : hist[hist.size() - 5]);
    return OFKS_OK;
}

// ------------------------------------------------------------------------- learned preconditioner
int ofks_precond_init(ofks_ctx *c, int32_t width, uint64_t seed) {
    if (!c) return OFKS_EINVAL;
    if (!c->n) return ofks_fail(c, OFKS_ESTATE, "precond_init: no mesh");
    if (width != 8 && width != 16 && width != 32 && width != 64)
        return ofks_fail(c, OFKS_EINVAL, "precond_init: width must be 8, 16, 32 or 64");
    cudaSetDevice(c->device);
    return gcn_setup(c, width, seed, c->row_deg);
}

int ofks_precond_get_weights(ofks_ctx *c, float *w, int64_t cap, int64_t *count) {
    if (!c || !count) return OFKS_EINVAL;
    if (!c->gcn.H) return ofks_fail(c, OFKS_ESTATE, "precond_get_weights: no network");
    const int64_t m = gcn_param_count(c->gcn.H);
    *count = m;
    if (!w) return OFKS_OK;
    if (cap < m) return ofks_fail(c, OFKS_EINVAL, "precond_get_weights: need %lld floats", (long long)m);
    cudaSetDevice(c->device);
    return ofks_cuda_check(c, cudaMemcpy(w, c->gcn.w, sizeof(float) * m, cudaMemcpyDeviceToHost), "get_weights");
}

int ofks_precond_set_weights(ofks_ctx *c, const float *w, int64_t count) {
    if (!c || !w) return OFKS_EINVAL;
    if (!c->n) return ofks_fail(c, OFKS_ESTATE, "precond_set_weights: no mesh");
    int width = 0;
    for (int h : {8, 16, 32, 64})
        if (gcn_param_count(h) == count) width = h;
    if (!width) return ofks_fail(c, OFKS_EINVAL, "precond_set_weights: %lld values match no width", (long long)count);
    cudaSetDevice(c->device);
    if (c->gcn.H != width) {
        int rc = gcn_setup(c, width, 0, c->row_deg);
        if (rc) return rc;
    }
    return ofks_cuda_check(c, cudaMemcpy(c->gcn.w, w, sizeof(float) * count, cudaMemcpyHostToDevice), "set_weights");
}

int ofks_precondition(ofks_ctx *c, int32_t mode, const double *G, const double *shifts, double *D) {
    if (!c || !G || !shifts || !D) return OFKS_EINVAL;
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "precondition: no mesh/params");
    if (mode != OFKS_PC_PCG && mode != OFKS_PC_EXACT && mode != OFKS_PC_LEARNED)
        return ofks_fail(c, OFKS_EINVAL, "precondition: unknown mode %d", mode);
    cudaSetDevice(c->device);
    const int ld = c->ld;
    if (mode == OFKS_PC_LEARNED) {
        if (!c->gcn.H) return ofks_fail(c, OFKS_ESTATE, "precondition: no network");
        int rc;
        if (!c->d_shift_in && cudaMalloc((void **)&c->d_shift_in, sizeof(double) * 256) != cudaSuccess)
            return ofks_fail(c, OFKS_ENOMEM, "shift buffer");
        if ((rc = upload_block(c, G, c->b64.Z))) return rc;
        cudaMemcpyAsync(c->d_shift_in, shifts, sizeof(double) * c->p, cudaMemcpyHostToDevice, c->stream);
        if ((rc = gcn_forward_prepare(c))) return rc;
        gcn_pack<double>(c, c->b64.Z, c->gcn.G32);
        if ((rc = gcn_forward(c, c->d_shift_in, false))) return rc;
        gcn_unpack<double>(c, c->gcn.Dn, c->b64.Q);
        // columns with shift >= 0: D = G
        std::vector<double> act(ld, 0.0);
        for (int j = 0; j < c->p; ++j) act[j] = shifts[j] < 0 ? 1.0 : 0.0;
        cudaMemcpyAsync(c->d_colA + CB_ACTIVE * ld, act.data(), sizeof(double) * ld, cudaMemcpyHostToDevice, c->stream);
        Blocks<double> tmp = c->b64;
        tmp.G[c->cur] = c->b64.Z;
        tmp.D[c->cur] = c->b64.Q;
        launch_direction_select(c, tmp);
        return download_block(c, c->b64.Q, D);
    }
    // PCG / exact: run the iteration's preconditioner on (G, shifts) in float64
    std::vector<double> col(2 * (size_t)ld, 0.0);
    for (int j = 0; j < c->p; ++j) {
        col[j] = shifts[j] < 0 ? shifts[j] : 0.0;
        col[ld + j] = shifts[j] < 0 ? 1.0 : 0.0;
    }
    cudaMemcpyAsync(c->d_colA + CB_SHIFT * ld, col.data(), sizeof(double) * 2 * ld, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(c->d_colA + CB_ACC * ld, 0, sizeof(double) * ld, c->stream);
    cudaMemsetAsync(c->d_colA + CB_WARM * ld, 0, sizeof(double) * ld, c->stream);
    int rc = upload_block(c, G, c->b64.G[c->cur]);
    if (rc) return rc;
    const int saved = c->prm.precond, phase = c->phase;
    c->prm.precond = mode;
    // a mixed context runs the float32 preconditioner of its float32 iterations (G rounded to
    // float32 on the way in, D widened on the way out)
    const bool f32 = mode == OFKS_PC_PCG && c->prm.precision == OFKS_MIXED && c->mixed_alloc;
    const int64_t cnt = c->n * (int64_t)ld;
    if (f32) {
        launch_convert(c, (const double *)c->b64.G[c->cur], c->b32.G[c->cur], cnt);
        c->phase = 32;
        rc = precondition_t<float>(c);
        if (!rc) launch_convert(c, (const float *)c->b32.D[c->cur], c->b64.D[c->cur], cnt);
    } else {
        c->phase = 64;
        rc = precondition_t<double>(c);
    }
    c->prm.precond = saved;
    c->phase = phase;
    if (rc) return rc;
    return download_block(c, c->b64.D[c->cur], D);
}

static int train_common(ofks_ctx *c, const double *G, const double *shifts, const double *Dstar, double *loss) {
    if (!c->gcn.H) return ofks_fail(c, OFKS_ESTATE, "no network (ofks_precond_init)");
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "no mesh/params");
    if (!c->d_shift_in && cudaMalloc((void **)&c->d_shift_in, sizeof(double) * 256) != cudaSuccess)
        return ofks_fail(c, OFKS_ENOMEM, "shift buffer");
    int rc;
    if ((rc = upload_block(c, G, c->b64.Z)) || (rc = upload_block(c, Dstar, c->b64.R))) return rc;
    cudaMemcpyAsync(c->d_shift_in, shifts, sizeof(double) * c->p, cudaMemcpyHostToDevice, c->stream);
    if ((rc = gcn_forward_prepare(c))) return rc;
    gcn_pack<double>(c, c->b64.Z, c->gcn.G32);
    gcn_pack<double>(c, c->b64.R, c->gcn.Ds);
    if ((rc = gcn_forward(c, c->d_shift_in, true))) return rc;
    return gcn_backward(c, c->d_shift_in, loss);
}

int ofks_train_precond_step(ofks_ctx *c, const double *G, const double *shifts, const double *Dstar, double lr,
                            double *loss) {
    if (!c || !G || !shifts || !Dstar || !loss || !(lr > 0)) return OFKS_EINVAL;
    cudaSetDevice(c->device);
    int rc = train_common(c, G, shifts, Dstar, loss);
    if (rc) return rc;
    if ((rc = gcn_adam(c, lr))) return rc;
    return ofks_cuda_check(c, cudaStreamSynchronize(c->stream), "train step");
}

int ofks_precond_grads(ofks_ctx *c, const double *G, const double *shifts, const double *Dstar, double *grads,
                       int64_t cap, double *loss) {
    if (!c || !G || !shifts || !Dstar || !grads || !loss) return OFKS_EINVAL;
    cudaSetDevice(c->device);
    int rc = train_common(c, G, shifts, Dstar, loss);
    if (rc) return rc;
    const int64_t m = gcn_param_count(c->gcn.H);
    if (cap < m) return ofks_fail(c, OFKS_EINVAL, "precond_grads: need %lld values", (long long)m);
    return ofks_cuda_check(c, cudaMemcpy(grads, c->gcn.grad, sizeof(double) * m, cudaMemcpyDeviceToHost), "grads");
}

// ---- pairs files of the learned preconditioner
struct PairsHeader {
    char magic[8];
    int64_t n;
    int32_t p, zero;
};

int ofks_record_pair(ofks_ctx *c, const char *path, int32_t *active) {
    if (!c || !path) return OFKS_EINVAL;
    if (!c->have_X) return ofks_fail(c, OFKS_ESTATE, "record_pair: no orbitals");
    const int64_t n = c->n, p = c->p;
    std::vector<double> G, Lam, D;
    try {
        G.resize((size_t)(n * p));
        D.resize((size_t)(n * p));
        Lam.resize((size_t)(p * p));
    } catch (const std::bad_alloc &) {
        return ofks_fail(c, OFKS_ENOMEM, "record_pair: host buffers");
    }
    int rc;
    if ((rc = ofks_evaluate(c, nullptr)) || (rc = ofks_get_field(c, OFKS_F_G, G.data(), n * p)) ||
        (rc = ofks_get_field(c, OFKS_F_LAMBDA, Lam.data(), p * p)))
        return rc;
    std::vector<double> shifts((size_t)p);
    int32_t nact = 0;
    for (int64_t j = 0; j < p; ++j) {
        shifts[j] = Lam[(size_t)(j * p + j)];
        nact += shifts[j] < 0.0;
    }
    if ((rc = ofks_precondition(c, OFKS_PC_EXACT, G.data(), shifts.data(), D.data()))) return rc;
    FILE *f = fopen(path, "r+b");
    PairsHeader h{};
    if (f) {
        if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "OFKSPR1", 8) != 0 || h.n != n || h.p != p) {
            fclose(f);
            return ofks_fail(c, OFKS_EINVAL, "record_pair: %s holds pairs of another shape", path);
        }
        fseek(f, 0, SEEK_END);
    } else {
        f = fopen(path, "wb");
        if (!f) return ofks_fail(c, OFKS_EINVAL, "record_pair: cannot create %s", path);
        memcpy(h.magic, "OFKSPR1", 8);
        h.n = n;
        h.p = (int32_t)p;
        if (fwrite(&h, sizeof(h), 1, f) != 1) {
            fclose(f);
            return ofks_fail(c, OFKS_EINVAL, "record_pair: write to %s failed", path);
        }
    }
    bool ok = fwrite(shifts.data(), sizeof(double), shifts.size(), f) == shifts.size() &&
              fwrite(G.data(), sizeof(double), G.size(), f) == G.size() &&
              fwrite(D.data(), sizeof(double), D.size(), f) == D.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) return ofks_fail(c, OFKS_EINVAL, "record_pair: write to %s failed", path);
    if (active) *active = nact;
    return OFKS_OK;
}

// SplitMix64 (Steele, Lea and Flood 2014): the pair order of one epoch
static uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int ofks_train_precond(ofks_ctx *c, const char *path, int32_t epochs, uint64_t seed) {
    if (!c || !path || epochs < 1) return OFKS_EINVAL;
    if (!c->gcn.H) return ofks_fail(c, OFKS_ESTATE, "train_precond: no network (ofks_precond_init)");
    if (!c->n || !c->p) return ofks_fail(c, OFKS_ESTATE, "train_precond: no mesh/params");
    FILE *f = fopen(path, "rb");
    if (!f) return ofks_fail(c, OFKS_EINVAL, "train_precond: cannot open %s", path);
    PairsHeader h{};
    const int64_t n = c->n, p = c->p;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "OFKSPR1", 8) != 0 || h.n != n || h.p != p) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "train_precond: %s is not a pairs file of this mesh and p", path);
    }
    const int64_t rec = (int64_t)sizeof(double) * (p + 2 * n * p);
    fseek(f, 0, SEEK_END);
    const int64_t size = (int64_t)ftell(f);
    const int64_t count = (size - (int64_t)sizeof(h)) / rec;
    if (count < 1 || (int64_t)sizeof(h) + count * rec != size) {
        fclose(f);
        return ofks_fail(c, OFKS_EINVAL, "train_precond: %s holds %lld bytes, not whole pairs", path, (long long)size);
    }
    std::vector<double> buf;
    try {
        buf.resize((size_t)(p + 2 * n * p));
    } catch (const std::bad_alloc &) {
        fclose(f);
        return ofks_fail(c, OFKS_ENOMEM, "train_precond: host buffer");
    }
    cudaSetDevice(c->device);
    std::vector<int64_t> order((size_t)count);
    int64_t steps = 0;
    double epoch_loss = 0.0;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
        uint64_t st = seed ^ (0xD1B54A32D192ED03ULL * (uint64_t)(ep + 1));
        for (int64_t i = count - 1; i > 0; --i) {                 // Fisher-Yates
            const int64_t j = (int64_t)(splitmix64(st) % (uint64_t)(i + 1));
            std::swap(order[(size_t)i], order[(size_t)j]);
        }
        double sum = 0.0;
        for (int64_t i = 0; i < count; ++i) {
            if (fseek(f, (long)((int64_t)sizeof(h) + order[(size_t)i] * rec), SEEK_SET) != 0 ||
                fread(buf.data(), sizeof(double), buf.size(), f) != buf.size()) {
                fclose(f);
                return ofks_fail(c, OFKS_EINVAL, "train_precond: read of %s failed", path);
            }
            double loss = 0.0;
            int rc = ofks_train_precond_step(c, buf.data() + p, buf.data(), buf.data() + p + n * p, 1e-3, &loss);
            if (rc) {
                fclose(f);
                return rc;
            }
            sum += loss;
            ++steps;
        }
        epoch_loss = sum / (double)count;
    }
    fclose(f);
    c->train_loss = epoch_loss;
    c->train_steps += steps;
    return OFKS_OK;
}

int ofks_train_info(ofks_ctx *c, double *last_epoch_loss, int64_t *steps) {
    if (!c) return OFKS_EINVAL;
    if (last_epoch_loss) *last_epoch_loss = c->train_loss;
    if (steps) *steps = c->train_steps;
    return OFKS_OK;
}

int ofks_profile(ofks_ctx *c, int32_t on) {
    if (!c) return OFKS_EINVAL;
    prof_resolve(c);
    c->prof = on != 0;
    if (on) {
        for (int i = 0; i < PF_COUNT; ++i) { c->prof_n[i] = 0; c->prof_ms[i] = 0; }
        c->kernels_at_prof = c->kernels;
    }
    return OFKS_OK;
}

int ofks_profile_get(ofks_ctx *c, int32_t id, int64_t *launches, double *ms, const char **name) {
    if (!c || id < 0 || id > PF_COUNT) return OFKS_EINVAL;
    prof_resolve(c);
    if (id == PF_COUNT) {   // every kernel launch since profiling was switched on
        if (launches) *launches = c->kernels - c->kernels_at_prof;
        if (ms) *ms = 0.0;
        if (name) *name = "all_kernels";
        return OFKS_OK;
    }
    if (launches) *launches = c->prof_n[id];
    if (ms) *ms = c->prof_ms[id];
    if (name) *name = kPfNames[id];
    return OFKS_OK;
}

}  // extern "C"
