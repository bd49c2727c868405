"""Mixed-precision form against the float64 oracle.

The float32 iterations (float64 only for the p x p Grams' accumulation, the energy sum and the
convergence test) follow the oracle to float32 accuracy; after the hand-over at
(kkt + fea)/kkt0 < mixed_tol the float64 sweep reaches the oracle's fixed point to the same
tolerances as the plain form: E within 1e-8 Ha, eigenvalues within 1e-7 Ha, fea <= 1e-10.
"""
import numpy as np
import pytest

from oracle import pcal
from paper_2007_14228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofks():
    from paper_2007_14228_gb300 import build
    build.build()
    from paper_2007_14228_gb300 import ofks as mod
    return mod


def pair(ofks, s, **kw):
    m = I.make_mesh(s)
    params = dict(beta=10.0, precision="mixed")
    params.update(kw)
    ctx = ofks.context_for(s, m, **params)
    okw = {k: v for k, v in params.items() if k in ("beta", "tol", "max_iter")}
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, **okw))
    V = I.initial_block(m.n_free, s.p, 0)
    return ctx, pr, V


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("cells,p", [((6, 6, 6), 2), ((10, 10, 10), 2)])
def test_float32_steps_follow_the_oracle(ofks, cells, p):
    s = I.lih().with_cells(cells).with_p(p)
    ctx, pr, V = pair(ofks, s)
    ctx.init_orbitals(V)
    st = pcal.State(X=pr.initial_guess(V))
    for k in range(5):
        g = ctx.step(1)
        o = pcal.iterate(pr, st)
        assert g["switch_iter"] == -1
        assert abs(g["e_total"] - o["E"]) < 2e-5 * max(1.0, abs(o["E"])), (k, g["e_total"], o["E"])
        assert abs(g["kkt"] - o["kkt"]) < 1e-4 * o["kkt"]
    assert rel(ctx.get_orbitals(), st.X) < 1e-3
    ctx.close()


def test_mixed_solve_reaches_the_float64_fixed_point(ofks):
    s = I.lih().with_cells((6, 6, 6))
    ctx, pr, V = pair(ofks, s, tol=1e-12, max_iter=4000, mixed_tol=1e-5)
    ctx.init_orbitals(V)
    res = ctx.solve()
    assert res["converged"] == 1 and res["switch_iter"] > 0
    eig = ctx.rayleigh_ritz()
    pr.prm.max_iter = 4000
    pr.prm.tol = 1e-12
    st = pcal.solve(pr, pr.initial_guess(V))
    eig_o, _ = pr.rayleigh_ritz(st.X)
    assert abs(res["e_total"] - st.history[-1]["E"]) < 1e-8
    np.testing.assert_allclose(eig, eig_o, atol=1e-7)
    assert res["fea"] <= 1e-10
    ctx.close()


def test_mixed_wide_block_steps(ofks):
    # p = 41 on the reduced chain grid: float4 chunks, wide Grams and PCG in float32
    s = I.chain(cells=(26, 14, 8))
    ctx, pr, V = pair(ofks, s)
    ctx.init_orbitals(V)
    st = pcal.State(X=pr.initial_guess(V))
    for k in range(3):
        g = ctx.step(1)
        o = pcal.iterate(pr, st)
        assert abs(g["e_total"] - o["E"]) < 2e-5 * abs(o["E"]), (k, g["e_total"], o["E"])
        assert abs(g["kkt"] - o["kkt"]) < 1e-4 * o["kkt"]
    ctx.close()


def _renumbered(m0, seed=3):
    perm = np.random.default_rng(seed).permutation(len(m0.xyz))     # new id -> old id
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return I.Mesh(m0.xyz[perm].copy(), inv[m0.tet10], m0.dirichlet[perm].copy(), m0.lattice, m0.axes)


@pytest.mark.parametrize("case", ["chain_p41", "h2o_p5", "lih_p2", "lih_renumbered_p3"])
def test_float32_preconditioner_matches_the_oracle(ofks, case):
    # the float32 PCG of the mixed form (8 iterations of Eq. precondition-T) against the oracle's
    # float64 PCG: the type-grouped SELL with chunk-major Z on lattice meshes (p = 41, 5), the
    # row-major kernels for p <= 2 and on meshes whose ids are not a lattice
    if case == "chain_p41":
        s = I.chain(cells=(26, 14, 8))
        m = I.make_mesh(s)
    elif case == "h2o_p5":
        R = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])
        s = I.System("h2o_like", np.array([8.0, 1.0, 1.0]), R, np.full(3, -8.0), np.full(3, 8.0), (10, 10, 10), 5, 2.0)
        m = I.make_mesh(s)
    elif case == "lih_p2":
        s = I.lih().with_cells((8, 8, 8))
        m = I.make_mesh(s)
    else:
        s = I.lih().with_cells((8, 8, 8)).with_p(3, occ=1.0)
        m = _renumbered(I.make_mesh(s))
    ctx = ofks.context_for(s, m, beta=10.0, precision="mixed")
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, hartree=False, xc=False))
    rng = np.random.default_rng(7)
    G = rng.standard_normal((m.n_free, s.p))
    shifts = -rng.uniform(0.05, 2.0, s.p)
    shifts[0] = 0.3                                   # one column with T = I
    D = ctx.precondition("pcg", G, shifts)
    Do = pr.precondition(G, shifts)
    assert np.max(np.abs(D - Do)) < 1e-4 * np.max(np.abs(Do)), np.max(np.abs(D - Do)) / np.max(np.abs(Do))
    assert np.array_equal(D[:, 0].astype(np.float32), G[:, 0].astype(np.float32))
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compact_pcg_matches_full_width_and_the_oracle(ofks, precision):
    # Eq. precondition-T solves one system per column with Lambda_ii < 0; the compact form runs the
    # PCG on those columns only, gathered into a block of their count rounded up to 4 (here 24 of
    # 41, scattered over the block), and must give what the PCG on all columns gives
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((m.n_free, s.p))
    shifts = -rng.uniform(0.05, 2.0, s.p)
    inactive = rng.choice(s.p, 17, replace=False)
    shifts[inactive] = rng.uniform(0.05, 1.0, inactive.size)      # T = I there
    D = {}
    for compact in (1, 0):
        ctx = ofks.context_for(s, m, beta=10.0, precision=precision, pcg_compact=compact)
        D[compact] = ctx.precondition("pcg", G, shifts)
        ctx.close()
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, hartree=False, xc=False))
    Do = pr.precondition(G, shifts)
    scale = np.max(np.abs(Do))
    tol_oracle, tol_pair = (1e-10, 1e-12) if precision == "fp64" else (1e-4, 1e-5)
    assert np.max(np.abs(D[1] - Do)) < tol_oracle * scale, np.max(np.abs(D[1] - Do)) / scale
    assert np.max(np.abs(D[1] - D[0])) < tol_pair * scale, np.max(np.abs(D[1] - D[0])) / scale
    if precision == "fp64":
        assert np.array_equal(D[1][:, inactive], G[:, inactive])
    else:
        assert np.array_equal(D[1][:, inactive].astype(np.float32), G[:, inactive].astype(np.float32))


def test_staged_pcg_apply_matches_chunk_major_and_the_oracle(ofks):
    # the float32 PCG at compact width 24: the staged operator apply on row-major blocks
    # (pcg_staged = 1) and the chunk-major blocks on the type-grouped SELL (0) solve the same
    # systems; both agree with the oracle's float64 PCG to float32 accuracy
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    rng = np.random.default_rng(19)
    G = rng.standard_normal((m.n_free, s.p))
    shifts = -rng.uniform(0.05, 2.0, s.p)
    inactive = rng.choice(s.p, 19, replace=False)
    shifts[inactive] = rng.uniform(0.05, 1.0, inactive.size)
    D = {}
    for staged in (1, 0):
        ctx = ofks.context_for(s, m, beta=10.0, precision="mixed", pcg_staged=staged)
        D[staged] = ctx.precondition("pcg", G, shifts)
        ctx.close()
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, hartree=False, xc=False))
    Do = pr.precondition(G, shifts)
    scale = np.max(np.abs(Do))
    assert np.max(np.abs(D[1] - Do)) < 1e-4 * scale, np.max(np.abs(D[1] - Do)) / scale
    assert np.max(np.abs(D[1] - D[0])) < 1e-5 * scale, np.max(np.abs(D[1] - D[0])) / scale
    assert np.array_equal(D[1][:, inactive].astype(np.float32), G[:, inactive].astype(np.float32))


@pytest.mark.parametrize("case", ["chain_p41", "h2o_p5"])
def test_tensor_core_grams_match(ofks, case):
    # Lambda0 = X^T H X and S = X^T B X and the gradient G = H X + B X C with kkt (both with a
    # three-way bf16 split, six products) of the float32 form from the tensor cores, against the
    # float32 CUDA-core kernels and the float64 form, all at the same iterate
    if case == "chain_p41":
        s = I.chain(cells=(26, 14, 8))
    else:
        R = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])
        s = I.System("h2o_like", np.array([8.0, 1.0, 1.0]), R, np.full(3, -8.0), np.full(3, 8.0), (10, 10, 10), 5, 2.0)
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    ctx = ofks.context_for(s, m, beta=10.0, precision="fp64")
    ctx.init_orbitals(V)
    ctx.step(3)
    X = ctx.get_orbitals()                  # the same iterate for all three: after three steps
    ctx.close()
    res = {}
    for name, kw in (("tc", dict(precision="mixed", gram_tc=1)), ("cuda", dict(precision="mixed", gram_tc=0)),
                     ("fp64", dict(precision="fp64"))):
        ctx = ofks.context_for(s, m, beta=10.0, **kw)
        ctx.set_orbitals(X)
        r = ctx.evaluate()
        res[name] = (ctx.get_field("Lambda0"), ctx.get_field("S"), ctx.get_field("G"), r["kkt"])
        ctx.close()
    # the gradient G = H X + B X C (tensor cores: three-way bf16 split) and kkt = |H X - B X Lambda0|
    g_ref = res["fp64"][2]
    gs = np.max(np.abs(g_ref))
    assert np.max(np.abs(res["tc"][2] - g_ref)) < 1e-4 * gs, np.max(np.abs(res["tc"][2] - g_ref)) / gs
    assert np.max(np.abs(res["tc"][2] - res["cuda"][2])) < 1e-5 * gs
    assert abs(res["tc"][3] - res["fp64"][3]) < 1e-4 * res["fp64"][3]
    for k in (0, 1):
        ref = res["fp64"][k]
        scale = np.max(np.abs(ref))
        # (a two-way split, three products, was 2e-5 off)
        assert np.max(np.abs(res["tc"][k] - ref)) < 5e-6 * scale, (k, np.max(np.abs(res["tc"][k] - ref)) / scale)
        assert np.max(np.abs(res["tc"][k] - res["cuda"][k])) < 5e-6 * scale
        assert np.max(np.abs(res["tc"][k] - res["cuda"][k])) < 2e-5 * scale
        assert np.allclose(res["tc"][k], res["tc"][k].T, rtol=0, atol=1e-12 * scale)
    # and against the oracle itself at the same iterate
    check_against_oracle(s, m, X, res["tc"], 2e-5, 1e-4)


def check_against_oracle(s, m, X, got, tol_gram, tol_grad):
    """Lambda0, S, G of Eq. (lambda2)'s multipliers and kkt from the oracle at X against `got`."""
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, beta=10.0))
    H = pr.hamiltonian(pr.potentials(pr.density(X)))
    HX, BX = H @ X, pr.Bf @ X
    L0, S = pcal.sym(X.T @ HX), X.T @ BX
    G = pcal.lagrangian_gradient(HX, BX, pcal.multipliers(X, HX, BX, L0, S, 10.0), S, 10.0)
    kkt = np.linalg.norm(HX - BX @ L0)
    for k, ref in ((0, L0), (1, S)):
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got[k] - ref)) < tol_gram * scale, (k, np.max(np.abs(got[k] - ref)) / scale)
    gs = np.max(np.abs(G))
    assert np.max(np.abs(got[2] - G)) < tol_grad * gs, np.max(np.abs(got[2] - G)) / gs
    assert abs(got[3] - kkt) < tol_grad * kkt


@pytest.mark.parametrize("pw", [70, 130])
def test_wide_float32_gradient_and_grams_match(ofks, pw):
    # ld > 64 (72: two 64-column slices, the second 8 wide; 132: three): the float32 gradient
    # G = H X + B X C with kkt from the column-sliced CUDA-core kernel and the float32 Grams, against
    # the float64 form at the same iterate
    s = I.chain(cells=(26, 14, 8)).with_p(pw, occ=1.0)
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    ctx = ofks.context_for(s, m, beta=10.0, precision="fp64")
    ctx.init_orbitals(V)
    ctx.step(3)
    X = ctx.get_orbitals()
    ctx.close()
    res = {}
    for name, kw in (("f32", dict(precision="mixed")), ("fp64", dict(precision="fp64"))):
        ctx = ofks.context_for(s, m, beta=10.0, **kw)
        ctx.set_orbitals(X)
        r = ctx.evaluate()
        res[name] = (ctx.get_field("Lambda0"), ctx.get_field("S"), ctx.get_field("G"), r["kkt"])
        ctx.close()
    g_ref = res["fp64"][2]
    gs = np.max(np.abs(g_ref))
    assert np.max(np.abs(res["f32"][2] - g_ref)) < 1e-4 * gs, np.max(np.abs(res["f32"][2] - g_ref)) / gs
    assert abs(res["f32"][3] - res["fp64"][3]) < 1e-4 * res["fp64"][3]
    for k in (0, 1):
        ref = res["fp64"][k]
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(res["f32"][k] - ref)) < 2e-5 * scale, (k, np.max(np.abs(res["f32"][k] - ref)) / scale)
    check_against_oracle(s, m, X, res["f32"], 2e-5, 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cuda_graphs_match_direct_launches(ofks, precision):
    # the fixed-count PCG loop and the Hartree CG chunks replayed from captured graphs run the same
    # kernels in the same order as direct launches: the same results up to the atomics' summation
    # order, on the lattice path (chain, p = 41: compact chunk-major PCG) and at p = 2 (LiH)
    for s in (I.chain(cells=(26, 14, 8)), I.lih().with_cells((8, 8, 8))):
        m = I.make_mesh(s)
        V = I.initial_block(m.n_free, s.p, 0)
        rng = np.random.default_rng(3)
        G = rng.standard_normal((m.n_free, s.p))
        shifts = -rng.uniform(0.05, 2.0, s.p)
        shifts[::3] = 0.4                              # some columns with T = I
        out = {}
        for graphs in (1, 0):
            ctx = ofks.context_for(s, m, beta=10.0, precision=precision, cuda_graphs=graphs)
            D1 = ctx.precondition("pcg", G, shifts)
            D2 = ctx.precondition("pcg", G, shifts)    # the second call replays the captured loop
            ctx.init_orbitals(V)
            # float32 trajectories far from the minimizer diverge with the atomics' order within tens
            # of iterations whatever launches them: the mixed form is compared after 3 iterations
            r = ctx.step(30 if precision == "fp64" else 3)
            out[graphs] = (D1, D2, r["e_total"], ctx.get_orbitals())
            ctx.close()
        scale = np.max(np.abs(out[0][0]))
        tol = 1e-12 if precision == "fp64" else 1e-6
        for k in (0, 1):
            assert np.max(np.abs(out[1][k] - out[0][0])) <= tol * scale
        etol, xtol = (1e-9, 1e-6) if precision == "fp64" else (1e-6, 1e-4)
        assert abs(out[1][2] - out[0][2]) <= etol * abs(out[0][2]), (out[1][2], out[0][2])
        assert np.max(np.abs(out[1][3] - out[0][3])) <= xtol * np.max(np.abs(out[0][3]))


def test_exact_preconditioner_matches_the_oracle(ofks):
    # OFKS_PC_EXACT: the PCG of Eq. precondition-T run to a 1e-12 relative residual (float64, the
    # compact column block and all columns), against the oracle's own exact solve
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    rng = np.random.default_rng(13)
    G = rng.standard_normal((m.n_free, s.p))
    shifts = -rng.uniform(0.05, 2.0, s.p)
    inactive = rng.choice(s.p, 17, replace=False)
    shifts[inactive] = 0.3
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R,
                      pcal.Params(p=s.p, occ=s.occ, hartree=False, xc=False, precond="exact"))
    Do = pr.precondition(G, shifts)
    scale = np.max(np.abs(Do))
    for compact in (1, 0):
        ctx = ofks.context_for(s, m, beta=10.0, precision="fp64", pcg_compact=compact)
        D = ctx.precondition("exact", G, shifts)
        ctx.close()
        assert np.max(np.abs(D - Do)) < 1e-8 * scale, (compact, np.max(np.abs(D - Do)) / scale)
        assert np.array_equal(D[:, inactive], G[:, inactive])


def test_separable_pcg_solves_the_preconditioner_systems(ofks):
    # the float32 PCG of Eq. precondition-T preconditioned by the separable operator (fast
    # diagonalization on the tensor cores, all columns at once): 30 iterations reach the oracle's
    # exact T_k^-1 G_k to float32 accuracy, and 8 of them are far closer than 8 Jacobi-PCG ones
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0, precision="mixed")
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, 0))
    ctx.step(120)
    ctx.evaluate()
    G = ctx.get_field("G")
    lam = np.diag(ctx.get_field("Lambda")).copy()
    act = lam < 0
    assert act.sum() >= 4
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, precond="exact"))
    Dx = pr.precondition(G, lam)
    err = {}
    for pc, k in (("separable", 30), ("separable", 8), ("jacobi", 8)):
        ctx.set_params(pcg_pc=pc, pcg_iters=k)
        D = ctx.precondition("pcg", G, lam)
        e = np.linalg.norm(D[:, act] - Dx[:, act], axis=0) / np.linalg.norm(Dx[:, act], axis=0)
        err[(pc, k)] = float(np.max(e))
        np.testing.assert_array_equal(D[:, ~act], G[:, ~act])      # T = I columns
    assert err[("separable", 30)] < 1e-4, err
    assert err[("separable", 8)] < 0.1 * err[("jacobi", 8)], err
    ctx.close()


def test_separable_pcg_keeps_the_fixed_point(ofks):
    # only the accuracy of the directions changes: the same energy as with the Jacobi PCG, in no
    # more iterations (reduced chain, mixed form, to (kkt + fea)/kkt0 < 1e-10: at 1e-8 the
    # relative test still admits fea ~ 1e-6, an energy ~1e-5 Ha from the fixed point)
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    out = {}
    for pc in ("jacobi", "separable"):
        ctx = ofks.context_for(s, m, beta=10.0, precision="mixed", tol=1e-10, max_iter=6000, pcg_pc=pc)
        ctx.init_orbitals(V)
        r = ctx.solve()
        out[pc] = (r["iters"], r["e_total"], ctx.rayleigh_ritz())
        ctx.close()
    assert abs(out["jacobi"][1] - out["separable"][1]) < 1e-6
    np.testing.assert_allclose(out["jacobi"][2], out["separable"][2], atol=1e-5)
    assert out["separable"][0] <= out["jacobi"][0], (out["separable"][0], out["jacobi"][0])


def test_separable_pcg_in_float64(ofks):
    # the float64 PCG (row-major blocks) with the separable preconditioner: run to a tight residual
    # (exact mode) it gives the oracle's T^-1 G to float64 accuracy; with 8 iterations it is far
    # closer than the Jacobi PCG
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0)
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, 0))
    ctx.step(120)
    ctx.evaluate()
    G = ctx.get_field("G")
    lam = np.diag(ctx.get_field("Lambda")).copy()
    act = lam < 0
    assert act.sum() >= 4
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, precond="exact"))
    Dx = pr.precondition(G, lam)
    ctx.set_params(pcg_pc="separable")
    D = ctx.precondition("exact", G, lam)
    np.testing.assert_allclose(D, Dx, rtol=0, atol=1e-8 * np.max(np.abs(Dx)))
    err = {}
    for pc in ("separable", "jacobi"):
        ctx.set_params(pcg_pc=pc, pcg_iters=8)
        D = ctx.precondition("pcg", G, lam)
        err[pc] = float(np.max(np.linalg.norm(D[:, act] - Dx[:, act], axis=0) / np.linalg.norm(Dx[:, act], axis=0)))
    assert err["separable"] < 0.1 * err["jacobi"], err
    ctx.close()


@pytest.mark.parametrize("pc", ["jacobi", "separable"])
def test_type_ordered_pcg_blocks_match_the_row_major_pcg(ofks, pc):
    # the float32 PCG on chunk-major blocks whose rows are the free nodes in lattice-type order
    # (type-grouped SELL apply, type-order gathers and scatters) against the same PCG on row-major
    # blocks in the free nodes' own order (the staged apply on the main SELL, pcg_staged = 1):
    # the same operator with the same per-row summation order, so only the grouping of the
    # column sums differs
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0, precision="mixed", pcg_pc=pc)
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, 0))
    ctx.step(120)
    ctx.evaluate()
    G = ctx.get_field("G")
    lam = np.diag(ctx.get_field("Lambda")).copy()
    lam = np.where(np.arange(lam.size) % 2 == 0, lam, np.abs(lam) + 0.1)   # every other column active
    na = int((lam < 0).sum())
    assert 5 <= na <= 32                              # two chunks or more, and a width the staged form takes
    out = {}
    for staged in (0, 1):
        ctx.set_params(pcg_staged=staged, pcg_iters=8)
        out[staged] = ctx.precondition("pcg", G, lam)
    scale = np.max(np.abs(out[0]))
    assert np.max(np.abs(out[1] - out[0])) < 1e-4 * scale, np.max(np.abs(out[1] - out[0])) / scale
    # columns of non-negative multiplier take D = G in both
    np.testing.assert_array_equal(out[0][:, lam >= 0], G[:, lam >= 0])
    ctx.close()


@pytest.mark.parametrize("cells", [(6, 6, 6), (14, 10, 8)])
def test_float32_phase_hartree_potential_matches_the_oracle(ofks, cells):
    # during the float32 iterations the Hartree potential (float32 density, float64 CG to
    # poisson_tol_mixed = 1e-8 with the split tensor-core separable preconditioner) solves the
    # oracle's Poisson problem for the current orbitals
    s = I.lih().with_cells(cells).with_p(2)
    ctx, pr, V = pair(ofks, s)
    assert ctx.poisson_info()["precond"] == "separable"
    ctx.init_orbitals(V)
    g = ctx.step(4)
    assert g["switch_iter"] == -1
    ctx.evaluate()
    X = ctx.get_orbitals()
    pot = pr.potentials(pr.density(X))
    assert rel(ctx.get_field("U"), pot["U"]) < 1e-6
    ctx.close()
