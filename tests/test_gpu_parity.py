"""GPU path (libofks.so through the C ABI) against the CPU oracle on identical seeded inputs.

Tolerances (float64 on both sides, different summation order and atomic accumulation):
  * matrix products, density, Grams: relative 1e-12 of the block's scale
  * Hartree potential: the GPU solves by CG to a 1e-12 relative residual, the oracle
    exactly (direct) on these sizes: relative 1e-9
  * one PCAL step: element-wise 1e-9 relative; the first 10-15 iterates: 1e-8 relative
  * converged solves (tol 1e-10 on both sides): E within 1e-8 Ha, eigenvalues within
    1e-7 Ha, ||X^T B X - I||_F <= 1e-10
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import pcal
from paper_2007_14228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofks():
    from paper_2007_14228_gb300 import build
    build.build()
    from paper_2007_14228_gb300 import ofks as mod
    return mod


def water_like():
    # O at the origin and two H in the z = 0 plane: 10 electrons, p = 5 (ld 8 padding)
    R = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])
    return I.System("h2o_like", np.array([8.0, 1.0, 1.0]), R, np.full(3, -8.0), np.full(3, 8.0),
                    (10, 10, 10), 5, 2.0)


def small_chain():
    # 10-carbon chain on a reduced grid: p = 41 exercises the wide-block paths
    return I.chain(cells=(26, 14, 8))


CASES = {
    "lih6": lambda: I.lih().with_cells((6, 6, 6)),
    "lih10": lambda: I.lih().with_cells((10, 10, 10)),
    "h2o_p5": water_like,
    "lih8_p3": lambda: I.lih().with_cells((8, 8, 8)).with_p(3, occ=1.0),
    "chain_p41": small_chain,
}


def build_pair(ofks, system, seed=0, **params):
    m = I.make_mesh(system)
    kw = dict(beta=10.0)
    kw.update(params)
    ctx = ofks.context_for(system, m, **kw)
    okw = {k: v for k, v in kw.items() if k in pcal.Params.__dataclass_fields__}
    for k in ("hartree", "xc"):
        if k in okw:
            okw[k] = bool(okw[k])
    prm = pcal.Params(p=system.p, occ=system.occ, **okw)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, system.Z, system.R, prm)
    V = I.initial_block(m.n_free, system.p, seed)
    return ctx, pr, V, m


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("case", list(CASES))
def test_spmm_matches_oracle(ofks, case):
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s)
    X = np.random.default_rng(7).standard_normal((pr.n, s.p))
    assert rel(ctx.apply("L", X), pr.Lf @ X) < 1e-12
    assert rel(ctx.apply("B", X), pr.Bf @ X) < 1e-12
    # structural pattern: every free (i, j) pair sharing a tetrahedron (scipy drops exact zeros)
    fidx = np.full(m.n_nodes, -1)
    fidx[m.free_ids()] = np.arange(m.n_free)
    tf = fidx[m.tet10]
    a = np.repeat(tf, 10, axis=1).ravel()
    b = np.tile(tf, (1, 10)).ravel()
    keep = (a >= 0) & (b >= 0)
    assert ctx.sizes()["nnz"] == len(np.unique(a[keep].astype(np.int64) * m.n_free + b[keep]))
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_evaluate_matches_oracle(ofks, case):
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s)
    X0 = pr.initial_guess(V)
    ctx.set_orbitals(X0)
    r = ctx.evaluate()
    rho = pr.density(X0)
    pot = pr.potentials(rho)
    H = pr.hamiltonian(pot)
    assert rel(ctx.get_field("vext_q"), pr.Vext_q) < 1e-13
    assert rel(ctx.get_field("rho_q"), rho) < 1e-12
    assert rel(ctx.get_field("U"), pot["U"]) < 1e-9
    assert rel(ctx.get_field("vh_q"), pot["VH"]) < 1e-9
    assert rel(ctx.get_field("vxc_q"), pot["Vxc"]) < 1e-12
    assert rel(ctx.get_field("exc_q"), pot["eps_xc"]) < 1e-12
    HX = H @ X0
    assert rel(ctx.get_field("HX"), HX) < 1e-9
    L0 = X0.T @ HX
    assert rel(ctx.get_field("Lambda0"), 0.5 * (L0 + L0.T)) < 1e-9
    assert rel(ctx.get_field("S"), X0.T @ (pr.Bf @ X0)) < 1e-12
    E = pr.energy(X0, pot)["total"]
    assert abs(r["e_total"] - E) < 1e-9 * max(1.0, abs(E))
    # kkt and fea of Sec. 4.1
    BX = pr.Bf @ X0
    kkt = np.linalg.norm(HX - BX @ (0.5 * (L0 + L0.T)))
    assert abs(r["kkt"] - kkt) < 1e-9 * kkt
    ctx.close()


@pytest.mark.parametrize("case", ["lih6", "h2o_p5", "chain_p41"])
def test_init_matches_cholesky_gram_schmidt(ofks, case):
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s)
    ctx.init_orbitals(V)
    X0 = pr.initial_guess(V)
    assert rel(ctx.get_orbitals(), X0) < 1e-10
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_single_step_matches_oracle(ofks, case):
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s)
    X0 = pr.initial_guess(V)
    ctx.set_orbitals(X0)
    g = ctx.step(1)
    st = pcal.State(X=X0.copy())
    o = pcal.iterate(pr, st)
    assert abs(g["eta"] - st.eta) < 1e-9 * st.eta
    assert rel(ctx.get_field("D"), o["D"]) < 1e-9
    assert rel(ctx.get_orbitals(), st.X) < 1e-9
    ctx.close()


@pytest.mark.parametrize("case", ["lih6", "h2o_p5", "chain_p41"])
def test_trajectory_matches_oracle(ofks, case):
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s)
    ctx.init_orbitals(V)
    st = pcal.State(X=pr.initial_guess(V))
    for k in range(12):
        g = ctx.step(1)
        o = pcal.iterate(pr, st)
        assert abs(g["e_total"] - o["E"]) < 1e-8 * max(1.0, abs(o["E"])), (k, g["e_total"], o["E"])
        assert abs(g["kkt"] - o["kkt"]) < 1e-7 * o["kkt"], (k, g["kkt"], o["kkt"])
        assert abs(g["fea"] - o["fea"]) < 1e-7 * o["fea"] + 1e-13, (k, g["fea"], o["fea"])
    assert rel(ctx.get_orbitals(), st.X) < 1e-6
    ctx.close()


def test_converged_solve_matches_oracle(ofks):
    s = CASES["lih6"]()
    ctx, pr, V, m = build_pair(ofks, s, tol=1e-12, max_iter=4000)
    ctx.init_orbitals(V)
    res = ctx.solve()
    assert res["converged"] == 1
    E_gpu = res["e_total"]
    eig_gpu = ctx.rayleigh_ritz()
    pr.prm.max_iter = 4000
    st = pcal.solve(pr, pr.initial_guess(V))
    assert st.converged
    E_or = st.history[-1]["E"]
    eig_or, _ = pr.rayleigh_ritz(st.X)
    assert abs(E_gpu - E_or) < 1e-8, (E_gpu, E_or)
    np.testing.assert_allclose(eig_gpu, eig_or, atol=1e-7)
    assert res["fea"] <= 1e-10
    ctx.close()


def test_linear_problem_matches_dense_eigenproblem(ofks):
    s = CASES["lih6"]()
    ctx, pr, V, m = build_pair(ofks, s, hartree=0, xc=0, tol=1e-11, max_iter=4000)
    ctx.init_orbitals(V)
    ctx.solve()
    eig = ctx.rayleigh_ritz()
    H = pr.hamiltonian(pr.potentials(np.zeros_like(pr.Vext_q))).toarray()
    ref = sla.eigh(H, pr.Bf.toarray(), eigvals_only=True, subset_by_index=[0, s.p - 1])
    np.testing.assert_allclose(eig, ref, atol=1e-9)
    ctx.close()


def test_converged_wide_block_matches_dense_eigenproblem(ofks):
    # p = 41 on the reduced chain (n = 20,655), linear problem (no Hartree, no xc): the converged
    # PCAL block and Rayleigh-Ritz give the 41 lowest eigenvalues of the dense pencil (L/2 + M_ext, B)
    import scipy.sparse.linalg as spla
    s = I.chain(cells=(26, 14, 8))
    ctx, pr, V, m = build_pair(ofks, s, hartree=0, xc=0, tol=1e-11, max_iter=20000)
    ctx.init_orbitals(V)
    res = ctx.solve()
    assert res["converged"] == 1
    assert res["fea"] <= 1e-10
    eig = ctx.rayleigh_ritz()
    H = pr.hamiltonian(pr.potentials(np.zeros_like(pr.Vext_q))).tocsc()
    ref = np.sort(spla.eigsh(H, k=s.p, M=pr.Bf.tocsc(), sigma=-60.0, which="LM", return_eigenvectors=False))
    np.testing.assert_allclose(eig, ref, atol=1e-7)
    ctx.close()


def test_single_orbital_feasibility(ofks):
    s = I.hydrogenic(2.0, half=10.0, cells=(6, 6, 6), p=1)
    ctx, pr, V, m = build_pair(ofks, s)
    ctx.init_orbitals(V)
    ctx.step(60)
    h = ctx.history()
    assert np.max(h[:, 4]) < 1e-14
    ctx.close()


def test_rayleigh_ritz_keeps_energy_and_orders_eigenvalues(ofks):
    # at a converged (feasible) iterate the post-processing leaves E unchanged (Sec. 4.3)
    s = CASES["h2o_p5"]()
    ctx, pr, V, m = build_pair(ofks, s, tol=1e-10, max_iter=4000)
    ctx.init_orbitals(V)
    res = ctx.solve()
    assert res["converged"] == 1
    E0 = ctx.evaluate()["e_total"]
    eig = ctx.rayleigh_ritz()
    E1 = ctx.evaluate()["e_total"]
    assert abs(E1 - E0) < 1e-10 * max(1.0, abs(E0))
    assert np.all(np.diff(eig) >= 0)
    # the rotated block is B-orthonormal and diagonalizes X^T H X
    L0 = ctx.get_field("Lambda0")
    np.testing.assert_allclose(np.diag(L0), eig, atol=1e-9)
    assert np.max(np.abs(L0 - np.diag(np.diag(L0)))) < 1e-9
    assert np.max(np.abs(ctx.get_field("S") - np.eye(s.p))) < 1e-10
    ctx.close()


def test_state_roundtrip_continues_the_run(ofks, tmp_path):
    s = CASES["lih6"]()
    ctx, pr, V, m = build_pair(ofks, s)
    ctx.init_orbitals(V)
    ctx.step(6)
    path = str(tmp_path / "state.bin")
    ctx.save_state(path)
    ref = ctx.step(6)
    ctx2 = ofks.context_for(s, m, beta=10.0)
    ctx2.load_state(path)
    got = ctx2.step(6)
    assert got["iters"] == ref["iters"]
    assert abs(got["e_total"] - ref["e_total"]) < 1e-10 * abs(ref["e_total"])
    assert abs(got["kkt"] - ref["kkt"]) < 1e-7 * ref["kkt"]
    ctx.close()
    ctx2.close()


def test_errors_are_reported(ofks):
    s = CASES["lih6"]()
    m = I.make_mesh(s)
    ctx = ofks.Context(0)
    bad = m.tet10.copy()
    bad[3, 4] = m.n_nodes + 5
    with pytest.raises(ofks.OfksError) as e:
        ctx.set_mesh(m.xyz, bad, m.dirichlet)
    assert e.value.code == ofks.EINVAL
    ctx.set_mesh(m.xyz, m.tet10, m.dirichlet)
    with pytest.raises(ofks.OfksError) as e:
        ctx.set_params(p=m.n_free + 1)
    assert e.value.code == ofks.EINVAL
    ctx.set_params(p=2)
    with pytest.raises(ofks.OfksError) as e:
        ctx.step(1)
    assert e.value.code == ofks.ESTATE
    ctx.set_nuclei(s.Z, s.R)
    V = I.initial_block(m.n_free, 2, 0)
    V[:, 1] = V[:, 0]                      # rank deficient: no Cholesky factor
    with pytest.raises(ofks.OfksError) as e:
        ctx.init_orbitals(V)
    assert e.value.code == ofks.ENOTCONV
    ctx.close()


def _rows_by_local_assembly(m, rows_free, X):
    """(L X)[rows], (B X)[rows] from the oracle's element matrices of the touching tets only."""
    from oracle import fem
    free = m.free_ids()
    fidx = np.full(m.n_nodes, -1)
    fidx[free] = np.arange(len(free))
    want = set(rows_free.tolist())
    tf = fidx[m.tet10]
    touch = np.nonzero(np.isin(tf, rows_free).any(axis=1))[0]
    t = m.tet10[touch]
    tff = tf[touch]
    vol, glam = fem.tet_geometry(m.xyz, t)
    g = fem.basis_gradients(fem.quad_bary(), glam)
    Lloc = np.einsum("t,tqad,tqbd->tab", vol / 4.0, g, g)
    Bloc = vol[:, None, None] * fem.reference_mass()[None]
    pos = {r: i for i, r in enumerate(rows_free.tolist())}
    LX = np.zeros((len(rows_free), X.shape[1]))
    BX = np.zeros_like(LX)
    for e in range(len(t)):
        for a in range(10):
            ra = tff[e, a]
            if ra < 0 or ra not in want:
                continue
            for b in range(10):
                rb = tff[e, b]
                if rb < 0:
                    continue
                LX[pos[ra]] += Lloc[e, a, b] * X[rb]
                BX[pos[ra]] += Bloc[e, a, b] * X[rb]
    return LX, BX


def test_full_size_chain_sampled_rows_and_invariants(ofks):
    # the bench workload (C10H22 chain, 80 x 44 x 43 cells, p = 41) in the bench's launch
    # configuration: sampled SpMM rows and densities against the oracle, invariants of the step
    from oracle import fem, xc
    s = I.chain()
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0)
    V = I.initial_block(m.n_free, s.p, 0)
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(m.n_free, 64, replace=False))
    LXg = ctx.apply("L", V)
    BXg = ctx.apply("B", V)
    LXo, BXo = _rows_by_local_assembly(m, rows, V)
    assert rel(LXg[rows], LXo) < 1e-12
    assert rel(BXg[rows], BXo) < 1e-12
    ctx.set_orbitals(V)
    ctx.evaluate()
    rho_g = ctx.get_field("rho_q")
    tets = rng.choice(m.n_tets, 200, replace=False)
    Va = np.zeros((m.n_nodes, s.p))
    Va[m.free_ids()] = V
    psi = fem.values_at_quad(Va, m.tet10[tets])
    rho_o = s.occ * np.sum(psi * psi, axis=2)
    assert rel(rho_g[tets], rho_o) < 1e-12
    eps_o, vxc_o = xc.lda(rho_o)
    assert rel(ctx.get_field("vxc_q")[tets], vxc_o) < 1e-12
    # invariants after steps: unit B-norm columns, symmetric multipliers
    ctx.init_orbitals(V)
    ctx.step(2)
    ctx.evaluate()
    S = ctx.get_field("S")
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-12
    L0 = ctx.get_field("Lambda0")
    assert np.max(np.abs(L0 - L0.T)) == 0.0
    ctx.close()


def test_full_size_lih_first_steps_match_oracle(ofks):
    # the 24^3 LiH workload: three iterations against the oracle (CG Hartree at this size)
    s = I.lih()
    ctx, pr, V, m = build_pair(ofks, s)
    ctx.init_orbitals(V)
    st = pcal.State(X=pr.initial_guess(V))
    for k in range(3):
        g = ctx.step(1)
        o = pcal.iterate(pr, st)
        assert abs(g["e_total"] - o["E"]) < 1e-9 * abs(o["E"]), (k, g["e_total"], o["E"])
        assert abs(g["kkt"] - o["kkt"]) < 1e-8 * o["kkt"]
    ctx.close()


@pytest.mark.parametrize("pc,max_iters", [("jacobi", 2000), ("multigrid", 400), ("separable", 60)])
def test_hartree_preconditioners_agree_with_oracle(ofks, pc, max_iters):
    # the Hartree CG with the Jacobi, multigrid or separable preconditioner reaches the same
    # potential; the separable one keeps the count near twenty on the graded lattice
    s = CASES["chain_p41"]()
    ctx, pr, V, m = build_pair(ofks, s, poisson_pc=pc)
    assert ctx.poisson_info()["precond"] == pc
    X0 = pr.initial_guess(V)
    ctx.set_orbitals(X0)
    r = ctx.evaluate()
    pot = pr.potentials(pr.density(X0))
    assert rel(ctx.get_field("U"), pot["U"]) < 1e-9
    assert 0 < r["hartree_iters"] < max_iters, r["hartree_iters"]
    ctx.close()


@pytest.mark.parametrize("case", ["lih10", "chain_p41"])
@pytest.mark.parametrize("csr", [0, 1])
def test_hartree_lattice_and_csr_forms_agree_with_oracle(ofks, case, csr):
    # the lattice-stencil SpMV (symmetric half, no column indices) and the CSR give the oracle's
    # potential; the lattice form is the default on these meshes
    s = CASES[case]()
    ctx, pr, V, m = build_pair(ofks, s, poisson_csr=csr)
    info = ctx.poisson_info()
    assert info["format"] == ("csr" if csr else "lattice"), info
    assert info["lattice"] == tuple(m.lattice)
    assert info["rows"] == int(np.sum(m.dirichlet == 0))
    X0 = pr.initial_guess(V)
    ctx.set_orbitals(X0)
    ctx.evaluate()
    pot = pr.potentials(pr.density(X0))
    assert rel(ctx.get_field("U"), pot["U"]) < 1e-9
    ctx.close()


@pytest.mark.parametrize("pc,used", [("separable", "jacobi"), ("multigrid", "multigrid")])
def test_hartree_on_renumbered_mesh_uses_csr(ofks, pc, used):
    # node ids that do not follow a lattice: the CSR form runs (the separable preconditioner
    # falls back to Jacobi, multigrid to smoothed aggregation) and still matches the oracle
    s = CASES["lih10"]()
    m0 = I.make_mesh(s)
    perm = np.random.default_rng(3).permutation(len(m0.xyz))     # new id -> old id
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    m = I.Mesh(m0.xyz[perm].copy(), inv[m0.tet10], m0.dirichlet[perm].copy(), m0.lattice, m0.axes)
    ctx = ofks.context_for(s, m, beta=10.0, poisson_pc=pc)
    assert ctx.poisson_info()["format"] == "csr"
    assert ctx.poisson_info()["precond"] == used
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, beta=10.0))
    X0 = pr.initial_guess(I.initial_block(m.n_free, s.p, 0))
    ctx.set_orbitals(X0)
    ctx.evaluate()
    pot = pr.potentials(pr.density(X0))
    assert rel(ctx.get_field("U"), pot["U"]) < 1e-9
    ctx.close()


@pytest.mark.parametrize("case", ["lih10", "chain_p41"])
def test_separable_preconditioner_tensor_cores_match_cuda_cores(ofks, case):
    # the tensor-core contractions (bf16 operands, every intermediate tensor as a high and a low
    # bf16 part) and the float32 CUDA-core ones precondition the same CG: both reach the oracle's
    # potential in nearly the same number of iterations
    s = CASES[case]()
    iters = {}
    for tc in (1, 0):
        ctx, pr, V, m = build_pair(ofks, s, poisson_sep_tc=tc)
        assert ctx.poisson_info()["precond"] == "separable"
        X0 = pr.initial_guess(V)
        ctx.set_orbitals(X0)
        r = ctx.evaluate()
        pot = pr.potentials(pr.density(X0))
        assert rel(ctx.get_field("U"), pot["U"]) < 1e-9
        iters[tc] = r["hartree_iters"]
        ctx.close()
    assert abs(iters[1] - iters[0]) <= max(3, iters[0] // 5), iters
