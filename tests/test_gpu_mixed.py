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
