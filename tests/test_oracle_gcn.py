"""Pins of the oracle's learned-preconditioner network.

* with its zero-initialized last layer the network returns exactly the Jacobi step G / diag
* the hand-written backward equals central finite differences of the loss
* a few Adam steps on exact preconditioned directions T^{-1} G lower the loss
* the energy-norm loss: 1 for D = 0 on every column of negative shift (E = -D*, and
  D*^T T D* = G^T D* because T D* = G), 0 for D = D*, blind to the columns of non-negative shift,
  and its backward equals central finite differences
"""
import numpy as np
import pytest

from oracle import gcn, pcal
from paper_2007_14228_gb300 import inputs as I


@pytest.fixture(scope="module")
def tiny():
    s = I.lih().with_cells((6, 4, 4))
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=2, hartree=False, xc=False,
                                                                          precond="exact"))
    A = gcn.mean_aggregator(gcn.dof_graph(m.tet10, m.dirichlet))
    rng = np.random.default_rng(4)
    G = rng.standard_normal((pr.n, 2))
    shifts = np.array([-0.8, -0.2])
    Dstar = pr.precondition(G, shifts)
    return pr, A, G, shifts, Dstar


def test_aggregator_rows_average(tiny):
    pr, A, *_ = tiny
    np.testing.assert_allclose(A @ np.ones(pr.n), 1.0, atol=1e-14)


def test_initial_network_is_the_jacobi_step(tiny):
    pr, A, G, shifts, _ = tiny
    f, s, diag = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts)
    D, _, _ = gcn.predict(gcn.init_params(width=8), f, s, A)
    np.testing.assert_allclose(D, G / diag, rtol=1e-13)


def test_backward_matches_finite_differences(tiny):
    pr, A, G, shifts, Dstar = tiny
    f, s, _ = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts)
    params = gcn.init_params(width=6, seed=1)
    rng = np.random.default_rng(9)
    params[2]["W"] = 0.1 * rng.standard_normal(params[2]["W"].shape)
    params[2]["U"] = 0.1 * rng.standard_normal(params[2]["U"].shape)

    def loss_of(pp):
        D, _, _ = gcn.predict(pp, f, s, A)
        return gcn.loss_and_dy(D, Dstar, s)[0]

    D, y, cache = gcn.predict(params, f, s, A)
    _, dy = gcn.loss_and_dy(D, Dstar, s)
    grads = gcn.backward(params, cache, dy, A)
    h = 1e-6
    for (l, k, idx) in [(0, "W", (1, 2)), (0, "U", (0, 3)), (1, "W", (4, 5)), (1, "b", (2,)), (2, "U", (3, 0)),
                        (2, "b", (0,)), (0, "b", (1,)), (1, "U", (0, 1))]:
        pp = [{kk: v.copy() for kk, v in P.items()} for P in params]
        pp[l][k][idx] += h
        lp = loss_of(pp)
        pp[l][k][idx] -= 2 * h
        lm = loss_of(pp)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[l][k][idx]) < 1e-6 * max(1.0, abs(fd)), (l, k, idx, fd, grads[l][k][idx])


def test_adam_steps_reduce_the_loss(tiny):
    pr, A, G, shifts, Dstar = tiny
    f, s, _ = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts)
    params = gcn.init_params(width=16, seed=2)
    state = {}
    D, _, _ = gcn.predict(params, f, s, A)
    l0 = gcn.loss_and_dy(D, Dstar, s)[0]
    for _ in range(60):
        D, y, cache = gcn.predict(params, f, s, A)
        _, dy = gcn.loss_and_dy(D, Dstar, s)
        params = gcn.adam_step(params, gcn.backward(params, cache, dy, A), state, lr=3e-3)
    D, _, _ = gcn.predict(params, f, s, A)
    assert gcn.loss_and_dy(D, Dstar, s)[0] < 0.7 * l0


def test_dof_graph_is_the_mesh_adjacency():
    # the graph holds every nonzero of the stiffness and the Kuhn-split P2 neighbourhoods:
    # an interior cell vertex sees itself, its 14 edge neighbours, the 14 midpoints of those
    # edges and the 36 midpoints of the edges of its link (a triangulated sphere with 14 vertices
    # and 24 triangles, so 36 edges by Euler's formula): 65 DoFs
    s = I.lih().with_cells((6, 4, 4))
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=2, hartree=False, xc=False))
    Gr = gcn.dof_graph(m.tet10, m.dirichlet)
    Lnz = pr.Lf.tocsr()
    Lnz.data[:] = 1.0
    assert (Lnz - Lnz.multiply(Gr)).nnz == 0
    Lx, Ly, Lz = m.lattice
    free = np.cumsum(m.dirichlet == 0) - 1
    v = free[(4 * Ly + 4) * Lz + 4]
    assert np.diff(Gr.indptr)[v] == 65


def energy_case(tiny, shifts3):
    pr, A, *_ = tiny
    rng = np.random.default_rng(11)
    G = rng.standard_normal((pr.n, 3))
    Dstar = pr.precondition(G, shifts3)
    f, s, _ = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts3)
    return pr, A, G, Dstar, f, s


def test_energy_loss_of_the_zero_direction_is_one(tiny):
    shifts3 = np.array([-0.8, 0.3, -0.2])          # the middle column has T = I and is left out
    pr, A, G, Dstar, f, s = energy_case(tiny, shifts3)
    loss, dy = gcn.energy_loss_and_dy(np.zeros_like(G), Dstar, G, s, pr.Lf, pr.Bf, shifts3)
    assert abs(loss - 1.0) < 1e-10
    assert np.all(dy[:, 1] == 0.0)
    loss0, _ = gcn.energy_loss_and_dy(Dstar, Dstar, G, s, pr.Lf, pr.Bf, shifts3)
    assert loss0 == 0.0
    # a column's loss is the squared energy norm of its error relative to that of D*: half of D*
    # leaves a quarter
    loss_half, _ = gcn.energy_loss_and_dy(0.5 * Dstar, Dstar, G, s, pr.Lf, pr.Bf, shifts3)
    assert abs(loss_half - 0.25) < 1e-10


def test_energy_backward_matches_finite_differences(tiny):
    shifts3 = np.array([-0.8, 0.3, -0.2])
    pr, A, G, Dstar, f, s = energy_case(tiny, shifts3)
    params = gcn.init_params(width=6, seed=3)
    rng = np.random.default_rng(12)
    params[2]["W"] = 0.1 * rng.standard_normal(params[2]["W"].shape)
    params[2]["U"] = 0.1 * rng.standard_normal(params[2]["U"].shape)

    def loss_of(pp):
        D, _, _ = gcn.predict(pp, f, s, A)
        return gcn.energy_loss_and_dy(D, Dstar, G, s, pr.Lf, pr.Bf, shifts3)[0]

    D, y, cache = gcn.predict(params, f, s, A)
    _, dy = gcn.energy_loss_and_dy(D, Dstar, G, s, pr.Lf, pr.Bf, shifts3)
    grads = gcn.backward(params, cache, dy, A)
    h = 1e-6
    for (l, k, idx) in [(0, "W", (2, 1)), (0, "U", (1, 3)), (1, "W", (3, 5)), (1, "b", (4,)), (2, "U", (2, 0)),
                        (2, "b", (0,)), (2, "W", (5, 0))]:
        pp = [{kk: v.copy() for kk, v in P.items()} for P in params]
        pp[l][k][idx] += h
        lp = loss_of(pp)
        pp[l][k][idx] -= 2 * h
        lm = loss_of(pp)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[l][k][idx]) < 1e-6 * max(1.0, abs(fd)), (l, k, idx, fd, grads[l][k][idx])
