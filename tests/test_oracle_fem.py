"""Pins of the oracle's P2 element and assembly against exact integrals.

Quadratic polynomials lie in the P2 space, so their nodal interpolants reproduce them
exactly; the mass and stiffness forms of such functions equal closed-form integrals
over the box.  A wrong basis function, gradient, quadrature point or volume breaks one.
"""
import os

import numpy as np
import pytest

from oracle import fem
from paper_2007_14228_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_reference_mass_matches_textbook_table():
    ref = np.loadtxt(os.path.join(GOLDEN, "p2_tet_mass_x420.txt"))
    np.testing.assert_allclose(fem.reference_mass() * 420.0, ref, rtol=0, atol=1e-12)


def test_basis_partition_of_unity_and_nodality():
    rng = np.random.default_rng(1)
    lam = rng.dirichlet(np.ones(4), size=50)
    np.testing.assert_allclose(fem.basis_values(lam).sum(axis=1), 1.0, atol=1e-14)
    nodes = np.zeros((10, 4))
    for a in range(4):
        nodes[a, a] = 1.0
    for e, (a, b) in enumerate(fem.EDGES):
        nodes[4 + e, a] = nodes[4 + e, b] = 0.5
    np.testing.assert_allclose(fem.basis_values(nodes), np.eye(10), atol=1e-15)


def test_quadrature_exact_for_degree_two():
    # sum_q w_q f(x_q) on one tet equals the exact integral of lam_a lam_b (monomial formula)
    lam = fem.quad_bary()
    w = np.full(4, 0.25)          # weights / |T|
    for a in range(4):
        for b in range(4):
            exact = (2.0 if a == b else 1.0) / 20.0    # 6 * a!b!/5! with |alpha| = 2
            assert abs(np.sum(w * lam[:, a] * lam[:, b]) - exact) < 1e-15


@pytest.fixture(scope="module")
def box_mesh():
    s = I.lih().with_cells((6, 4, 5))
    m = I.make_mesh(s)
    L, B = fem.assemble_LB(m.xyz, m.tet10)
    return s, m, L, B


def _box_integral(lo, hi, px, py, pz):
    """Exact integral of x^px y^py z^pz over the box."""
    out = 1.0
    for d, k in enumerate((px, py, pz)):
        out *= (hi[d] ** (k + 1) - lo[d] ** (k + 1)) / (k + 1)
    return out


def test_volume_and_constant_in_kernel(box_mesh):
    s, m, L, B = box_mesh
    one = np.ones(m.n_nodes)
    vol = np.prod(s.box_hi - s.box_lo)
    assert abs(one @ (B @ one) - vol) < 1e-9 * vol
    assert np.max(np.abs(L @ one)) < 1e-10


def test_mass_and_stiffness_of_quadratics(box_mesh):
    s, m, L, B = box_mesh
    lo, hi = s.box_lo, s.box_hi
    x, y, z = m.xyz.T
    # u = x^2 + y z - 2 z: int u^2 and int |grad u|^2 in closed form
    u = x ** 2 + y * z - 2.0 * z
    uu = (_box_integral(lo, hi, 4, 0, 0) + _box_integral(lo, hi, 0, 2, 2) + 4 * _box_integral(lo, hi, 0, 0, 2)
          + 2 * _box_integral(lo, hi, 2, 1, 1) - 4 * _box_integral(lo, hi, 2, 0, 1)
          - 4 * _box_integral(lo, hi, 0, 1, 2))
    assert abs(u @ (B @ u) - uu) < 1e-9 * abs(uu)
    # grad u = (2x, z, y - 2)
    gg = (4 * _box_integral(lo, hi, 2, 0, 0) + _box_integral(lo, hi, 0, 0, 2) + _box_integral(lo, hi, 0, 2, 0)
          - 4 * _box_integral(lo, hi, 0, 1, 0) + 4 * _box_integral(lo, hi, 0, 0, 0))
    assert abs(u @ (L @ u) - gg) < 1e-9 * abs(gg)
    # bilinear cross term with a second quadratic v = x y
    v = x * y
    uv = (_box_integral(lo, hi, 3, 1, 0) + _box_integral(lo, hi, 1, 2, 1) - 2 * _box_integral(lo, hi, 1, 1, 1))
    scale = np.sqrt(uu * (v @ (B @ v)))
    assert abs(u @ (B @ v) - uv) < 1e-12 * scale


def test_values_at_quadrature_reproduce_quadratics(box_mesh):
    s, m, L, B = box_mesh
    x, y, z = m.xyz.T
    u = 3 * x * z - y ** 2 + 0.5
    xq = fem.quad_points(m.xyz, m.tet10)
    uq = fem.values_at_quad(u, m.tet10)
    exact = 3 * xq[..., 0] * xq[..., 2] - xq[..., 1] ** 2 + 0.5
    np.testing.assert_allclose(uq, exact, atol=1e-11)


def test_potential_matrix_of_constant_is_mass_quadrature(box_mesh):
    # M_V with V = 1 integrates N_i N_j by the 4-point rule: exact for v^T M u with u, v linear
    s, m, L, B = box_mesh
    vol, _ = fem.tet_geometry(m.xyz, m.tet10)
    pa = fem.PotentialAssembler(m.n_nodes, m.tet10, vol)
    M1 = pa.assemble(np.ones((m.n_tets, 4)))
    x, y, z = m.xyz.T
    lo, hi = s.box_lo, s.box_hi
    assert abs(x @ (M1 @ y) - _box_integral(lo, hi, 1, 1, 0)) < 1e-9
    # V = x: int V u v for u = y, v = 1 is degree 2 -> exact
    M2 = pa.assemble(xq_x := fem.quad_points(m.xyz, m.tet10)[..., 0])
    assert abs(y @ (M2 @ np.ones(m.n_nodes)) - _box_integral(lo, hi, 1, 1, 0)) < 1e-9
    assert xq_x.shape == (m.n_tets, 4)


def test_mesh_structure():
    s = I.lih().with_cells((6, 7, 5))
    m = I.make_mesh(s)
    sz = I.sizes(s)
    assert m.n_free == sz["n"] and m.n_nodes == sz["n_nodes"] and m.n_tets == sz["n_tets"]
    vol, _ = fem.tet_geometry(m.xyz, m.tet10)
    assert np.all(vol > 0)
    assert abs(vol.sum() - np.prod(s.box_hi - s.box_lo)) < 1e-9
    # every nucleus is a mesh vertex
    for R in s.R:
        assert np.min(np.linalg.norm(m.xyz - R, axis=1)) < 1e-12
    # conforming: every interior face is shared by exactly two tets
    faces = np.sort(m.tet10[:, [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]].reshape(-1, 3), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert set(np.unique(counts)) <= {1, 2}
    n_bnd_faces = np.sum(counts == 1)
    Nx, Ny, Nz = s.cells
    assert n_bnd_faces == 4 * (Nx * Ny + Ny * Nz + Nx * Nz)
