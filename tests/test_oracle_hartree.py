"""Pins of the oracle's Hartree solve against the Gaussian-charge closed form.

rho = Q (a/pi)^{3/2} exp(-a |x - c|^2) has V_H = Q erf(sqrt(a) r)/r and
E_H = (1/2) int V_H rho = Q^2 sqrt(a / (2 pi)).  The discretization error shrinks under
mesh refinement; the multipole boundary values match the exact far field.
"""
import numpy as np
import pytest
from scipy.special import erf

from oracle import fem
from oracle.hartree import Hartree
from paper_2007_14228_gb300 import inputs as I


def _setup(cells, lmax=2, half=10.0):
    s = I.hydrogenic(1.0, half=half, cells=cells)
    m = I.make_mesh(s)
    L, _ = fem.assemble_LB(m.xyz, m.tet10)
    vol, _ = fem.tet_geometry(m.xyz, m.tet10)
    xq = fem.quad_points(m.xyz, m.tet10)
    return m, Hartree(m.xyz, m.tet10, m.dirichlet, L, vol, xq, lmax), vol, xq


def _gauss(x, c, Q, a):
    r2 = ((x - c) ** 2).sum(axis=-1)
    return Q * (a / np.pi) ** 1.5 * np.exp(-a * r2)


def _vexact(x, c, Q, a):
    r = np.sqrt(((x - c) ** 2).sum(axis=-1))
    return Q * erf(np.sqrt(a) * r) / r


@pytest.mark.parametrize("cells", [(12, 12, 12)])
def test_gaussian_charge_potential_and_energy(cells):
    Q, a, c = 2.0, 1.0, np.zeros(3)
    m, h, vol, xq = _setup(cells)
    rho = _gauss(xq, c, Q, a)
    U = h.solve(rho)
    VH = fem.values_at_quad(U, m.tet10)
    w = vol[:, None] / 4.0
    EH = 0.5 * np.sum(w * VH * rho)
    EH_exact = Q * Q * np.sqrt(a / (2.0 * np.pi))
    err_E = abs(EH - EH_exact) / EH_exact
    err_V = np.max(np.abs(VH - _vexact(xq, c, Q, a)))
    tol = {12: (2.5e-2, 5e-2)}[cells[0]]
    assert err_E < tol[0], err_E
    assert err_V < tol[1], err_V


def test_refinement_reduces_error():
    Q, a, c = 2.0, 1.0, np.zeros(3)
    errs = []
    for cells in [(8, 8, 8), (10, 10, 10), (12, 12, 12)]:
        m, h, vol, xq = _setup(cells)
        rho = _gauss(xq, c, Q, a)
        VH = fem.values_at_quad(h.solve(rho), m.tet10)
        EH = 0.5 * np.sum(vol[:, None] / 4.0 * VH * rho)
        errs.append(abs(EH - Q * Q * np.sqrt(a / (2 * np.pi))))
    assert errs[0] > errs[1] > errs[2]


def test_multipole_boundary_values_match_far_field():
    # off-centre charge: compare with the brute-force Coulomb sum of the same quadrature
    # charges; the l <= 2 expansion leaves only the O(a^3/R^4) octupole remainder
    Q, a, c = 2.0, 1.0, np.array([1.0, 0.5, -0.3])
    m, h2, vol, xq = _setup((8, 8, 8), lmax=2)
    _, h0, _, _ = _setup((8, 8, 8), lmax=0)
    rho = _gauss(xq, c, Q, a)
    xb = m.xyz[h2.Bd]
    wq = np.repeat(vol / 4.0, 4) * rho.ravel()
    pts = xq.reshape(-1, 3)
    exact = np.array([np.sum(wq / np.sqrt(((pts - x) ** 2).sum(axis=1))) for x in xb])
    e2 = np.max(np.abs(h2.boundary_values(rho) - exact))
    e0 = np.max(np.abs(h0.boundary_values(rho) - exact))
    assert e2 < 1e-3 and e2 < e0 / 10.0, (e2, e0)
    # moments of the quadrature charge against the analytic moments of the Gaussian
    Qm, d, Qij = h2.moments(rho)
    assert abs(Qm - Q) < 0.05 * Q
    yc = c - h2.center
    np.testing.assert_allclose(d / Qm, yc, atol=0.05)


def test_zero_boundary_map_is_symmetric():
    # with homogeneous Dirichlet data rho -> int V_H[rho] sigma is symmetric in (rho, sigma)
    m, h, vol, xq = _setup((5, 5, 5), lmax=-1)
    rng = np.random.default_rng(3)
    r1, r2 = rng.random(xq.shape[:2]), rng.random(xq.shape[:2])
    w = vol[:, None] / 4.0
    a12 = np.sum(w * fem.values_at_quad(h.solve(r1), m.tet10) * r2)
    a21 = np.sum(w * fem.values_at_quad(h.solve(r2), m.tet10) * r1)
    assert abs(a12 - a21) < 1e-10 * abs(a12)


def test_cg_path_matches_direct_solve():
    Q, a, c = 2.0, 1.0, np.array([0.5, -0.2, 0.1])
    s = I.hydrogenic(1.0, half=10.0, cells=(10, 10, 10))
    m = I.make_mesh(s)
    L, _ = fem.assemble_LB(m.xyz, m.tet10)
    vol, _ = fem.tet_geometry(m.xyz, m.tet10)
    xq = fem.quad_points(m.xyz, m.tet10)
    rho = _gauss(xq, c, Q, a)
    Ud = Hartree(m.xyz, m.tet10, m.dirichlet, L, vol, xq, 2, solver="direct").solve(rho)
    Uc = Hartree(m.xyz, m.tet10, m.dirichlet, L, vol, xq, 2, solver="cg").solve(rho)
    assert np.max(np.abs(Ud - Uc)) < 1e-10 * np.max(np.abs(Ud))


def test_moments_equal_the_node_sum_over_the_load():
    # Every multipole moment function (1, y, 3 y_i y_j - |y|^2 delta_ij) is quadratic and P2 on a
    # straight-sided tetrahedron interpolates quadratics exactly, so the quadrature moments equal
    # sum_i f(y_i) b_i with the load b_i = sum_T sum_q w_q rho_q N_i(x_q): the identity the GPU
    # uses to get the moments from the assembled Poisson load (one pass over the nodes)
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    L, _ = fem.assemble_LB(m.xyz, m.tet10)
    vol, _ = fem.tet_geometry(m.xyz, m.tet10)
    xq = fem.quad_points(m.xyz, m.tet10)
    h = Hartree(m.xyz, m.tet10, m.dirichlet, L, vol, xq, 2)
    rho = np.random.default_rng(5).uniform(0.0, 2.0, (m.tet10.shape[0], 4))
    Q, d, Qij = h.moments(rho)
    b = fem.quad_to_nodes(rho, m.tet10, vol, m.xyz.shape[0])
    y = m.xyz - h.center
    r2 = (y * y).sum(axis=1)
    Qn, dn = b.sum(), (b[:, None] * y).sum(axis=0)
    Qijn = 3.0 * np.einsum("i,ij,ik->jk", b, y, y) - np.eye(3) * (b * r2).sum()
    assert abs(Qn - Q) <= 1e-12 * abs(Q)
    scale = np.sqrt((y * y).sum(axis=1)).max()
    assert np.max(np.abs(dn - d)) <= 1e-12 * abs(Q) * scale
    assert np.max(np.abs(Qijn - Qij)) <= 1e-12 * abs(Q) * scale ** 2
    # a dropped or wrong-signed term of the identity breaks it: the moments of a shifted origin differ
    assert np.max(np.abs(3.0 * np.einsum("i,ij,ik->jk", b, y + 0.1, y + 0.1) - np.eye(3) * (b * ((y + 0.1) ** 2).sum(axis=1)).sum() - Qij)) > 1e-6 * abs(Q)
