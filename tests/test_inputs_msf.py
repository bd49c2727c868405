"""The mesh-size-function grading of the input meshes (paper Eq. meshsizefunction, Sec. 4.2).

h(r) = min_j gamma1 Z_j^(-2/5) r_j^(6/5), capped at gamma2, sets the shape of the spacing along
each axis (scaled to the cell budget, held at its value 0.05 bohr from the largest charge
nearer than that).  The checks: the spacing grows as r^(6/5) away from a nucleus, heavier
nuclei get finer cells at the same distance (Z^(-2/5)), the axis is a valid grid with every
nucleus on a vertex, and on a carbon-like hydrogenic ion the 1s level is closer to -Z^2/2 than on
the tanh-graded grid of the same size.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import pcal
from paper_2007_14228_gb300 import inputs as I


def spacing_at(v, x):
    """Cell width of the cell containing x."""
    k = np.searchsorted(v, x) - 1
    return v[k + 1] - v[k], 0.5 * (v[k] + v[k + 1])


def test_spacing_follows_the_six_fifths_power():
    v = I.axis_vertices_msf(-12.0, 12.0, 400, [0.0], [6.0])
    h1, m1 = spacing_at(v, 1.0)
    h4, m4 = spacing_at(v, 4.0)
    assert h4 / h1 == pytest.approx((m4 / m1) ** 1.2, rel=0.05)


def test_heavier_nucleus_gets_finer_cells():
    # a Z = 8 and a Z = 1 nucleus 10 bohr apart: at 1.5 bohr from each, widths in the ratio 8^(-2/5)
    v = I.axis_vertices_msf(-12.0, 22.0, 600, [0.0, 10.0], [8.0, 1.0])
    ha, ma = spacing_at(v, 1.5)
    hb, mb = spacing_at(v, 8.5)
    ratio = (ha / abs(ma) ** 1.2) / (hb / abs(mb - 10.0) ** 1.2)
    assert ratio == pytest.approx(8.0 ** -0.4, rel=0.05)


@pytest.mark.parametrize("name", ["lih", "chain", "lattice60"])
def test_axis_is_a_valid_grid_with_nuclei_on_vertices(name):
    s = I.SYSTEMS[name]()
    for d in range(3):
        v = I.axis_vertices_msf(s.box_lo[d], s.box_hi[d], s.cells[d], s.R[:, d], s.Z)
        assert len(v) == s.cells[d] + 1 and np.all(np.diff(v) > 0)
        assert v[0] == s.box_lo[d] and v[-1] == s.box_hi[d]
        for x in set(np.round(s.R[:, d], 9)):
            assert np.min(np.abs(v - x)) < 0.3       # every nucleus on (or merged onto) a vertex


def _level(system, grading):
    m = I.make_mesh(system, grading=grading)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, system.Z, system.R,
                      pcal.Params(p=1, occ=1.0, hartree=False, xc=False))
    H = pr.hamiltonian(pr.potentials(np.zeros_like(pr.Vext_q)))
    w = spla.eigsh(H.tocsc(), k=1, M=pr.Bf.tocsc(), sigma=-2.0 * system.Z[0] ** 2, which="LM",
                   return_eigenvectors=False)
    return w[0]


def test_size_function_grid_resolves_a_carbon_core_better():
    s = I.hydrogenic(6.0, half=10.0, cells=(12, 12, 12))
    exact = -18.0
    assert abs(_level(s, "msf") - exact) < abs(_level(s, "tanh") - exact)
