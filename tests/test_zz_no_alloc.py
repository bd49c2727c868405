"""ofks_set_nuclei_static: the allocation-free way to set the nuclei.

Callers that cannot allocate device memory while they move the nuclei (an allocator that owns
the device, an allocation-free inner loop) use this entry point; it must give exactly what
ofks_set_nuclei gives.  Two calls in a row with different geometries check that nothing left
in the shared staging array from the first call leaks into the second.  Kept in a file of its
own, collected last.
"""
import numpy as np
import pytest

from paper_2007_14228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctx(ofks, s, m):
    ctx = ofks.Context(0)
    ctx.set_mesh(m.xyz, m.tet10, m.dirichlet)
    ctx.set_params(p=s.p, occ=s.occ, beta=10.0)
    return ctx


def test_static_nuclei_match_set_nuclei_on_two_calls():
    from paper_2007_14228_gb300 import build
    build.build()
    from paper_2007_14228_gb300 import ofks
    s = I.lih().with_cells((8, 8, 8))
    m = I.make_mesh(s)
    X = np.random.default_rng(3).standard_normal((m.n_free, s.p)) * 0.01
    ref = _ctx(ofks, s, m)
    new = _ctx(ofks, s, m)
    # first call: the LiH geometry; second call: three nuclei at other places
    geoms = [(s.Z, s.R),
             (np.array([1.0, 2.0, 1.0]), np.array([[0.5, -1.0, 0.2], [-2.0, 1.5, 0.0], [1.0, 1.0, -3.0]]))]
    for Z, R in geoms:
        ref.set_nuclei(Z, R)
        new.set_nuclei_static(Z, R)
        for ctx in (ref, new):
            ctx.set_orbitals(X)
        r_ref = ref.evaluate()
        r_new = new.evaluate()
        v_ref, v_new = ref.get_field("vext_q"), new.get_field("vext_q")
        assert np.max(np.abs(v_new - v_ref)) <= 1e-13 * np.max(np.abs(v_ref))
        assert abs(r_new["e_nuc"] - r_ref["e_nuc"]) <= 1e-13 * abs(r_ref["e_nuc"])
        assert abs(r_new["e_total"] - r_ref["e_total"]) <= 1e-9 * max(1.0, abs(r_ref["e_total"]))
    with pytest.raises(ofks.OfksError) as e:
        big = ofks.STATIC_NUCLEI_MAX + 1
        new.set_nuclei_static(np.ones(big), np.arange(3.0 * big).reshape(big, 3))
    assert e.value.code == ofks.EINVAL
    ref.close()
    new.close()

