"""The C-ABI library builds, loads without a GPU and exports every entry point of include/ofks.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_14228_gb300 import build, ofks
    path = build.build()
    return ofks.load(path)


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ofks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ofks_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("ofks_create", "ofks_set_mesh", "ofks_set_nuclei", "ofks_set_params", "ofks_init_orbitals",
                 "ofks_solve", "ofks_step", "ofks_rayleigh_ritz", "ofks_get_orbitals", "ofks_get_history",
                 "ofks_save_state", "ofks_load_state", "ofks_last_error", "ofks_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2007_14228_gb300 import ofks
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(ofks.SYMBOLS) <= set(declared_symbols())


def test_default_params_without_gpu(lib):
    from paper_2007_14228_gb300 import ofks
    prm = ofks.default_params(p=3, precond="exact", eta_rule="fixed", eta_fixed=2.0)
    assert prm.p == 3 and prm.beta == 10.0 and prm.tol == 1e-8 and prm.precond == 2 and prm.eta_rule == 5
    assert prm.pcg_iters == 8 and prm.multipole_lmax == 2 and prm.hartree == 1 and prm.xc == 1
    assert prm.poisson_csr == 0 and prm.poisson_adaptive == 0 and prm.poisson_pc == 2


def test_updated_params_keep_the_other_fields(lib):
    # the binding's set_params applies keyword overrides on top of the parameters last set, so a
    # later change of one field (pcg_iters) keeps p, occ and the rest
    from paper_2007_14228_gb300 import ofks
    a = ofks.default_params(p=41, occ=2.0, precond="exact", beta=10.0)
    b = ofks.updated_params(a, pcg_iters=3, precision="mixed")
    assert (b.p, b.occ, b.precond, b.beta) == (41, 2.0, ofks.PC["exact"], 10.0)
    assert (b.pcg_iters, b.precision) == (3, ofks.PRECISION["mixed"])
    assert a.pcg_iters != 3 and a.precision == ofks.PRECISION["fp64"]


def test_missing_library_fails_loudly(tmp_path):
    from paper_2007_14228_gb300 import ofks
    saved = ofks._lib
    try:
        ofks._lib = None
        with pytest.raises(ofks.OfksError):
            ofks.load(str(tmp_path / "libofks.so"))
    finally:
        ofks._lib = saved


def _struct_fields(name):
    """(field, C type) of a typedef'd struct of include/ofks.h, in declaration order."""
    text = open(os.path.join(ROOT, "include", "ofks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for nm in names.split(","):
            out.append((nm.strip(), ctype))
    return out


@pytest.mark.parametrize("cname,pyname", [("ofks_params", "Params"), ("ofks_result", "Result")])
def test_python_structs_mirror_the_header(cname, pyname):
    # the ctypes structures must list the header's fields in the same order with the same types,
    # or every field after a mismatch is read at the wrong offset
    import ctypes as C

    from paper_2007_14228_gb300 import ofks
    ctype_of = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "uint64_t": C.c_uint64}
    header = _struct_fields(cname)
    py = getattr(ofks, pyname)._fields_
    assert [h[0] for h in header] == [f[0] for f in py]
    for (nm, ct), (_, pt) in zip(header, py):
        assert ctype_of[ct] is pt, (nm, ct, pt)
    assert C.sizeof(getattr(ofks, pyname)) % 8 == 0
