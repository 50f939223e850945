"""The C-ABI library loads on a machine without a GPU and exports every
function include/mg.h declares; the Python binding covers each of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char|long long)\s*\*?\s*(mg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g

    g.build()
    from paper_2605_30082_gb300 import _lib

    return _lib.LIB_PATH


def test_header_parses():
    names = header_functions()
    assert {"mg_create", "mg_set_density", "mg_solve", "mg_adjoint", "mg_destroy"} <= set(names)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    from paper_2605_30082_gb300 import _lib

    assert set(header_functions()) == set(_lib.SIGNATURES)
    _lib.lib()  # loads and sets every signature without a GPU


def test_host_side_argument_checks(libpath):
    """Option validation runs on the host: bad options fail before any device call."""
    from paper_2605_30082_gb300 import _lib

    L = _lib.lib()
    o = _lib.mg_default_opts()
    assert o.pre == 2 and o.post == 2 and o.coarsest == 4 and o.rtol == 1e-10
    h = ctypes.c_void_p()
    for field, bad in [("nx", 0), ("h", -1.0), ("precision", 7), ("coarsest", 1), ("prolong", 3),
                       ("max_cycles", -1), ("pre", -1)]:
        oo = _lib.mg_default_opts()
        setattr(oo, field, bad)
        assert L.mg_create(ctypes.byref(oo), None, ctypes.byref(h)) == _lib.MG_ERR_ARG
        assert not h.value
    # a grid whose coarsest level exceeds the dense-solve limit
    oo = _lib.mg_default_opts()
    oo.nx, oo.ny, oo.nz = 33, 33, 33
    assert L.mg_create(ctypes.byref(oo), None, ctypes.byref(h)) == _lib.MG_ERR_ARG
    assert L.mg_create(None, None, ctypes.byref(h)) == _lib.MG_ERR_ARG
    assert L.mg_destroy(None) == _lib.MG_OK
    assert L.mg_solve(None, None, None, None) == _lib.MG_ERR_ARG


def test_product_does_not_import_oracle():
    """The CUDA path's package never names the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_30082_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mg_oracle" not in txt and "liboracle" not in txt, f


def _header_struct_fields(text, name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", text)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)  # array extents
        parts = decl.split(None, 1)[1]          # drop the type
        names += [p.strip().lstrip("*") for p in parts.split(",")]
    return names


@pytest.mark.parametrize("name", ["mg_opts", "mg_stats"])
def test_ctypes_structs_mirror_the_header(name):
    from paper_2605_30082_gb300 import _lib

    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    assert _header_struct_fields(text, name) == [f[0] for f in getattr(_lib, name)._fields_]
