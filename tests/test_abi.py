"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point declared in include/bt.h; the binding has no path
to the oracle."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b((?:bt|abd|ivp|cyc)_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0912_3678_gb300 import build
    build.build()
    from paper_0912_3678_gb300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("bt_plan_create", "bt_factor", "bt_solve", "bt_refine", "bt_residual", "bt_plan_destroy",
                 "abd_plan_create", "abd_factor", "abd_solve", "abd_refine", "ivp_parareal"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header(lib):
    from paper_0912_3678_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_status_strings(lib):
    import paper_0912_3678_gb300 as bt
    assert bt.bt_status_string(0) == "ok"
    assert "singular" in bt.bt_status_string(3)


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_0912_3678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", f
            if f.endswith((".cu", ".cuh", ".h")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read().lower(), f


def test_missing_library_fails_loudly(tmp_path):
    from paper_0912_3678_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def _header_struct(name):
    """Field (C type, name) pairs of `typedef struct { ... } name;` in include/bt.h."""
    text = open(os.path.join(ROOT, "include", "bt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    return [tuple(f.rsplit(None, 1)) for f in (x.strip() for x in body.split(";")) if f]


@pytest.mark.parametrize("cname,pyname", [("bt_tuning", "BtTuning"), ("bt_batch_desc", "BtBatchDesc")])
def test_binding_structs_match_header(cname, pyname):
    """The ctypes mirrors of the ABI's structs have the header's fields, in its
    order, with the same C types."""
    import ctypes

    from paper_0912_3678_gb300 import _lib
    ctype = {"int64_t": ctypes.c_int64, "int": ctypes.c_int, "double": ctypes.c_double,
             "bt_tuning": _lib.BtTuning}
    fields = _header_struct(cname)
    py = getattr(_lib, pyname)._fields_
    assert [f[1].lstrip("*") for f in fields] == [p[0] for p in py]
    for (ct, nm), (pn, pt) in zip(fields, py):
        if nm.startswith("*") or ct.endswith("*"):
            assert pt is ctypes.c_void_p, nm
        else:
            assert pt is ctype[ct], nm
