"""The C ABI library builds, loads without a GPU and exports every entry
point include/rbsog.h declares; the Python binding names the same set.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "rbsog.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rbsog_[a-z_]+)\s*\(", txt)))


def test_header_declares_expected_calls():
    names = declared()
    for must in ("rbsog_create", "rbsog_set_params", "rbsog_compute_forces", "rbsog_step",
                 "rbsog_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2205_13824_gb300.binding as B
    lib = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(B.EXPORTS) == declared()


def test_python_binding_has_same_names():
    import paper_2205_13824_gb300.binding as B
    for n in declared():
        assert callable(getattr(B, n)), n


def test_struct_layouts_match_header():
    """ctypes mirrors of the by-value structs list the header's fields in order."""
    import paper_2205_13824_gb300.binding as B
    txt = open(os.path.join(ROOT, "include", "rbsog.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for cname, py in (("rbsog_params", B.rbsog_params), ("rbsog_energies", B.rbsog_energies),
                      ("rbsog_info", B.rbsog_info)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", txt).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = decl.split(None, 1)[1]
            for n in names.split(","):
                fields.append(re.sub(r"\[.*\]", "", n).strip())
        assert [f[0] for f in py._fields_] == fields, cname


def test_product_fails_loudly_without_library(tmp_path, monkeypatch):
    """With the shared library absent the binding refuses to import (no
    silent CPU path)."""
    import importlib.util
    import paper_2205_13824_gb300.binding as B
    spec = importlib.util.spec_from_file_location("binding_copy", B.__file__)
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False if p.endswith("librbsog.so") else True)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
