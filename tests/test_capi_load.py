"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/swig.h declares (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "swig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(swig_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_28265_gb300 import build, swig
    if not os.path.exists(swig.LIB_PATH):
        build.build()
    return swig.load_library()


def test_library_exports_every_declared_symbol(lib):
    from paper_2607_28265_gb300 import swig
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared entry points
    assert set(swig.SIGNATURES) == set(names)


def test_no_cpu_fallback_in_binding():
    src = open(os.path.join(ROOT, "paper_2607_28265_gb300", "swig.py")).read()
    assert "oracle" not in src


def _c_kind(decl):
    """Category of one C parameter or return type from include/swig.h."""
    d = " ".join(decl.replace("const ", "").split())
    is_ptr = "*" in d or "[" in d
    base = d.split("*")[0].split("[")[0].strip().split(" ")[0]
    if is_ptr:
        return {"double": "dptr", "float": "fptr", "int": "iptr", "int64_t": "i64ptr"}.get(base, "ptr")
    return {"int": "int", "int64_t": "i64", "long": "i64", "uint64_t": "u64", "double": "double",
            "void": "void"}[base]


def _py_kind(t):
    import ctypes
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p):
        return "any_ptr"
    if isinstance(t, type) and issubclass(t, ctypes._Pointer):
        target = t._type_
        return {ctypes.c_double: "dptr", ctypes.c_float: "fptr", ctypes.c_int: "iptr",
                ctypes.c_int64: "i64ptr"}.get(target, "ptr")
    return {ctypes.c_int: "int", ctypes.c_int64: "i64", ctypes.c_longlong: "i64", ctypes.c_uint64: "u64",
            ctypes.c_double: "double"}[t]


def test_binding_signatures_match_the_header():
    """Every prototype's return and argument types against the ctypes
    signature the binding declares (c_void_p may stand for any pointer:
    device buffers and streams travel as void*)."""
    from paper_2607_28265_gb300 import swig
    src = open(os.path.join(ROOT, "include", "swig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = re.findall(r"(int|void|const char\s*\*)\s*(swig_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src)
    assert len(protos) == len(swig.SIGNATURES)
    for ret, name, args in protos:
        pret, pargs = swig.SIGNATURES[name]
        want_ret = "ptr" if "*" in ret else _c_kind(ret)
        got_ret = _py_kind(pret)
        assert got_ret == want_ret or (got_ret == "any_ptr" and want_ret == "ptr"), name
        cargs = [a for a in (x.strip() for x in args.split(",")) if a]
        kinds = [_c_kind(a.rsplit(" ", 1)[0] + (" *" if a.rsplit(" ", 1)[1].startswith("*") else "")
                         + ("[]" if "[" in a else "")) for a in cargs]
        assert len(kinds) == len(pargs), name
        for i, (ck, pt) in enumerate(zip(kinds, pargs)):
            pk = _py_kind(pt)
            ok = pk == ck or (pk == "any_ptr" and ck.endswith("ptr"))
            assert ok, (name, i, ck, pk)
