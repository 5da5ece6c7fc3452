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
