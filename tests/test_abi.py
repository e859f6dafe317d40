"""The C-ABI library builds, loads and exports every entry point include/sci.h declares
(no compute calls: these run without a GPU)."""
import os
import re

from paper_2501_18185_gb300 import build, sci

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:int|const char \*)\s*\**\s*(sci_\w+)\s*\(", src, flags=re.M))


def test_header_declares_the_boundary():
    names = _declared()
    assert names == set(sci.SIGNATURES), names ^ set(sci.SIGNATURES)


def test_library_exports_every_declared_symbol():
    build.build()
    L = sci.load()
    for name in _declared():
        assert hasattr(L, name), name


def test_missing_library_fails_loudly(tmp_path):
    import pytest

    with pytest.raises(RuntimeError):
        sci.load(str(tmp_path / "libsci.so"))
