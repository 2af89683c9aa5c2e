"""CPU checks of the native library: it builds for sm_103a, loads, and
exports every entry point declared in include/cde.h (no GPU call)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cde_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_all_symbols():
    from __graft_entry__ import build
    build()
    from paper_1206_5278_gb300 import cde
    L = cde.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(cde.EXPORTED)
    assert "sm_103a" in cde.cde_version()


def test_last_error_is_empty_string_initially():
    from paper_1206_5278_gb300 import cde
    assert isinstance(cde.last_error(), str)
