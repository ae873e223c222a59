"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pgcp.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pgcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgcp_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_declared_symbols():
    from paper_1903_12359_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1903_12359_gb300 import api
    assert set(_declared()) <= set(api.SIGNATURES)
    o = api.default_options()
    assert o.variant == api.DISK and o.precision == api.FP32_REFINED and o.tol == 1e-10


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1903_12359_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
