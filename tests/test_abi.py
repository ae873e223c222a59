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


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof and field offsets of the option, statistics and distortion structs
    as a C compiler lays them out from include/pgcp.h, against the ctypes
    binding (a stale binding would pass garbage through the ABI)."""
    import shutil
    import subprocess
    from paper_1903_12359_gb300 import api
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pgcp_options": api.Options, "pgcp_stats": api.Stats, "pgcp_distortion": api.Distortion,
               "pgcp_mesh_desc": api.MeshDesc, "pgcp_area_result": api.AreaResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pgcp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for ln in filter(None, got):
        cname, what, val = ln.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if what == "size" else getattr(py, what).offset
        assert int(val) == want, (cname, what, int(val), want)
    o = api.default_options()
    assert o.deterministic == 0 and o.local_precision == api.DF64_REFINED


def test_coordinate_tensors_are_checked_before_any_launch():
    """metrics, area and no-alloc entry points read U as float64 [nv][dim]: the
    binding refuses another dtype, shape or a host tensor before it calls the
    library (no GPU is touched here)."""
    import torch
    from paper_1903_12359_gb300 import api
    nv = 10
    for closed, dim in ((False, 2), (True, 3)):
        with pytest.raises(ValueError, match="float64"):
            api.check_coords(torch.zeros((nv, dim), dtype=torch.float32), nv, closed)
        with pytest.raises(ValueError, match="shape"):
            api.check_coords(torch.zeros((nv, 5 - dim), dtype=torch.float64), nv, closed)
        with pytest.raises(ValueError, match="shape"):
            api.check_coords(torch.zeros((nv + 1, dim), dtype=torch.float64), nv, closed)
        with pytest.raises(ValueError, match="shape"):
            api.check_coords(torch.zeros(nv * dim, dtype=torch.float64), nv, closed)
        with pytest.raises(ValueError, match="CUDA"):
            api.check_coords(torch.zeros((nv, dim), dtype=torch.float64), nv, closed)
    with pytest.raises(ValueError, match="tensor"):
        api.check_coords([[0.0, 0.0]] * nv, nv, False)
