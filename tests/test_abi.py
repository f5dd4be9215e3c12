"""The C-ABI library builds, loads and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1901_07294_gb300 as wd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:int|const\s+char\s*\*|void|double|size_t)\s*\**\s*(\w+)\s*\(", txt, flags=re.M)
    return names


def test_library_loads_and_exports_all_declared_symbols():
    lib = wd.load()
    declared = _declared_functions()
    assert "dslash_apply" in declared and "dslash_eo_apply" in declared
    for name in declared:
        assert hasattr(lib, name), name
    # the binding covers exactly what the header declares
    assert set(wd.exported_symbols()) == set(declared)


def test_version_and_field_sizes():
    assert wd.load().wd_version() >= 100
    V = 8 ** 4
    assert wd.field_bytes((8, 8, 8, 8), wd.SITES_FULL, wd.F32) == V * 24 * 4
    assert wd.field_bytes((8, 8, 8, 8), wd.SITES_EVEN, wd.F64) == V // 2 * 24 * 8
    assert wd.field_bytes((8, 8, 8, 8), wd.SITES_ODD, wd.F16, nrhs=3) == 3 * (V // 2) * (48 + 4)
    assert wd.field_bytes((4, 6, 8, 10), wd.SITES_FULL, wd.BF16) == 4 * 6 * 8 * 10 * 52


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 1), (4, 4, 4, -2)])
def test_bad_dims_rejected(dims):
    with pytest.raises(wd.WdError) as e:
        wd.field_bytes(dims, wd.SITES_FULL, wd.F32)
    assert e.value.status == wd.WD_EINVAL


def test_bad_precision_and_nrhs_rejected():
    for prec, nrhs in ((7, 1), (-1, 1), (wd.F32, 0)):
        with pytest.raises(wd.WdError) as e:
            wd.field_bytes((4, 4, 4, 4), wd.SITES_FULL, prec, nrhs)
        assert e.value.status == wd.WD_EINVAL


_MIRRORS = [("wd_tune_entry", "TuneEntry"), ("wd_cg_opts", "CgOpts"), ("wd_cg_stats", "CgStats"),
            ("wd_solve_desc", "SolveDesc"), ("wd_solve_result", "SolveResult"), ("rq_counters", "RqCounters"),
            ("wd_device_props", "DeviceProps")]


def test_struct_mirrors_match_the_header(tmp_path):
    """Every ctypes mirror of a C-ABI struct has the header's size and field offsets (a C
    program compiled against include/wdirac.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "wdirac.h"', "int main(void) {"]
    for cname, pyname in _MIRRORS:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in getattr(wd, pyname)._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(p[0], p[1]): int(p[2]) for p in (l.split() for l in out) if len(p) == 3}
    for cname, pyname in _MIRRORS:
        cls = getattr(wd, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_double_word_field_sizes():
    """A double-word field holds each real as two FP32 numbers: the FP64 byte count."""
    for sites in (wd.SITES_FULL, wd.SITES_EVEN):
        assert wd.field_bytes((4, 6, 8, 10), sites, wd.DF) == wd.field_bytes((4, 6, 8, 10), sites, wd.F64)
