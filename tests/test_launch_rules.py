"""Source rules of the launch path (no GPU needed).

wd_launch launches with programmatic dependent launch: a kernel may be dispatched while
the kernel before it in its stream or graph is still running.  That is safe only if the
kernel's first statement is grid_dependency_enter(), which waits for the predecessor to
complete with its writes visible before any memory access.  These tests read the CUDA
sources and check that every kernel handed to wd_launch starts that way.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1901_07294_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            txt = open(os.path.join(CSRC, f)).read()
            out[f] = re.sub(r"//[^\n]*", "", txt)
    return out


def _launched_kernels(src):
    names = set()
    for f, txt in src.items():
        if f != "launch.cuh":   # where wd_launch itself is defined
            names.update(re.findall(r"\bwd_launch\(\s*([A-Za-z_]\w*)", txt))
    return names


def _first_statements(src, name):
    """First statement of each __global__ definition of `name`."""
    firsts = []
    pat = re.compile(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(")
    for txt in src.values():
        for m in pat.finditer(txt):
            # skip the parameter list (balanced parentheses) to the body's brace
            i, depth = m.end(), 1
            while depth:
                depth += {"(": 1, ")": -1}.get(txt[i], 0)
                i += 1
            body = txt[txt.index("{", i) + 1:]
            firsts.append(body.lstrip().split(";", 1)[0].strip())
    return firsts


def test_every_launched_kernel_waits_for_its_predecessor_first():
    src = _sources()
    names = _launched_kernels(src)
    # the operator, BLAS, solver-loop, pack and face kernels all go through wd_launch
    for must in ("hop_kernel", "blas_kernel", "hop_sp_kernel", "hop_df_row_kernel", "hop_mrhs_kernel",
                 "hop_group_kernel", "gs_control_kernel", "gg_control_kernel", "pack_lex_kernel",
                 "dd_gather_kernel"):
        assert must in names, must
    for name in sorted(names):
        firsts = _first_statements(src, name)
        assert firsts, f"no __global__ definition found for {name}"
        for f in firsts:
            assert f == "grid_dependency_enter()", f"{name} starts with {f!r}"


def test_grid_dependency_enter_waits_before_it_triggers():
    txt = _sources()["wd_device.cuh"]
    body = txt[txt.index("void grid_dependency_enter()"):]
    body = body[:body.index("}")]
    assert body.index("griddepcontrol.wait") < body.index("griddepcontrol.launch_dependents")
