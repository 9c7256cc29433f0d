"""The Python binding's ctypes structures have the C ABI's layout: a small C
program compiled against include/dg.h prints the size and field offsets of
dg_mesh_desc and dg_mesh_info_t, which must equal the ctypes mirrors in dg.py
(a field added to the header and not to the binding would shift every later
field silently)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1601_07944_gb300 import dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DESC_FIELDS = ["n_elem", "elem_xy", "nbr", "nbr_face", "p", "n_edge_pts", "gamma", "vol_rule"]
INFO_FIELDS = ["n_elem", "n_face", "p", "n_modes", "n_vol_pts", "n_edge_pts", "gamma", "n_boundary_face"]


def _c_layout(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dg.h"', "int main(void) {"]
    lines.append('  printf("desc %zu\\n", sizeof(dg_mesh_desc));')
    for f in DESC_FIELDS:
        lines.append('  printf("desc.%s %%zu\\n", offsetof(dg_mesh_desc, %s));' % (f, f))
    lines.append('  printf("info %zu\\n", sizeof(dg_mesh_info_t));')
    for f in INFO_FIELDS:
        lines.append('  printf("info.%s %%zu\\n", offsetof(dg_mesh_info_t, %s));' % (f, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    return {k: int(v) for k, v in (line.split() for line in out if line.strip())}


def test_ctypes_mirrors_match_the_header(tmp_path):
    lay = _c_layout(tmp_path)
    assert lay["desc"] == ctypes.sizeof(dg._Desc)
    for f in DESC_FIELDS:
        assert lay["desc." + f] == getattr(dg._Desc, f).offset, f
    assert lay["info"] == ctypes.sizeof(dg._Info)
    for f in INFO_FIELDS:
        assert lay["info." + f] == getattr(dg._Info, f).offset, f
    assert [f for f, _ in dg._Desc._fields_] == DESC_FIELDS
    assert [f for f, _ in dg._Info._fields_] == INFO_FIELDS
