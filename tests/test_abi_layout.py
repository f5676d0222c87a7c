"""The Python binding's ctypes mirrors of the C structs (mhc_plan_opts, mhc_stats) have the
same size and field offsets as the structs of include/mhc.h: a small C program compiled
against the header prints them (host compiler only; no GPU, no library)."""
import os
import shutil
import subprocess

import pytest

from paper_1411_3691_gb300 import mhc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(tmp_path, cname, fields):
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mhc.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({cname}));']
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([shutil.which("gcc") or "gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
@pytest.mark.parametrize("cname, pytype", [("mhc_plan_opts", mhc.PlanOpts), ("mhc_stats", mhc.Stats)])
def test_struct_layout_matches_header(tmp_path, cname, pytype):
    fields = [name for name, _ in pytype._fields_]
    got = _c_layout(tmp_path, cname, fields)
    assert got["size"] == _sizeof(pytype), (cname, got["size"], _sizeof(pytype))
    for name in fields:
        assert got[name] == getattr(pytype, name).offset, (cname, name, got[name], getattr(pytype, name).offset)


def _sizeof(t):
    import ctypes
    return ctypes.sizeof(t)
