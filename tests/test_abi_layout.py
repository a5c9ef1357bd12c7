"""The Python binding mirrors the C structs of include/fsmlmc.h by hand: every field's offset and
every struct's size, as a C compiler lays them out, must match the ctypes classes. A small C
program built from the header prints them (gcc; no GPU)."""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2212_04430_gb300 import fsmlmc as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [("fs_solve_params", fb.SolveParams), ("fs_sys_stats", fb.SysStats), ("fs_mlmc_params", fb.MlmcParams),
           ("fs_job", fb.Job), ("fs_job_result", fb.JobResult), ("fs_server_report", fb.ServerReport)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fsmlmc.h"', 'int main(void) {']
    for cname, cls in STRUCTS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ['  return 0;', '}']
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.parametrize("cname,cls", STRUCTS, ids=[s[0] for s in STRUCTS])
def test_struct_layout_matches_the_header(c_layout, cname, cls):
    assert c_layout[(cname, "sizeof")] == ctypes.sizeof(cls), cname
    for field, _ in cls._fields_:
        assert c_layout[(cname, field)] == getattr(cls, field).offset, (cname, field)
