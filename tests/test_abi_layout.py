"""The binding's ctypes structures against the C header: a small C program compiled against
include/hbgls.h prints the size of every struct and the offset of every field the binding declares, and
both must agree with ctypes (same names, same offsets, same sizes), so the two cannot drift apart."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2411_14315_gb300 import hbgls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [hbgls.hb_mesh, hbgls.hb_solve_opts, hbgls.hb_report, hbgls.hb_march_opts, hbgls.hb_march_report,
           hbgls.hb_info, hbgls.hb_mpnn_config]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hbgls.h"', "int main(void) {"]
    for s in STRUCTS:
        name = s.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in s._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(line.split()[:2]): int(line.split()[2]) for line in out.splitlines()}


@pytest.mark.parametrize("s", STRUCTS, ids=lambda s: s.__name__)
def test_ctypes_struct_matches_the_header(c_layout, s):
    name = s.__name__
    assert c_layout[(name, "size")] == C.sizeof(s), name
    for f, _ in s._fields_:
        assert c_layout[(name, f)] == getattr(s, f).offset, (name, f)
