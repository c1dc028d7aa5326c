"""The Python binding's ctypes structures match the C header field by field: a small C program
compiled against include/hca_dbscan.h prints the size and every field offset of hca_stats,
hca_tuning and hca_request, and the test compares them with the ctypes layouts.  Needs gcc,
no GPU and no built library."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(tmp_path, c_name, fields):
    src = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hca_dbscan.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({c_name}));']
    lines += [f'  printf("%zu\\n", offsetof({c_name}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("py_name,c_name", [("HcaStats", "hca_stats"), ("HcaTuning", "hca_tuning"),
                                            ("HcaRequest", "hca_request")])
def test_ctypes_layout_matches_header(tmp_path, py_name, c_name):
    import paper_1912_00323_gb300 as pkg  # the structures only; the library is not loaded
    cls = getattr(pkg, py_name)
    fields = [f for f, _ in cls._fields_]
    size, offsets = _c_layout(tmp_path, c_name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets
