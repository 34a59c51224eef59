"""The ctypes mirrors of the C-ABI structs (cpcp_options, cpcp_info,
cpcp_problem) match include/cpcp.h field by field: the same fields in the same
order at the same offsets, and the same size.  The offsets come from a small C
program compiled against the header with gcc (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cpcp.h")


def c_fields(struct_name):
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct_name + r"\s*;", src)
    assert m, struct_name
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(",")
        first = re.sub(r"\[.*?\]", "", parts[0]).replace("*", " ").split()
        names.append(first[-1])
        for p in parts[1:]:
            names.append(re.sub(r"\[.*?\]", "", p).replace("*", " ").split()[-1])
    return names


@pytest.fixture(scope="module")
def cpcp_mod():
    # the binding's struct definitions only (the module itself needs the built library)
    src = open(os.path.join(ROOT, "paper_2206_13369_gb300", "cpcp.py")).read()
    ns = {}
    code = src[src.index("class Options"):src.index("_vp, _i64, _int, _dbl")]
    code2 = src[src.index("class Problem"):src.index("def _load")]
    exec("import ctypes as C\n" + code + "\n_vp, _i64, _int, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double\n" + code2,
         ns)
    return ns


@pytest.mark.parametrize("struct_name,cls", [("cpcp_options", "Options"), ("cpcp_info", "Info"),
                                             ("cpcp_problem", "Problem")])
def test_struct_layout_matches_header(tmp_path, cpcp_mod, struct_name, cls):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    names = c_fields(struct_name)
    py = cpcp_mod[cls]
    py_names = [f[0] for f in py._fields_]
    assert len(names) == len(py_names), (names, py_names)
    prog = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {",
            f'  printf("%zu\\n", sizeof({struct_name}));']
    for n in names:
        prog.append(f'  printf("%zu\\n", offsetof({struct_name}, {n}));')
    prog.append("  return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(c), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(py), (struct_name, out[0], ctypes.sizeof(py))
    for cname, pname, off in zip(names, py_names, out[1:]):
        assert getattr(py, pname).offset == off, (struct_name, cname, pname, off, getattr(py, pname).offset)
