"""The binding's ctypes structures against the C header's layout: gcc
compiles a probe that prints sizeof and every field's offsetof for each
typedef, and the ctypes class must agree field by field (a field added to a
header but not to the binding, or in another order, fails here)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    ("_PointDesc", "rift_ile_point_desc", "rift_ile.h"),
    ("_Draws", "rift_ile_draws", "rift_ile.h"),
    ("_Lse", "rift_ile_lse", "rift_ile.h"),
    ("_Dist", "rift_ile_dist", "rift_ile.h"),
    ("_CompDesc", "rift_ile_comp_desc", "rift_ile_response.h"),
    ("_PrecompDesc", "rift_ile_precompute_desc", "rift_ile_precompute.h"),
    ("_DirectRule", "rift_ile_direct_rule", "rift_ile_direct.h"),
]


@pytest.fixture(scope="module")
def layouts():
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    R = pytest.importorskip("paper_2609_37393_b300")
    lines = ["#include <stdio.h>", "#include <stddef.h>"]
    lines += [f'#include "{h}"' for h in sorted({p[2] for p in PAIRS})]
    lines.append("int main(void) {")
    for cls, ctype, _ in PAIRS:
        fields = [f[0] for f in getattr(R, cls)._fields_]
        lines.append(f'  printf("{cls} size %zu\\n", sizeof({ctype}));')
        for f in fields:
            lines.append(f'  printf("{cls} {f} %zu\\n", offsetof({ctype}, {f}));')
    lines.append("  return 0;\n}")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
    with open(src, "w") as fh:
        fh.write("\n".join(lines))
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cls, key, val = line.split()
        got[(cls, key)] = int(val)
    return R, got


@pytest.mark.parametrize("cls", [p[0] for p in PAIRS])
def test_ctypes_struct_matches_header(layouts, cls):
    R, got = layouts
    C = getattr(R, cls)
    assert got[(cls, "size")] == __import__("ctypes").sizeof(C)
    for name, _ in C._fields_:
        assert got[(cls, name)] == getattr(C, name).offset, name
