"""The C-ABI library loads without a GPU and exports every symbol that
the headers in include/ declare; the product package fails loudly without it and
never touches the oracle."""
import ctypes
import os
import re
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h)
           for h in ("rift_ile.h", "rift_ile_response.h", "rift_ile_precompute.h",
                     "rift_ile_direct.h")]
PKG = os.path.join(ROOT, "paper_2609_37393_b300")


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rift_ile_\w+)\s*\(", text)))


def library():
    so = os.path.join(PKG, "_rift_ile.so")
    if not os.path.exists(so):
        subprocess.check_call([sys.executable, os.path.join(PKG, "build.py")])
    return ctypes.CDLL(so)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("rift_ile_lnL", "rift_ile_lnL_grad", "rift_ile_lnZ", "rift_ile_lnZ_batch",
              "rift_ile_point_create", "rift_ile_point_destroy", "rift_ile_lnZ_merge",
              "rift_ile_comp_create", "rift_ile_comp_lnL", "rift_ile_comp_lnZ_state",
              "rift_ile_precompute"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_merge_is_host_only_and_exact():
    lib = library()

    class Lse(ctypes.Structure):
        _fields_ = [("m", ctypes.c_double), ("s", ctypes.c_double), ("s2", ctypes.c_double),
                    ("n", ctypes.c_double)]

    arr = (Lse * 2)(Lse(0.0, 2.0, 2.0, 2.0), Lse(1.0, 1.0, 1.0, 1.0))
    out = (ctypes.c_double * 3)()
    lib.rift_ile_lnZ_merge.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p]
    assert lib.rift_ile_lnZ_merge(arr, 2, out, None) == 0
    import math
    assert abs(out[0] - math.log((2 + math.e) / 3)) < 1e-15


def test_package_fails_loudly_without_library(tmp_path):
    dst = tmp_path / "paper_2609_37393_b300"
    dst.mkdir()
    shutil.copy(os.path.join(PKG, "__init__.py"), dst / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import paper_2609_37393_b300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "ImportError" in r.stderr


def test_product_never_uses_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "rift_oracle" not in text, f


def test_gauss_hermite_rule_is_the_textbook_one():
    """The host-side Gauss-Hermite rule of the direct kernel equals numpy's
    (Golub-Welsch) to rounding for every supported size."""
    import numpy as np
    import numpy.polynomial.hermite as H
    lib = library()
    lib.rift_ile_gauss_hermite.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    for n in (1, 2, 5, 16, 40, 64):
        x = np.empty(n)
        w = np.empty(n)
        assert lib.rift_ile_gauss_hermite(n, x.ctypes.data, w.ctypes.data) == 0
        xr, wr = H.hermgauss(n)
        assert np.max(np.abs(x - xr)) <= 1e-12 * max(1.0, np.max(np.abs(xr)))
        assert np.max(np.abs(w - wr) / wr) <= 1e-9
    assert lib.rift_ile_gauss_hermite(65, x.ctypes.data, w.ctypes.data) != 0
