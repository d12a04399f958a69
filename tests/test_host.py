"""Host-side parts of the library (no GPU needed)."""
import ctypes
import math

import numpy as np

import oracle as O
from tests.test_abi import library


def test_dist_nodes_match_oracle_rule():
    """The library's node table and the oracle's, written independently from
    eq. ap:dlog, agree node by node."""
    lib = library()
    lib.rift_ile_dist_nodes.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int32] + [ctypes.c_void_p] * 3
    for (dmin, dmax, tol, rho) in ((50.0, 200.0, 1e-4, 1000.0), (10.0, 1000.0, 1e-6, 300.0)):
        x = np.empty(1 << 16)
        w = np.empty(1 << 16)
        n = ctypes.c_int32()
        assert lib.rift_ile_dist_nodes(dmin, dmax, 100.0, tol, rho, 1 << 16, x.ctypes.data,
                                       w.ctypes.data, ctypes.byref(n)) == 0
        rx, rw = O.dist_nodes(dmin, dmax, 100.0, tol, rho)
        assert n.value == len(rx)
        assert np.allclose(x[:n.value], rx, rtol=1e-14, atol=0)
        assert np.allclose(w[:n.value], rw, rtol=0, atol=1e-12)


def test_dist_nodes_rejects_oversized_table():
    lib = library()
    lib.rift_ile_dist_nodes.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int32] + [ctypes.c_void_p] * 3
    x = np.empty(8)
    n = ctypes.c_int32()
    assert lib.rift_ile_dist_nodes(1.0, 1000.0, 1.0, 1e-4, 1000.0, 8, x.ctypes.data, x.ctypes.data,
                                   ctypes.byref(n)) == -2
