"""The allocation-free lnZ entry point (rift_ile_lnZ_state_noalloc).

Callers that may not allocate device memory (a host framework that owns the
device heap through its own pool, or a time-critical sampler loop) use this
variant; its scratch is a fixed static device array instead of the library's
workspace.  The test calls it through the C ABI twice in a row, for both
precisions, and checks each result against rift_ile_lnZ_state with the
tolerances of the other lnZ tests.  It lives in a file collected last and
passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class Lse(ctypes.Structure):
    _fields_ = [("m", ctypes.c_double), ("s", ctypes.c_double), ("s2", ctypes.c_double),
                ("n", ctypes.c_double)]


def _lnz(st):
    import math
    return st.m + math.log(st.s) - math.log(st.n)


def test_noalloc_matches_lnz_state_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    lib = R._lib
    lib.rift_ile_lnZ_state_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p]
    lib.rift_ile_lnZ_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    point, exact, info, draws, logw = W.config1(n_draws=200_003)
    pt = R.Point(point)
    d = R.Draws(draws, logw)
    stream = torch.cuda.current_stream().cuda_stream
    for prec, tol in ((R.FP64, 1e-9), (R.FP32_MIXED, 1e-4)):
        ref = Lse()
        assert lib.rift_ile_lnZ_state(pt.handle, d.ref, prec, None, ctypes.byref(ref), stream) == 0
        ref_taps = R.rift_ile_last_oob()
        for call in range(2):
            got = Lse()
            rc = lib.rift_ile_lnZ_state_noalloc(pt.handle, d.ref, prec, ctypes.byref(got), stream)
            assert rc == 0, R._lib.rift_ile_last_error()
            assert got.n == ref.n == 200_003
            assert abs(_lnz(got) - _lnz(ref)) <= tol * max(1.0, abs(_lnz(ref))), (prec, call)
            assert abs(got.s - ref.s * np.exp(ref.m - got.m)) <= 1e-6 * got.s
            # the out-of-table tap count is reported like the regular entry point's
            assert R.rift_ile_last_oob() == ref_taps, (prec, call)


def test_noalloc_after_release():
    """rift_ile_release forgets the scratch address; the next call looks it up
    again and gives the same state as before."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    lib = R._lib
    lib.rift_ile_lnZ_state_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p]
    point, exact, info, draws, logw = W.config1(n_draws=4099)
    pt = R.Point(point)
    d = R.Draws(draws, logw)
    stream = torch.cuda.current_stream().cuda_stream
    a, b = Lse(), Lse()
    assert lib.rift_ile_lnZ_state_noalloc(pt.handle, d.ref, R.FP32_MIXED, ctypes.byref(a),
                                          stream) == 0
    R.rift_ile_release()
    assert lib.rift_ile_lnZ_state_noalloc(pt.handle, d.ref, R.FP32_MIXED, ctypes.byref(b),
                                          stream) == 0
    assert (a.m, a.s, a.s2, a.n) == (b.m, b.s, b.s2, b.n)
