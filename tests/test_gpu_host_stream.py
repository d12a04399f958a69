"""lnZ from draws in host memory (rift_ile_lnZ_state_host): the chunked,
double-buffered copy + kernel pipeline gives the same LSE state as the
resident path on the same draws (to rounding: the block partials group the
draws differently), for page-locked and pageable host arrays, any chunk size
(including a ragged last chunk), both precisions and the distance
marginalisation; zero draws give the empty state."""
import math

import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


@pytest.fixture(scope="module")
def cfg():
    return W.config1(n_draws=(1 << 18) + 12345)


def close(a, b, prec=0):
    """Same state up to the grouping of the sums: FP64 partials agree to
    ~1e-15, the FP32-mixed per-thread sums of e^(v - m) to ~1e-7 relative."""
    tol = 1e-12 if prec == 0 else 1e-6
    lz_a, lz_b = a[0] + math.log(a[1]), b[0] + math.log(b[1])
    return abs(lz_a - lz_b) <= tol and a[3] == b[3] and \
        abs(a[2] / a[1] ** 2 - b[2] / b[1] ** 2) <= tol * (b[2] / b[1] ** 2)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("chunk", [0, 1 << 16, 100_003])
def test_host_stream_matches_resident(R, cfg, prec, chunk):
    point, exact, info, draws, logw = cfg
    pt = R.Point(point)
    ref = R.rift_ile_lnZ_state(pt, R.Draws(draws, logw), prec)
    pinned = {p: torch.from_numpy(np.ascontiguousarray(draws[p])).pin_memory() for p in W.PARAMS}
    hd = R.HostDraws(pinned, torch.from_numpy(np.ascontiguousarray(logw)).pin_memory())
    got = R.rift_ile_lnZ_state_host(pt, hd, prec, chunk=chunk)
    assert close(got, ref, prec), (got, ref)
    again = R.rift_ile_lnZ_state_host(pt, hd, prec, chunk=chunk)
    assert again == got  # deterministic


def test_host_stream_pageable_and_dist(R, cfg):
    point, exact, info, draws, logw = cfg
    pt = R.Point(point)
    nodes = R.rift_ile_dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)
    ref = R.rift_ile_lnZ_state(pt, R.Draws(draws, logw), R.FP32_MIXED, dist=nodes)
    got = R.rift_ile_lnZ_state_host(pt, R.HostDraws(draws, logw), R.FP32_MIXED, dist=nodes,
                                    chunk=50_000)
    assert close(got, ref, 1), (got, ref)


def test_host_stream_empty(R, cfg):
    point = cfg[0]
    pt = R.Point(point)
    empty = {p: np.zeros(0, dtype=np.float32) for p in W.PARAMS}
    st = R.rift_ile_lnZ_state_host(pt, R.HostDraws(empty), R.FP32_MIXED)
    assert st[0] == -math.inf and st[3] == 0.0


def test_host_draws_rejects_device_arrays(R, cfg):
    point, exact, info, draws, logw = cfg
    dev = {p: torch.as_tensor(np.asarray(draws[p][:8]), device="cuda") for p in W.PARAMS}
    with pytest.raises(ValueError):
        R.HostDraws(dev)
