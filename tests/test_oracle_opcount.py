"""The counted evaluation behind the algorithmic operation counts.

oracle/opcount.cpp evaluates the same lnL, gradient, distance marginal and
online lnZ as the oracle, with every floating-point operation counted; the
benchmark's roofline divides by those counts (oracle/flops.json).  Here the
counted evaluation is checked against the oracle to rounding, its counts
against hand counts of the plain formula's pieces, and the frozen file against
a fresh count.
"""
import math

import numpy as np
import pytest

import oracle as O
import workload as W
from test_oracle_pins import small_point


@pytest.fixture(scope="module")
def pts():
    p1, _, _, d1, w1 = W.config1(n_draws=512)
    p6, _, _, _ = small_point(modes=W.MODES10[:6], noise=True, snr=30.0, ndet=3)
    rng = np.random.default_rng(5)
    d6 = {p: np.asarray(v, dtype=np.float64) for p, v in W.Prior(50.0, 200.0, 0.01)
          .sample(rng, 256).items()}
    return [(p1, d1, w1), (p6, d6, np.zeros(256))]


def test_counted_values_equal_the_oracle(pts):
    for point, draws, logw in pts:
        pt = O.OraclePoint(point)
        ref, g = O.lnL_grad(pt, draws)
        r = O.op_counts(pt, draws, "grad")
        assert np.max(np.abs(r["values"] - ref) / np.maximum(1, np.abs(ref))) < 1e-12
        scale = np.abs(g) + np.sqrt(np.mean(g ** 2, axis=0))[None, :]
        assert np.max(np.abs(r["grad"] - g) / scale) < 1e-11
        # forward + online log-sum-exp against the oracle's two-pass lnZ
        z = O.op_counts(pt, draws, "lnZ", logw=logw)
        assert np.max(np.abs(z["values"] - ref) / np.maximum(1, np.abs(ref))) < 1e-12
        m, s, s2 = z["lse"]
        rz = O.lnZ(ref, logw)
        n = len(ref)
        assert abs(m + math.log(s) - math.log(n) - rz[0]) < 1e-12 * max(1, abs(rz[0]))
        assert abs(s - rz[2]) < 1e-10 * s
        # distance marginal and its gradient
        x, lnw = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, 60.0)
        dm, dg = O.lnL_distmarg(pt, draws, x, lnw, grad=True)
        c = O.op_counts(pt, draws, "dist_grad", x_nodes=x, lnw_nodes=lnw)
        fin = np.isfinite(dm)
        assert np.max(np.abs(c["values"][fin] - dm[fin]) / np.maximum(1, np.abs(dm[fin]))) < 1e-12
        dscale = np.abs(dg) + np.sqrt(np.mean(dg[fin] ** 2, axis=0))[None, :] + 1e-300
        assert np.max((np.abs(c["grad"] - dg) / dscale)[fin]) < 1e-10


def test_counts_are_per_draw_constants(pts):
    """lnL and its gradient take the same operations at every draw."""
    point, draws, _ = pts[0]
    pt = O.OraclePoint(point)
    a = O.op_counts(pt, {p: v[:7] for p, v in draws.items()}, "grad")
    b = O.op_counts(pt, {p: v[100:113] for p, v in draws.items()}, "grad")
    assert a["flops"] * 13 == b["flops"] * 7
    assert a["special"] * 13 == b["special"] * 7


def test_counts_against_hand_counts_of_the_formula():
    """The quadratic term's share: with M modes and K detectors the P/S
    products take 9M + 12 M(M-1)/2 flops once per draw and each detector
    10M + 12 M(M-1)/2 + 12 for its U and V forms; adding one
    detector class changes the count by exactly the per-detector work, and
    the M-dependence is quadratic with these coefficients."""
    counts = {}
    for K in (2, 3):
        for M in (2, 4, 6):
            point, _, _, pt = small_point(modes=W.MODES10[:M], ndet=K)
            th = np.array([[0.3, 0.2, 0.1, 0.7, 0.4, math.log(100.0), 0.0]])
            counts[K, M] = O.op_counts(pt, th, "grad")["flops"], O.op_counts(
                pt, th, "lnZ", logw=np.zeros(1))["flops"]
    # per-detector forward work is linear in M plus the quadratic forms
    for M in (2, 4, 6):
        per_det = counts[3, M][1] - counts[2, M][1]
        quad = 2 * M + 4 * M * (M - 1) // 2 + 8 * M + 8 * M * (M - 1) // 2 + 12
        tap = 6 + 10 + 14 * M   # position and offsets, weights, taps
        data = 8 * M - 2 + 3 + 1
        geom = 15 + 15 + 5 * 3 + 2 + 6
        assert per_det == quad + tap + data + geom, (M, per_det)


def test_frozen_counts_are_current():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(O.__file__), "freeze_flops.py")
    spec = importlib.util.spec_from_file_location("freeze_flops", path)
    F = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(F)
    import json
    fresh = json.loads(json.dumps(F.compute(), sort_keys=True))
    frozen = json.load(open(F.OUT))
    assert fresh == frozen
