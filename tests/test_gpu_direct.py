"""Direct marginalisation inside the likelihood (ERAI over phase and
polarisation, adaptive Gauss-Hermite in distance) on the GPU against the
oracle's reconstruction-then-quadrature, on the two-detector workload (SNR 20
with noise, complex128 table) and on the 3G network at SNR 30 (complex64
table): every draw within 1e-9 relative, -inf where no distance node lies in
the prior; the node skipping changes nothing above rounding; invalid rules
are refused.
"""
import math

import numpy as np
import pytest

import oracle.direct as OD
import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


def _cmp(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.all(got[~fin] == ref[~fin])
    assert np.max(np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))) <= 1e-9


def test_two_detector_workload(R):
    point, exact, info, draws, logw = W.config0(n_draws=40)
    d = {p: np.concatenate([[info["truth"][p]], np.asarray(draws[p])]) for p in W.PARAMS}
    pt = R.Point(point)
    got = R.rift_ile_lnL_direct(pt, R.Draws(d), 96, 48, 16, 50.0, 200.0).cpu().numpy()
    ref = OD.lnL_direct(point, d, 96, 48, 16, 50.0, 200.0)
    _cmp(got, ref)
    assert np.isfinite(got[0])


def test_3g_network_moderate_snr(R):
    point, exact, info, draws, logw = W.config_3g(1, 4, 30.0, 0.02, 24)
    pt = R.Point(point)
    got = R.rift_ile_lnL_direct(pt, R.Draws(draws), 128, 64, 16, 50.0, 200.0).cpu().numpy()
    ref = OD.lnL_direct(point, draws, 128, 64, 16, 50.0, 200.0)
    _cmp(got, ref)


def test_time_rule(R):
    """t integrated on a +-1 ms window (fixed-spacing rule), against the oracle."""
    point, exact, info, draws, logw = W.config0(n_draws=12)
    tr = info["truth"]
    d = {p: np.concatenate([[tr[p]], np.asarray(draws[p])]) for p in W.PARAMS}
    pt = R.Point(point)
    args = (64, 32, 16, 50.0, 200.0, 24, tr["t"] - 1e-3, tr["t"] + 1e-3)
    got = R.rift_ile_lnL_direct(pt, R.Draws(d), *args).cpu().numpy()
    ref = OD.lnL_direct(point, d, *args)
    _cmp(got, ref)
    assert np.isfinite(got[0])


def test_invalid_rules(R):
    point, exact, info, draws, logw = W.config0(n_draws=4)
    pt = R.Point(point)
    d = R.Draws(draws)
    for args in ((0, 8, 16, 50.0, 200.0), (8, 8, 65, 50.0, 200.0), (8, 8, 16, 200.0, 50.0),
                 (8, 8, 16, 50.0, 200.0, 4, 0.01, -0.01), (8, 8, 16, 50.0, 200.0, 0, 0.0, 0.0, 2),
                 (8, 8, 16, 50.0, 200.0, 4, -0.01, 0.01, -1),
                 (8, 8, 16, 50.0, 200.0, 2000, -0.01, 0.01, 2)):
        with pytest.raises(R.RiftError):
            R.rift_ile_lnL_direct(pt, d, *args)


def test_lnz_with_the_direct_marginal(R):
    """The evidence over (ra, dec, incl, t) draws with the direct marginal as
    integrand equals the oracle's LSE of the oracle's per-draw values."""
    import oracle as O
    point, exact, info, draws, logw = W.config0(n_draws=48)
    pt = R.Point(point)
    args = (64, 32, 16, 50.0, 200.0)
    z = R.rift_ile_lnZ_direct(pt, R.Draws(draws), *args)
    ref = OD.lnL_direct(point, draws, *args)
    zr = O.lnZ(ref, np.zeros(len(ref)))
    assert abs(z[0] - zr[0]) <= 1e-9 * max(1.0, abs(zr[0]))
    assert abs(z[2] - zr[2]) <= 1e-7 * zr[2]


@pytest.mark.parametrize("n_t,t_up", [(8, 3), (5, 4)])
def test_band_limited_time_rule(R, n_t, t_up):
    """eq. ap:tband: coarse data coefficients sinc-reconstructed at t_up fine
    nodes per interval, against the oracle's rule on the same draws."""
    point, exact, info, draws, logw = W.config0(n_draws=10)
    tr = info["truth"]
    d = {p: np.concatenate([[tr[p]], np.asarray(draws[p])]) for p in W.PARAMS}
    pt = R.Point(point)
    args = (64, 32, 16, 50.0, 200.0, n_t, tr["t"] - 1e-3, tr["t"] + 1e-3, t_up)
    got = R.rift_ile_lnL_direct(pt, R.Draws(d), *args).cpu().numpy()
    ref = OD.lnL_direct(point, d, *args)
    _cmp(got, ref)
    assert np.isfinite(got[0])
    # t_up = 1 is the fixed-spacing rule
    one = R.rift_ile_lnL_direct(pt, R.Draws(d), *args[:-1], 1).cpu().numpy()
    fixed = R.rift_ile_lnL_direct(pt, R.Draws(d), *args[:-1]).cpu().numpy()
    assert np.array_equal(one, fixed)


def test_mixed_distance_sum(R):
    """precision=FP32_MIXED: the prior-weighted Gauss-Hermite sum in float,
    everything else in double: within 1e-5 of the FP64 oracle (the north-star
    bound is 1e-3) on the 3G network and on the two-detector workload, with
    the same -inf pattern."""
    for point, exact, info, draws, logw in (W.config_3g(1, 4, 30.0, 0.02, 16),
                                            W.config0(n_draws=24)):
        pt = R.Point(point)
        args = (96, 48, 16, 50.0, 200.0)
        got = R.rift_ile_lnL_direct(pt, R.Draws(draws), *args, precision=R.FP32_MIXED).cpu().numpy()
        ref = OD.lnL_direct(point, draws, *args)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        assert np.max(np.abs(got[fin] - ref[fin])) <= 1e-5
    # the band-limited time rule in the mixed form too
    point, exact, info, draws, logw = W.config0(n_draws=6)
    tr = info["truth"]
    args = (64, 32, 16, 50.0, 200.0, 8, tr["t"] - 1e-3, tr["t"] + 1e-3, 3)
    pt = R.Point(point)
    got = R.rift_ile_lnL_direct(pt, R.Draws(draws), *args, precision=R.FP32_MIXED).cpu().numpy()
    ref = OD.lnL_direct(point, draws, *args)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.max(np.abs(got[fin] - ref[fin])) <= 1e-5
    with pytest.raises(R.RiftError):
        R.rift_ile_lnL_direct(pt, R.Draws(draws), 8, 8, 16, 1e-3, 1e7, precision=R.FP32_MIXED)
    with pytest.raises(R.RiftError):
        R.rift_ile_lnL_direct(pt, R.Draws(draws), 8, 8, 16, 50.0, 200.0, precision=7)


@pytest.mark.parametrize("n_phi,n_psi", [(256, 8), (12, 300), (205, 257)])
def test_grids_beyond_the_kernel_tables(R, n_phi, n_psi):
    """Phase grids beyond the column cache (n_phi > 204) and polarisation
    grids beyond the phase table (n_psi > 256) take the computed paths; both
    must agree with the oracle like the tabulated ones."""
    point, exact, info, draws, logw = W.config0(n_draws=6)
    tr = info["truth"]
    d = {p: np.concatenate([[tr[p]], np.asarray(draws[p])]) for p in W.PARAMS}
    pt = R.Point(point)
    args = (n_phi, n_psi, 16, 50.0, 200.0)
    got = R.rift_ile_lnL_direct(pt, R.Draws(d), *args).cpu().numpy()
    ref = OD.lnL_direct(point, d, *args)
    _cmp(got, ref)
    assert np.isfinite(got[0])
