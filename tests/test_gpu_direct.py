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


def _fine_point():
    """Noise-free two-detector point with its table at 16 384 Hz (band to
    512 Hz), as in the oracle's time-rule pins."""
    rng = np.random.default_rng(41)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:4], f_low=20.0, f_max=512.0, df=0.5, rate=16384.0,
        half_window=0.03, snr=20.0, truth=truth, gmst=0.4, d_ref=100.0, rng=rng, noise=False,
        q_dtype=np.complex128)
    return point, info


def _near_truth(info, n, rng):
    tr = info["truth"]
    d = {p: np.full(n, tr[p]) for p in W.PARAMS}
    d["ra"] = d["ra"] + rng.normal(0, 0.01, n)
    d["dec"] = d["dec"] + rng.normal(0, 0.01, n)
    d["incl"] = d["incl"] + rng.normal(0, 0.05, n)
    return d


def test_peak_local_time_rule_against_oracle(R):
    """eq. ap:tlocal on the band-limited fine nodes: GPU against the oracle,
    every draw within 1e-9 relative; the same value as the band-limited rule
    within the remainder bound the oracle reports; a tolerance no bound meets
    gives the band-limited rule itself."""
    point, info = _fine_point()
    tr = info["truth"]
    d = _near_truth(info, 6, np.random.default_rng(4))
    h, half = 1.0 / 2048, 32
    lo, hi = tr["t"] - half * h, tr["t"] + half * h
    pt = R.Point(point)
    args = (48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)
    got = R.rift_ile_lnL_direct(pt, R.Draws(d), *args, t_local=True).cpu().numpy()
    diag = []
    ref = OD.lnL_direct(point, d, *args, t_local=True, diag=diag)
    _cmp(got, ref)
    assert not any(g["fallback"] for g in diag)
    band = R.rift_ile_lnL_direct(pt, R.Draws(d), *args).cpu().numpy()
    for i, g in enumerate(diag):
        assert abs(got[i] - band[i]) <= 2 * math.exp(g["gap"]) + 1e-12 * abs(band[i])
    fb = R.rift_ile_lnL_direct(pt, R.Draws(d), *args, t_local=True, t_tol=1e-300).cpu().numpy()
    assert np.max(np.abs(fb - band) / np.abs(band)) <= 1e-13


def test_peak_local_time_rule_two_signals(R):
    """Two identical signals 300 table samples apart, tolerance 1e-8: both
    neighbourhoods kept, GPU against the oracle within 1e-9 relative."""
    point, info = _fine_point()
    Q = np.asarray(point["Q"])
    Q2 = np.zeros_like(Q)
    Q2[:, 300:, :] = Q[:, :-300, :]
    both = dict(point)
    both["Q"] = Q + Q2
    tr = info["truth"]
    dts = 300 * float(point["q_dt"])
    d = _near_truth(info, 4, np.random.default_rng(5))
    h, half = 1.0 / 2048, 48
    lo, hi = tr["t"] - half * h + dts / 2, tr["t"] + half * h + dts / 2
    args = (48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)
    got = R.rift_ile_lnL_direct(R.Point(both), R.Draws(d), *args, t_local=True,
                                t_tol=1e-8).cpu().numpy()
    diag = []
    ref = OD.lnL_direct(both, d, *args, t_local=True, t_tol=1e-8, diag=diag)
    _cmp(got, ref)
    assert all(len(g["maxima"]) >= 2 for g in diag)


def test_peak_local_rule_refuses_bad_arguments(R):
    point, info = _fine_point()
    pt = R.Point(point)
    d = _near_truth(info, 1, np.random.default_rng(6))
    tr = info["truth"]
    for kw in ({"t_local": True}, {"t_local": True, "t_c": 0.0, "t_up": 4},
               {"t_local": True, "t_tol": 2.0, "t_up": 4}):
        args = dict(n_t=16, t_lo=tr["t"] - 1e-3, t_hi=tr["t"] + 1e-3, t_up=kw.pop("t_up", 0))
        with pytest.raises(R.RiftError):
            R.rift_ile_lnL_direct(pt, R.Draws(d), 32, 16, 8, 50.0, 200.0, **args, **kw)


def test_mirrored_band_limited_rule_against_oracle(R):
    """The mirrored reconstruction of the fine coefficients (alone and under
    the peak-local rule): GPU against the oracle within 1e-9 relative; with
    the peak near the window's end the mirrored and truncated values differ."""
    point, info = _fine_point()
    tr = info["truth"]
    d = _near_truth(info, 5, np.random.default_rng(7))
    h, half = 1.0 / 2048, 16
    pt = R.Point(point)
    for shift in (0.0, 12 * h):  # peak centred, and 4 coarse samples from the end
        lo, hi = tr["t"] - half * h + shift, tr["t"] + half * h + shift
        args = (48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)
        got = R.rift_ile_lnL_direct(pt, R.Draws(d), *args, t_mirror=True).cpu().numpy()
        _cmp(got, OD.lnL_direct(point, d, *args, t_mirror=True))
        loc = R.rift_ile_lnL_direct(pt, R.Draws(d), *args, t_mirror=True, t_local=True,
                                    t_tol=1e-8).cpu().numpy()
        _cmp(loc, OD.lnL_direct(point, d, *args, t_mirror=True, t_local=True, t_tol=1e-8))
    trunc = R.rift_ile_lnL_direct(pt, R.Draws(d), *args).cpu().numpy()
    assert np.max(np.abs(trunc - got)) > 1e-6
