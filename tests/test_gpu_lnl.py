"""GPU parity of lnL and lnZ against the FP64 oracle (through the C ABI).

FP64 path: |dlnL| <= 1e-9 max(1, |lnL|) on every draw.  FP32-mixed path:
|dlnL| <= 1e-3 on draws within 50 nats of the best draw, |dlnZ| <= 1e-4 (the
stated precision targets), and on every draw |dlnL| <= 1e-4 (|T_d| + |T_q|):
the FP32 template coefficients perturb the template by ~u |h| (u = 2^-24),
which moves lnL by <delta h|d - h>, so far from the peak the error grows
with |d - h| while staying a small fraction of the two terms.
"""
import math

import numpy as np
import pytest

import oracle as O
import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


def _np(d):
    return {p: np.asarray(d[p]) for p in W.PARAMS}


def subset(d, idx):
    return {p: np.asarray(d[p])[idx] for p in W.PARAMS}


@pytest.fixture(scope="module")
def cfg0():
    return W.config0()


@pytest.fixture(scope="module")
def cfg1_small():
    return W.config1(n_draws=1 << 15)


@pytest.fixture(scope="module")
def cfg2_small():
    return W.config2(n_draws=1 << 15)


def fp64_tol(ref):
    return 1e-9 * np.maximum(1.0, np.abs(ref))


def test_fp64_config0_matches_oracle(R, cfg0):
    point, exact, info, draws, logw = cfg0
    pt = R.Point(point)
    got = R.rift_ile_lnL(pt, draws, R.FP64).cpu().numpy()
    ref = O.lnL(O.OraclePoint(point), draws)
    assert np.all(np.abs(got - ref) <= fp64_tol(ref)), np.max(np.abs(got - ref))


def test_fp64_config1_matches_oracle(R, cfg1_small):
    point, exact, info, draws, logw = cfg1_small
    pt = R.Point(point)
    got = R.rift_ile_lnL(pt, draws, R.FP64).cpu().numpy()
    ref = O.lnL(O.OraclePoint(point), draws)
    assert np.all(np.abs(got - ref) <= fp64_tol(ref)), np.max(np.abs(got - ref) / fp64_tol(ref))


@pytest.mark.parametrize("which", ["cfg0", "cfg1_small", "cfg2_small"])
def test_mixed_matches_oracle(R, which, request):
    point, exact, info, draws, logw = request.getfixturevalue(which)
    pt = R.Point(point)
    got = R.rift_ile_lnL(pt, draws, R.FP32_MIXED).cpu().numpy()
    ref, td, tq, _ = O.lnL(O.OraclePoint(point), draws, terms=True)
    err = np.abs(got - ref)
    near = ref >= ref.max() - 50.0
    assert near.sum() > 0
    assert err[near].max() <= 1e-3, (which, err[near].max())
    assert np.all(err <= 1e-4 * (np.abs(td) + np.abs(tq)) + 1e-6), (which, np.max(err / (np.abs(td) + np.abs(tq))))


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)])
def test_lnz_matches_oracle(R, cfg1_small, prec, tol):
    point, exact, info, draws, logw = cfg1_small
    pt = R.Point(point)
    Rd = R.Draws(draws, logw)
    lnz, sig, neff = R.rift_ile_lnZ(pt, Rd, prec)
    ref_l = O.lnL(O.OraclePoint(point), draws)
    rz, rs, rn = O.lnZ(ref_l, np.asarray(logw, dtype=np.float64))
    assert abs(lnz - rz) <= tol * max(1.0, abs(rz) if prec == 0 else 1.0), (lnz, rz)
    assert abs(sig - rs) <= 1e-3 * rs + 1e-9
    assert abs(neff - rn) <= 1e-4 * rn


def test_lnz_config0_prior_draws(R, cfg0):
    point, exact, info, draws, logw = cfg0
    pt = R.Point(point)
    ref = O.lnZ(O.lnL(O.OraclePoint(point), draws))
    for prec, tol in ((0, 1e-12), (1, 1e-6)):
        got = R.rift_ile_lnZ(pt, draws, prec)
        assert abs(got[0] - ref[0]) <= tol * max(1, abs(ref[0]))
        assert abs(got[2] - ref[2]) <= 1e-5 * ref[2]


def test_state_merge_equals_whole(R, cfg1_small):
    point, exact, info, draws, logw = cfg1_small
    pt = R.Point(point)
    n = len(draws["t"])
    parts = []
    for a, b in ((0, 1000), (1000, 20001), (20001, n)):
        idx = slice(a, b)
        parts.append(R.rift_ile_lnZ_state(pt, R.Draws(subset(draws, idx), np.asarray(logw)[idx]),
                                          R.FP32_MIXED))
    merged, _ = R.rift_ile_lnZ_merge(parts)
    whole = R.rift_ile_lnZ(pt, R.Draws(draws, logw), R.FP32_MIXED)
    assert abs(merged[0] - whole[0]) < 1e-6
    assert abs(merged[2] - whole[2]) < 1e-4 * whole[2]


@pytest.mark.parametrize("n", [1, 2, 31, 33, 255, 257, 1000003])
def test_ragged_sizes(R, n):
    point, exact, info, draws, logw = W.config1(n_draws=n)
    pt = R.Point(point)
    for prec in (0, 1):
        got = R.rift_ile_lnL(pt, draws, prec).cpu().numpy()
        assert got.shape == (n,)
        idx = np.unique(np.linspace(0, n - 1, min(n, 257)).astype(int))
        ref, td, tq, _ = O.lnL(O.OraclePoint(point), subset(draws, idx), terms=True)
        tol = fp64_tol(ref) if prec == 0 else 1e-4 * (np.abs(td) + np.abs(tq)) + 1e-6
        assert np.all(np.abs(got[idx] - ref) <= tol)


def test_empty_draws(R, cfg0):
    point = cfg0[0]
    pt = R.Point(point)
    empty = {p: np.zeros(0) for p in W.PARAMS}
    assert R.rift_ile_lnL(pt, empty, R.FP64).numel() == 0
    lnz, sig, neff = R.rift_ile_lnZ(pt, empty, R.FP32_MIXED)
    assert lnz == -math.inf and neff == 0.0


def test_nan_draw_and_out_of_table(R, cfg1_small):
    point, exact, info, draws, logw = cfg1_small
    d = subset(draws, np.arange(64))
    d["t"] = d["t"].copy()
    d["ra"] = d["ra"].copy()
    d["ra"][3] = np.nan
    d["t"][5] = 0.5  # far outside every table: all taps read zero
    pt = R.Point(point)
    ref, td, tq, oob = O.lnL(O.OraclePoint(point), d, terms=True)
    assert oob >= 4 * point["K"]
    for prec in (0, 1):
        got = R.rift_ile_lnL(pt, d, prec).cpu().numpy()
        assert np.isnan(got[3])
        ok = ~np.isnan(ref)
        assert np.all(np.abs(got[ok] - ref[ok]) <= 1e-4 * (np.abs(td[ok]) + np.abs(tq[ok])) + 1e-6)
        assert abs(got[5] - (-tq[5])) < 1e-6 * abs(tq[5]) + 1e-3
        R.rift_ile_lnZ(pt, subset(d, np.r_[0:3, 4:64]), prec)
        assert R.rift_ile_last_oob() >= 4 * point["K"]
        assert math.isnan(R.rift_ile_lnZ(pt, d, prec)[0])


def test_zero_prior_weight_draws(R, cfg1_small):
    """Draws with ln w = -inf (outside the prior) carry no weight; +inf
    dominates; NaN poisons lnZ, as in the oracle."""
    point, exact, info, draws, logw = cfg1_small
    lw = np.asarray(logw, dtype=np.float32).copy()
    lw[::7] = -np.inf
    pt = R.Point(point)
    ref = O.lnZ(O.lnL(O.OraclePoint(point), draws), lw.astype(np.float64))
    for prec, tol in ((0, 1e-9), (1, 1e-4)):
        got = R.rift_ile_lnZ(pt, R.Draws(draws, lw), prec)
        assert abs(got[0] - ref[0]) <= tol * max(1.0, abs(ref[0]) if prec == 0 else 1.0), (prec, got, ref)
        assert abs(got[2] - ref[2]) <= 1e-4 * ref[2]
    lw2 = lw.copy()
    lw2[3] = np.nan
    for prec in (0, 1):
        assert np.isnan(R.rift_ile_lnZ(pt, R.Draws(draws, lw2), prec)[0])


def test_deterministic(R, cfg1_small):
    point, exact, info, draws, logw = cfg1_small
    pt = R.Point(point)
    Rd = R.Draws(draws, logw)
    for prec in (0, 1):
        a = R.rift_ile_lnL(pt, Rd, prec)
        b = R.rift_ile_lnL(pt, Rd, prec)
        assert torch.equal(a, b)
        assert R.rift_ile_lnZ_state(pt, Rd, prec) == R.rift_ile_lnZ_state(pt, Rd, prec)


def test_invalid_arguments_are_rejected(R, cfg0):
    point = dict(cfg0[0])
    bad = dict(point)
    bad["ell"] = np.array([9, 2], dtype=np.int32)
    with pytest.raises(R.RiftError) as e:
        R.Point(bad)
    assert e.value.code == -3
    bad = dict(point)
    bad["q_dt"] = -1.0
    with pytest.raises(R.RiftError):
        R.Point(bad)
    pt = R.Point(point)
    with pytest.raises(R.RiftError):
        R.rift_ile_lnZ(pt, cfg0[3], 7)


@pytest.mark.parametrize("n_modes", [1, 3, 5])
def test_odd_mode_counts(R, n_modes):
    """Odd mode counts run the kernels compiled for the next even count with
    the whitened width padded past 2M; parity with the oracle holds."""
    rng = np.random.default_rng(W.seed_for(5, n_modes))
    truth = W.default_truth(rng, W.D_REF)
    point, exact, info = W.make_point(
        dets=W.random_l_detectors(rng, 3), modes=W.MODES10[:n_modes], f_low=5.0, f_max=2048.0,
        df=0.25, rate=32768.0, half_window=0.03, snr=300.0, truth=truth,
        gmst=float(rng.uniform(0, 2 * math.pi)), d_ref=W.D_REF, rng=rng, noise=False,
        q_dtype=np.complex64)
    sig = W.proposal_sigma(info, exact)
    draws, logw = W.mixture_draws(rng, W.Prior(0.5 * W.D_REF, 2.0 * W.D_REF, 0.01), truth, sig,
                                  20000)
    draws = W.as_float(draws, np.float32)
    pt = R.Point(point)
    assert pt.info()["M"] == n_modes
    ref = O.lnL(O.OraclePoint(point), draws)
    got64 = R.rift_ile_lnL(pt, draws, R.FP64).cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= fp64_tol(ref))
    got32 = R.rift_ile_lnL(pt, draws, R.FP32_MIXED).cpu().numpy()
    near = ref >= ref.max() - 50
    assert np.max(np.abs(got32 - ref)[near]) <= 1e-3
    rz = O.lnZ(ref, np.asarray(logw, dtype=np.float64))
    z = R.rift_ile_lnZ(pt, R.Draws(draws, logw.astype(np.float32)), R.FP32_MIXED)
    assert abs(z[0] - rz[0]) <= 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_async_state_equals_sync_state(R, cfg1_small, prec):
    """rift_ile_lnZ_state_async runs the same kernels as rift_ile_lnZ_state
    and leaves the same state in device memory, bit for bit; chained calls on
    one stream stay ordered; zero draws give the empty state."""
    point, exact, info, draws, logw = cfg1_small
    pt = R.Point(point)
    d = R.Draws(draws, logw)
    ref = R.rift_ile_lnZ_state(pt, d, prec)
    outs = [R.rift_ile_lnZ_state_async(pt, d, prec) for _ in range(3)]
    for o in outs:
        assert tuple(o.cpu().tolist()) == ref
    nodes = R.rift_ile_dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)
    ref_d = R.rift_ile_lnZ_state(pt, d, prec, dist=nodes)
    assert tuple(R.rift_ile_lnZ_state_async(pt, d, prec, dist=nodes).cpu().tolist()) == ref_d
    empty = {p: np.zeros(0, dtype=np.float32) for p in W.PARAMS}
    e = R.rift_ile_lnZ_state_async(pt, empty, prec).cpu().tolist()
    assert e[0] == -math.inf and e[1] == 0.0 and e[3] == 0.0
