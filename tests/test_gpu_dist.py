"""GPU parity of the distance-marginalised likelihood on the full 3G event
workload (ET triangle + CE 40 km + CE 20 km, ten modes, SNR 1000, 32768 Hz
table over +-50 ms): per-draw marginal lnL over the log-uniform lnD node
table of eq. ap:dlog, its lnZ, and chunked streaming merged by LSE states.
"""
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


@pytest.fixture(scope="module")
def cfg4():
    return W.config4(n_draws=1 << 14)


@pytest.fixture(scope="module")
def nodes(R):
    return R.rift_ile_dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)


def test_marginal_lnl_matches_oracle(R, cfg4, nodes):
    point, exact, info, draws, logw = cfg4
    pt = R.Point(point)
    ref = O.lnL_distmarg(O.OraclePoint(point), draws, *nodes)
    got64 = R.rift_ile_lnL_dist(pt, draws, nodes, R.FP64).cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= 1e-9 * np.maximum(1, np.abs(ref))), np.max(np.abs(got64 - ref))
    got32 = R.rift_ile_lnL_dist(pt, draws, nodes, R.FP32_MIXED).cpu().numpy()
    near = ref >= ref.max() - 50
    assert np.max(np.abs(got32 - ref)[near]) <= 1e-3, np.max(np.abs(got32 - ref)[near])
    _, td, tq, _ = O.lnL(O.OraclePoint(point), {**draws, "lnD": np.full(len(ref), np.log(100.0))},
                         terms=True)
    assert np.all(np.abs(got32 - ref) <= 1e-4 * (np.abs(td) + np.abs(tq)) + 1e-6)


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)])
def test_marginal_lnz_and_streaming(R, cfg4, nodes, prec, tol):
    point, exact, info, draws, logw = cfg4
    pt = R.Point(point)
    ref = O.lnZ(O.lnL_distmarg(O.OraclePoint(point), draws, *nodes), np.asarray(logw, dtype=np.float64))
    got = R.rift_ile_lnZ(pt, R.Draws(draws, logw), prec, dist=nodes)
    assert abs(got[0] - ref[0]) <= tol * max(1.0, abs(ref[0]) if prec == 0 else 1.0), (got, ref)
    n = len(draws["t"])
    states = []
    for a in range(0, n, 5000):
        sub = {p: np.asarray(draws[p])[a:a + 5000] for p in W.PARAMS}
        states.append(R.rift_ile_lnZ_state(pt, R.Draws(sub, np.asarray(logw)[a:a + 5000]), prec, dist=nodes))
    merged, _ = R.rift_ile_lnZ_merge(states)
    assert abs(merged[0] - got[0]) <= 1e-9 * max(1.0, abs(got[0]))


def test_marginal_gradient_matches_oracle(R, cfg4, nodes):
    """d lnL_marg / d theta = E[x] dK - E[x^2] dR/2 over the node posterior
    (lnD slot zero): FP64 to 1e-8 of each component's scale, FP32-mixed to
    1e-4 on draws within 50 nat of the best."""
    point, exact, info, draws, logw = cfg4
    pt = R.Point(point)
    ref, rg = O.lnL_distmarg(O.OraclePoint(point), draws, *nodes, grad=True)
    scale = np.abs(rg) + np.sqrt(np.mean(rg ** 2, axis=0))[None, :] + 1e-300
    near = ref >= ref.max() - 50
    for prec, tol in ((0, 1e-8), (1, 1e-4)):
        lnl, g = R.rift_ile_lnL_dist(pt, draws, nodes, prec, grad=True)
        lnl, g = lnl.cpu().numpy(), g.cpu().numpy().T
        assert np.all(g[:, 5] == 0)
        err = np.abs(g - rg) / scale
        sel = slice(None) if prec == 0 else near
        assert err[sel].max() < tol, (prec, err[sel].max(axis=0))
        assert np.max(np.abs(lnl - ref)[near]) <= (1e-6 if prec == 0 else 1e-3)


@pytest.mark.parametrize("kind", ["thinned", "jittered"])
def test_marginal_on_irregular_tables(R, cfg4, nodes, kind):
    """The node search on tables not uniform in ln x: thinned (every other
    node of the lower half dropped; the kernels bisect the whole table) and
    jittered (each ln x moved by up to 0.4 of the step; the kernels start
    from the estimated position and fall back where its bracket fails)."""
    point, exact, info, draws, logw = cfg4
    x, lnw = nodes
    if kind == "thinned":
        h = len(x) // 2
        keep = np.r_[np.arange(0, h, 2), np.arange(h, len(x))]
        x2, lnw2 = x[keep].copy(), lnw[keep].copy()
    else:
        step = np.log(x[0] / x[-1]) / (len(x) - 1)
        u = np.random.default_rng(7).uniform(-0.4, 0.4, len(x))
        x2, lnw2 = x * np.exp(u * step), lnw.copy()
        assert np.all(np.diff(x2) < 0)
    pt = R.Point(point)
    ref = O.lnL_distmarg(O.OraclePoint(point), draws, x2, lnw2)
    got32 = R.rift_ile_lnL_dist(pt, draws, (x2, lnw2), R.FP32_MIXED).cpu().numpy()
    near = ref >= ref.max() - 50
    assert np.max(np.abs(got32 - ref)[near]) <= 1e-3, np.max(np.abs(got32 - ref)[near])
    _, td, tq, _ = O.lnL(O.OraclePoint(point), {**draws, "lnD": np.full(len(ref), np.log(100.0))},
                         terms=True)
    assert np.all(np.abs(got32 - ref) <= 1e-4 * (np.abs(td) + np.abs(tq)) + 1e-6)


@pytest.mark.parametrize("kind", ["beyond", "below", "one", "two"])
def test_marginal_on_tables_away_from_the_peak(R, cfg4, kind):
    """Node tables that do not bracket x* = K/R of the draws (the injected
    distance is D_ref, x* ~ 1): every node at larger D (x < x*), every node
    at smaller D (x > x*), and tables of one and two nodes."""
    point, exact, info, draws, logw = cfg4
    if kind == "beyond":
        x, lnw = R.rift_ile_dist_nodes(150.0, 200.0, 100.0, 1e-4, 1000.0)
    elif kind == "below":
        x, lnw = R.rift_ile_dist_nodes(40.0, 80.0, 100.0, 1e-4, 1000.0)
    elif kind == "one":
        x, lnw = np.array([0.9]), np.array([0.0])
    else:
        x, lnw = np.array([1.05, 0.95]), np.array([-0.1, 0.2])
    pt = R.Point(point)
    ref = O.lnL_distmarg(O.OraclePoint(point), draws, x, lnw)
    got64 = R.rift_ile_lnL_dist(pt, draws, (x, lnw), R.FP64).cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= 1e-9 * np.maximum(1, np.abs(ref))), np.max(np.abs(got64 - ref))
    got32 = R.rift_ile_lnL_dist(pt, draws, (x, lnw), R.FP32_MIXED).cpu().numpy()
    near = ref >= ref.max() - 50
    assert np.max(np.abs(got32 - ref)[near]) <= 1e-3, np.max(np.abs(got32 - ref)[near])


def test_marginal_with_zero_weight_nodes(R, cfg4, nodes):
    """Nodes of zero weight (ln w = -inf) where the peak draws' x* falls,
    so that the scan starts on one: their terms add nothing, in both
    precisions, as in the oracle's sum."""
    point, exact, info, draws, logw = cfg4
    x, lnw = nodes
    lnw = lnw.copy()
    lnw[np.abs(np.log(x)) < 0.01] = -np.inf
    assert np.isinf(lnw).sum() >= 3
    pt = R.Point(point)
    ref = O.lnL_distmarg(O.OraclePoint(point), draws, x, lnw)
    assert np.all(np.isfinite(ref))
    got64 = R.rift_ile_lnL_dist(pt, draws, (x, lnw), R.FP64).cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= 1e-9 * np.maximum(1, np.abs(ref))), np.max(np.abs(got64 - ref))
    got32 = R.rift_ile_lnL_dist(pt, draws, (x, lnw), R.FP32_MIXED).cpu().numpy()
    assert np.all(np.isfinite(got32))
    near = ref >= ref.max() - 50
    assert np.max(np.abs(got32 - ref)[near]) <= 1e-3, np.max(np.abs(got32 - ref)[near])
