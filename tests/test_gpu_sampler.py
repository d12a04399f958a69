"""The warp-per-draw FP32-mixed kernel of the sampler regime (App. H: small
batches of draws per lnL + gradient call).

rift_ile_set_small_batch selects it (up to that many draws) or turns it off;
both kernels are run here on the same draws:

* the SNR-1000 differentiation workload (K=4, M=10) at 1, 31, 128, 1024 and
  8192 draws: lnL within 1e-3 nat of the FP64 oracle on draws within 50 nat
  of the best, every gradient component within 1e-4 of |g| + RMS g there, and
  within rounding of the one-thread-per-draw kernel;
* chained calls (programmatic dependent launch) reading draws that the
  kernel before them wrote, eagerly and in a CUDA graph;
* forward-only lnL, the full-event network (K=5, two detector classes,
  wider whitened width), odd mode counts, a NaN draw and draws whose taps
  leave the table, an empty batch.
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
    prev = R.rift_ile_set_small_batch(4096)
    yield R
    R.rift_ile_set_small_batch(prev)


@pytest.fixture(scope="module")
def cfg2():
    return W.config2(n_draws=8192)


def scale(g):
    return np.abs(g) + np.sqrt(np.mean(g ** 2, axis=0))[None, :]


def run(R, pt, draws, warp: bool, grad=True):
    R.rift_ile_set_small_batch(1 << 20 if warp else 0)
    try:
        if grad:
            lnl, g = R.rift_ile_lnL_grad(pt, draws, R.FP32_MIXED)
            return lnl.cpu().numpy(), g.cpu().numpy().T
        return R.rift_ile_lnL(pt, draws, R.FP32_MIXED).cpu().numpy(), None
    finally:
        R.rift_ile_set_small_batch(4096)


def sub(draws, n):
    return {p: np.asarray(draws[p])[:n] for p in W.PARAMS}


@pytest.mark.parametrize("n", [1, 31, 128, 1024, 8192])
def test_warp_kernel_matches_oracle_and_per_thread_kernel(R, cfg2, n):
    point, exact, info, draws, logw = cfg2
    d = sub(draws, n)
    pt = R.Point(point)
    lw, gw = run(R, pt, d, warp=True)
    lt, gt = run(R, pt, d, warp=False)
    rl, rg = O.lnL_grad(O.OraclePoint(point), d)
    near = rl >= rl.max() - 50
    assert np.max(np.abs(lw - rl)[near]) <= 1e-3
    err = np.abs(gw - rg) / scale(rg)
    assert err[near].max() < 1e-4, err[near].max(axis=0)
    # the two kernels differ by rounding only (reduction order, e^{i m phi});
    # far from the peak both errors grow as eps |e - w|^2 (1e-4 relative at
    # lnL ~ -1e5), so the whole-batch bound is relative
    assert np.max(np.abs(lw - lt)[near]) <= 2e-4
    assert np.max(np.abs(lw - lt) / np.maximum(1.0, np.abs(lt))) <= 1e-4
    assert np.max((np.abs(gw - gt) / scale(gt))[near]) < 2e-5


def test_warp_kernel_forward_only(R, cfg2):
    point, exact, info, draws, logw = cfg2
    d = sub(draws, 777)
    pt = R.Point(point)
    lw, _ = run(R, pt, d, warp=True, grad=False)
    lg, _ = run(R, pt, d, warp=True, grad=True)
    rl = O.lnL(O.OraclePoint(point), d)
    near = rl >= rl.max() - 50
    assert np.max(np.abs(lw - rl)[near]) <= 1e-3
    assert np.array_equal(lw, lg)  # the same arithmetic with or without the adjoint


def test_warp_kernel_event_network_two_classes(R):
    """K = 5 (ET triangle + CE 40 km + CE 20 km) with the two CE detectors'
    noise scaled (their Q, U and V by 1.7, a consistent point): two detector
    classes, so the per-class mat-vec, sums and iota/phi_ref terms run twice."""
    point, exact, info, draws, logw = W.config4(n_draws=512)
    point = dict(point)
    for key in ("Q", "U", "V"):
        a = np.array(point[key])
        a[3:] = (a[3:] * 1.7).astype(a.dtype)
        point[key] = a
    pt = R.Point(point)
    assert pt.info()["ncls"] == 2
    lw, gw = run(R, pt, draws, warp=True)
    rl, rg = O.lnL_grad(O.OraclePoint(point), draws)
    near = rl >= rl.max() - 50
    assert np.max(np.abs(lw - rl)[near]) <= 1e-3
    assert (np.abs(gw - rg) / scale(rg))[near].max() < 1e-4


@pytest.mark.parametrize("n_modes", [1, 3, 7])
def test_warp_kernel_odd_mode_counts(R, n_modes):
    rng = np.random.default_rng(50 + n_modes)
    dets = W.random_l_detectors(rng, 3)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:n_modes], f_low=20.0, f_max=512.0, df=0.5, rate=8192.0,
        half_window=0.05, snr=40.0, truth=truth, gmst=0.3, d_ref=100.0, rng=rng, noise=True,
        q_dtype=np.complex64)
    prior = W.Prior(50.0, 200.0, 0.01)
    sigma = {p: s for p, s in zip(W.PARAMS, (0.01, 0.01, 0.05, 0.05, 0.05, 0.05, 1e-4))}
    d, _ = W.mixture_draws(rng, prior, truth, sigma, 300)
    d = W.as_float(d, np.float32)
    pt = R.Point(point)
    lw, gw = run(R, pt, d, warp=True)
    rl, rg = O.lnL_grad(O.OraclePoint(point), d)
    near = rl >= rl.max() - 50
    assert np.max(np.abs(lw - rl)[near]) <= 1e-3
    assert (np.abs(gw - rg) / scale(rg))[near].max() < 1e-4


def test_warp_kernel_nan_and_out_of_table(R, cfg2):
    point, exact, info, draws, logw = cfg2
    d = {p: np.array(np.asarray(draws[p])[:64], dtype=np.float32) for p in W.PARAMS}
    d["ra"][3] = np.nan
    d["t"][5] = 0.5      # far outside the +-20 ms tables: every tap reads zero
    pt = R.Point(point)
    lw, gw = run(R, pt, d, warp=True)
    lt, gt = run(R, pt, d, warp=False)
    assert np.isnan(lw[3]) and np.all(np.isnan(gw[3]))
    assert np.isnan(lt[3])
    fin = np.ones(64, bool)
    fin[3] = False
    rl = O.lnL(O.OraclePoint(point), {p: d[p][fin] for p in W.PARAMS})
    assert np.max(np.abs(lw[fin] - rl) / np.maximum(1, np.abs(rl))) < 1e-5
    assert np.isfinite(lw[5]) and abs(lw[5] - lt[5]) <= 1e-6 * max(1.0, abs(lt[5]))


def test_warp_kernel_empty_batch(R, cfg2):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    lw, gw = run(R, pt, sub(draws, 0), warp=True)
    assert lw.shape == (0,) and gw.shape == (0, 7)


def test_chained_calls_see_their_predecessors_writes(R, cfg2):
    """The warp kernel is launched with programmatic stream serialisation: its
    prologue may overlap the previous kernel, but it reads the draws and
    writes its outputs only after that kernel completes.  Eight calls, each
    preceded by a copy kernel that writes its draws into the same buffers and
    all writing the same output buffers, eagerly and captured in one CUDA
    graph: each call's result equals the same call made alone."""
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    n = 128
    sets = [{p: torch.tensor(np.asarray(draws[p])[n * s:n * (s + 1)], dtype=torch.float64,
                             device="cuda") for p in W.PARAMS} for s in range(8)]
    R.rift_ile_set_small_batch(1 << 20)
    try:
        alone = [R.rift_ile_lnL_grad(pt, R.Draws(s), R.FP32_MIXED) for s in sets]
        buf = {p: torch.empty(n, dtype=torch.float64, device="cuda") for p in W.PARAMS}
        d = R.Draws(buf)
        lnl = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty((7, n), dtype=torch.float64, device="cuda")
        keep_l = torch.empty((8, n), dtype=torch.float64, device="cuda")
        keep_g = torch.empty((8, 7, n), dtype=torch.float64, device="cuda")

        def chain():
            for s in range(8):
                for p in W.PARAMS:
                    buf[p].copy_(sets[s][p])
                R.rift_ile_lnL_grad(pt, d, R.FP32_MIXED, lnl, g)
                keep_l[s].copy_(lnl)
                keep_g[s].copy_(g)

        def check():
            torch.cuda.synchronize()
            for s in range(8):
                assert torch.equal(keep_l[s], alone[s][0]), s
                assert torch.equal(keep_g[s], alone[s][1]), s

        chain()
        check()
        keep_l.zero_()
        keep_g.zero_()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            chain()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            chain()
        keep_l.zero_()
        keep_g.zero_()
        graph.replay()
        check()
    finally:
        R.rift_ile_set_small_batch(4096)


def test_prepared_call_matches_and_follows_its_buffers(R, cfg2):
    """prepare_lnL_grad / prepare_lnL: the marshalled-once launch gives the
    plain call's results bit for bit, and a later call sees draws written
    into the same buffers in place."""
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    n = 128
    a = {p: torch.tensor(np.asarray(draws[p])[:n], dtype=torch.float64, device="cuda")
         for p in W.PARAMS}
    b = {p: torch.tensor(np.asarray(draws[p])[n:2 * n], dtype=torch.float64, device="cuda")
         for p in W.PARAMS}
    buf = {p: a[p].clone() for p in W.PARAMS}
    d = R.Draws(buf)
    R.rift_ile_set_small_batch(1 << 20)
    try:
        call = R.prepare_lnL_grad(pt, d, R.FP32_MIXED)
        fwd = R.prepare_lnL(pt, d, R.FP32_MIXED)
        l, g = call()
        ref_l, ref_g = R.rift_ile_lnL_grad(pt, R.Draws(a), R.FP32_MIXED)
        assert torch.equal(l, ref_l) and torch.equal(g, ref_g)
        assert torch.equal(fwd(), R.rift_ile_lnL(pt, R.Draws(a), R.FP32_MIXED))
        for p in W.PARAMS:
            buf[p].copy_(b[p])
        l, g = call()
        ref_l, ref_g = R.rift_ile_lnL_grad(pt, R.Draws(b), R.FP32_MIXED)
        assert torch.equal(l, ref_l) and torch.equal(g, ref_g)
    finally:
        R.rift_ile_set_small_batch(4096)
