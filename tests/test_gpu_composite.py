"""Composite-index response on the GPU (Sec. III; Earth rotation Paths A/B,
finite arms Path D), FP64 path, against the composite oracle:

* the per-draw coefficients C~^k_a (closed forms on the GPU, DFTs of the
  static antenna factor and delay in the oracle) agree to rounding;
* lnL per draw and lnZ agree within 1e-9 relative on the small fixtures,
  for several truncation orders, ragged draw counts and float32 draws;
* Omega = 0 gives the static FP64 likelihood of the (p, n) = (0, 0) block;
* out-of-table taps read zero and are counted; an empty draw set gives the
  empty LSE state;
* on the 3G network at full size (2^22 draws, the bench's launch) sampled
  draws match the oracle and the fused lnZ matches the LSE of the lnL output.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.composite as OC
import workload as W
import workload.composite as WC

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


CASES = [(WC.ROTATION, 0), (WC.ROTATION, 1), (WC.ROTATION, 3), (WC.FINITE_ARM, 0),
         (WC.FINITE_ARM, 3), (WC.FINITE_ARM, 6)]
_cache = {}


def fixture(kind, p_max, n_draws=1500):
    key = (kind, p_max, n_draws)
    if key not in _cache:
        _cache[key] = WC.comp_small(kind, p_max, n_draws=n_draws)
    return _cache[key]


@pytest.mark.parametrize("kind,p_max", CASES)
def test_coefficients_match_oracle(R, kind, p_max):
    point, exact, info, draws, logw = fixture(kind, p_max)
    cp = R.CompPoint(point)
    got = R.rift_ile_comp_coeffs(cp, R.Draws(draws, logw)).cpu().numpy()
    pt = OC.CompPoint(point)
    for i in range(0, len(draws["ra"]), 37):
        for k in range(pt.K):
            ref = pt.coeffs(k, draws["ra"][i], draws["dec"][i], draws["psi"][i], draws["t"][i])
            assert np.max(np.abs(got[i, k] - ref)) <= 1e-13, (i, k, got[i, k], ref)


@pytest.mark.parametrize("kind,p_max", CASES)
def test_lnl_and_lnz_match_oracle(R, kind, p_max):
    point, exact, info, draws, logw = fixture(kind, p_max)
    cp = R.CompPoint(point)
    d = R.Draws(draws, logw)
    got = R.rift_ile_comp_lnL(cp, d).cpu().numpy()
    ref = OC.lnL(OC.CompPoint(point), draws)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-9
    z = R.rift_ile_comp_lnZ(cp, d)
    zr = O.lnZ(ref, logw)
    assert abs(z[0] - zr[0]) <= 1e-9 * max(1.0, abs(zr[0]))
    assert abs(z[2] - zr[2]) <= 1e-7 * zr[2]
    st = R.rift_ile_comp_lnZ_state_async(cp, d).cpu().numpy()
    assert np.array_equal(st, np.array(R.rift_ile_comp_lnZ_state(cp, d)))


@pytest.mark.parametrize("n", [1, 127, 129, 1000])
def test_ragged_counts_and_float32_draws(R, n):
    point, exact, info, draws, logw = fixture(WC.ROTATION, 1)
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    cp = R.CompPoint(point)
    ref = OC.lnL(OC.CompPoint(point), sub)
    got = R.rift_ile_comp_lnL(cp, R.Draws(sub)).cpu().numpy()
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-9
    # float32 draws are promoted exactly: compare with the oracle on the rounded values
    sub32 = {p: np.asarray(sub[p], dtype=np.float32) for p in W.PARAMS}
    ref32 = OC.lnL(OC.CompPoint(point), {p: sub32[p].astype(np.float64) for p in W.PARAMS})
    got32 = R.rift_ile_comp_lnL(cp, R.Draws(sub32)).cpu().numpy()
    assert np.max(np.abs(got32 - ref32) / np.maximum(1.0, np.abs(ref32))) <= 1e-9


@pytest.mark.parametrize("p_max,tol", [(0, 1e-10), (2, 1e-8)])
def test_omega_zero_is_static_gpu(R, p_max, tol):
    """At Omega = 0 the five harmonics sum to F_k and every p >= 1 term sums
    to zero; those terms are each ~(2 pi f |dt|)^p larger than their sum, so
    p_max = 2 agrees only to that amplification of the FP64 rounding."""
    point, exact, info, draws, logw = WC.comp_small(WC.ROTATION, p_max, n_draws=1024, omega=0.0)
    M = int(point["M"])
    sl = slice(2 * M, 3 * M)   # (p, n) = (0, 0)
    static = {"K": point["K"], "M": M, "ell": point["ell"], "em": point["em"],
              "Q": np.ascontiguousarray(point["Q"][:, :, sl]), "q_t0": point["q_t0"],
              "q_dt": point["q_dt"], "U": point["U"][:, sl, sl], "V": point["V"][:, sl, sl],
              "det_pos": point["det_pos"], "det_resp": point["det_resp"],
              "gmst": point["gmst"], "d_ref": point["d_ref"]}
    d = R.Draws(draws, logw)
    comp = R.rift_ile_comp_lnL(R.CompPoint(point), d).cpu().numpy()
    ref = R.rift_ile_lnL(R.Point(static), d, R.FP64).cpu().numpy()
    assert np.max(np.abs(comp - ref) / np.maximum(1.0, np.abs(ref))) <= tol


def test_out_of_table_taps_and_empty(R):
    point, exact, info, draws, logw = fixture(WC.FINITE_ARM, 3)
    cp = R.CompPoint(point)
    far = {p: np.asarray(draws[p])[:64].copy() for p in W.PARAMS}
    far["t"] = far["t"] + np.linspace(-0.05, 0.05, 64)   # beyond the +-25 ms tables
    got = R.rift_ile_comp_lnL(cp, R.Draws(far)).cpu().numpy()
    ref, td, tq, oob = OC.lnL(OC.CompPoint(point), far, terms=True)
    assert oob > 0
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-9
    R.rift_ile_comp_lnZ_state(cp, R.Draws(far))
    assert R.rift_ile_last_oob() == oob
    empty = {p: np.zeros(0) for p in W.PARAMS}
    st = R.rift_ile_comp_lnZ_state(cp, R.Draws(empty))
    assert st[0] == -math.inf and st[1] == 0.0 and st[3] == 0.0


def test_rejects_unsupported(R):
    point, exact, info, draws, logw = fixture(WC.ROTATION, 0)
    bad = dict(point)
    bad["p_max"] = 4
    with pytest.raises(R.RiftError):
        R.CompPoint(bad)


@pytest.fixture(scope="module")
def big():
    return WC.comp_3g(WC.ROTATION, 0, n_draws=1 << 22)


def test_full_size_path_a_sampled(R, big):
    """3G network, ten modes, Path A, 2^22 float32 draws in one launch (the
    bench's configuration): 512 sampled draws against the oracle, and the
    fused lnZ against the LSE of the per-draw output."""
    point, exact, info, draws, logw = big
    cp = R.CompPoint(point)
    d = R.Draws(draws, logw)
    lnl = R.rift_ile_comp_lnL(cp, d)
    idx = np.concatenate([torch.topk(lnl, 256).indices.cpu().numpy(),
                          np.arange(0, d.n, d.n // 256)])
    sub = {p: np.asarray(draws[p])[idx].astype(np.float64) for p in W.PARAMS}
    ref = OC.lnL(OC.CompPoint(point), sub)
    got = lnl.cpu().numpy()[idx]
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-9
    z = R.rift_ile_comp_lnZ(cp, d)
    lw = torch.as_tensor(np.asarray(logw, dtype=np.float64), device="cuda")
    v = lnl + lw
    m = v.max()
    ref_z = float(m + torch.log(torch.exp(v - m).sum()) - math.log(d.n))
    assert abs(z[0] - ref_z) <= 1e-9 * abs(ref_z)


@pytest.mark.parametrize("kind,p_max", CASES)
def test_gradient_matches_oracle(R, kind, p_max):
    """The adjoint (closed-form coefficient derivatives) against the oracle's
    chain rule (coefficient derivatives by central differences), per
    component relative to |g| + RMS g over the draws."""
    point, exact, info, draws, logw = fixture(kind, p_max)
    n = 160
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    cp = R.CompPoint(point)
    lnl, g = R.rift_ile_comp_lnL_grad(cp, R.Draws(sub))
    lnl, g = lnl.cpu().numpy(), g.cpu().numpy()
    fwd = R.rift_ile_comp_lnL(cp, R.Draws(sub)).cpu().numpy()
    assert np.max(np.abs(lnl - fwd) / np.maximum(1.0, np.abs(fwd))) <= 1e-9
    ref_l, ref_g = OC.lnL_grad(OC.CompPoint(point), sub)
    assert np.max(np.abs(lnl - ref_l) / np.maximum(1.0, np.abs(ref_l))) <= 1e-9
    for j, p in enumerate(W.PARAMS):
        s = np.abs(ref_g[:, j]) + np.sqrt(np.mean(ref_g[:, j] ** 2))
        assert np.max(np.abs(g[j] - ref_g[:, j]) / s) <= 1e-8, (p, np.max(np.abs(g[j] - ref_g[:, j]) / s))


def test_autograd_on_composite_point(R):
    """torch.autograd through the composite adjoint: backward equals the C-ABI
    gradient times grad_output, and gradcheck passes in FP64."""
    point, exact, info, draws, logw = fixture(WC.ROTATION, 1)
    cp = R.CompPoint(point)
    n = 64
    th = [torch.tensor(np.asarray(draws[p])[:n], dtype=torch.float64, device="cuda",
                       requires_grad=True) for p in W.PARAMS]
    lnl = R.lnL(cp, *th)
    wts = torch.linspace(-1.0, 2.0, n, dtype=torch.float64, device="cuda")
    (lnl * wts).sum().backward()
    ref_l, ref_g = R.rift_ile_comp_lnL_grad(cp, R.Draws({p: np.asarray(draws[p])[:n] for p in W.PARAMS}))
    assert torch.equal(lnl.detach(), ref_l)
    for j in range(7):
        assert torch.equal(th[j].grad, ref_g[j] * wts)
    # gradcheck on Path A (no cancelling p >= 1 terms to amplify FP64 rounding)
    point0, _, _, draws0, _ = fixture(WC.ROTATION, 0)
    cp0 = R.CompPoint(point0)
    small = tuple(torch.tensor(np.asarray(draws0[p])[:4], dtype=torch.float64, device="cuda",
                               requires_grad=True) for p in W.PARAMS)

    def f(ra, dec, psi, incl, phase, lnD, tau):
        return R.lnL(cp0, ra, dec, psi, incl, phase, lnD, tau * 1e-4)

    small = small[:6] + (small[6].detach().mul(1e4).requires_grad_(),)
    assert torch.autograd.gradcheck(f, small, eps=1e-6, atol=1e-3, rtol=1e-4, nondet_tol=0.0)


def test_sharded_lnz_merges_to_the_whole(R):
    """Draws split into shards (as ranks would hold them) give LSE states whose
    host merge equals the state of all draws at once (the one exchange of the
    sharded path)."""
    point, exact, info, draws, logw = fixture(WC.ROTATION, 1)
    cp = R.CompPoint(point)
    whole = R.rift_ile_comp_lnZ_state(cp, R.Draws(draws, logw))
    n = len(draws["ra"])
    states = []
    for r in range(3):
        lo, hi = R.shard_bounds(n, r, 3)
        sub = {p: np.asarray(draws[p])[lo:hi] for p in W.PARAMS}
        states.append(R.rift_ile_comp_lnZ_state(cp, R.Draws(sub, np.asarray(logw)[lo:hi])))
    merged, mstate = R.rift_ile_lnZ_merge(states)
    ref = R.rift_ile_lnZ_merge([whole])[0]
    assert abs(merged[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert abs(merged[2] - ref[2]) <= 1e-10 * ref[2]
    assert mstate[3] == n


def _three_detector_point(kind, p_max, lengths):
    import math as _m
    rng = np.random.default_rng(WC.seed_for(30 + kind, 0))
    gmst = rng.uniform(0, 2 * _m.pi)
    truth = WC._truth(rng)
    dets = [WC.random_detectors_arms(rng, 1, L)[0] for L in lengths]
    point, exact, info = WC.make_comp_point(
        kind=kind, p_max=p_max, dets=dets, modes=WC.MODES4, f_low=20.0,
        f_max=1024.0 if kind == WC.ROTATION else 2048.0, df=0.25, rate=8192.0,
        half_window=0.025, snr=20.0, truth=truth, gmst=gmst, d_ref=W.D_REF, rng=rng, omega=2.0)
    sig = W.proposal_sigma(info, exact)
    draws, logw = W.mixture_draws(np.random.default_rng(WC.seed_for(30 + kind, 1)),
                                  W.Prior(0.5 * W.D_REF, 2.0 * W.D_REF, 0.01), truth, sig, 96)
    return point, W.as_float(draws, np.float64)


@pytest.mark.parametrize("kind,p_max,lengths", [
    (WC.ROTATION, 3, (4e3, 4e3, 4e3)),           # 3 x 32 response indices: per-detector forms
    (WC.FINITE_ARM, 3, (1e4, 1e4, 4e4)),         # two detector classes share forms
])
def test_detector_classes_and_per_detector_path(R, kind, p_max, lengths):
    point, draws = _three_detector_point(kind, p_max, lengths)
    cp = R.CompPoint(point)
    l, g = R.rift_ile_comp_lnL_grad(cp, R.Draws(draws))
    fwd = R.rift_ile_comp_lnL(cp, R.Draws(draws)).cpu().numpy()
    ref_l, ref_g = OC.lnL_grad(OC.CompPoint(point), draws)
    tol = 1e-8 if p_max >= 2 and kind == WC.ROTATION else 1e-9
    assert np.max(np.abs(fwd - ref_l) / np.maximum(1.0, np.abs(ref_l))) <= tol
    assert np.max(np.abs(l.cpu().numpy() - ref_l) / np.maximum(1.0, np.abs(ref_l))) <= tol
    g = g.cpu().numpy()
    for j, p in enumerate(W.PARAMS):
        s = np.abs(ref_g[:, j]) + np.sqrt(np.mean(ref_g[:, j] ** 2))
        assert np.max(np.abs(g[j] - ref_g[:, j]) / s) <= 1e-7, p


def test_graph_capture_of_the_fused_step(R):
    """The asynchronous composite lnZ step (fused kernel + merge, no host
    synchronisation) can be captured in a CUDA graph and replayed, with the
    result equal bit for bit to the eager step."""
    point, exact, info, draws, logw = fixture(WC.ROTATION, 0)
    cp = R.CompPoint(point)
    d = R.Draws(draws, logw)
    eager = R.rift_ile_comp_lnZ_state_async(cp, d).clone()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s2):
        R.rift_ile_comp_lnZ_state_async(cp, d, out=out)
    torch.cuda.current_stream().wait_stream(s2)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        R.rift_ile_comp_lnZ_state_async(cp, d, out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
