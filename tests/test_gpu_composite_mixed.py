"""FP32-mixed composite-index response (Sec. III, eq. slowrot:lnL:Decomposed in
whitened coordinates; rift_ile_comp_mixed_build and the *_mixed entry points)
against the composite oracle:

* lnL per draw within a per-case tolerance of the oracle for the draws within
  50 nat of the best (the ones that carry the evidence), and within
  TOL_FAR + 1e-5 |lnL| for every draw, for rotation Paths A and B and finite
  arms (Path D), and lnZ within TOL_Z.  The mixed kernels read the angles as
  float32 (as the static mixed path does), so the draws are rounded to float32
  and the oracle evaluates the rounded values.  The rotation fixtures use a
  stress sidereal rate (2 rad/s) at which the p >= 1 terms of the expansion
  are much larger than their sum: Path B there is held to 1e-3 nat; at
  p_max = 3 the expansion's terms exceed the likelihood by ~1e5 and the
  dropped eigen-directions carry that much, so the whitened form does not
  apply (the FP64 path covers it);
* the width the build keeps shrinks as tol grows, and a rebuild replaces the
  tables;
* ragged draw counts, float32 draws, out-of-table taps (counted as the FP64
  path counts them), a non-finite arrival time (NaN), the empty draw set;
* the adjoint (rift_ile_comp_lnL_grad_mixed): lnL as the forward gives it, and
  each gradient component against the oracle's chain rule within TOL_G of
  |g| + RMS g (the terms that multiply the residual are FP32); NaN rows for a
  non-finite arrival time; the empty draw set;
* calls before the build, and tol outside (0, 1), are errors;
* on the 3G network at full size (2^22 draws, the bench's launch), sampled
  draws against the oracle and the fused lnZ against the FP64 path's; the
  adjoint of Paths A, B and D against the FP64 adjoint; torch.autograd
  through a CompPoint switching to the mixed form once it is built.
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

TOL_NEAR = 1e-4   # nat, draws within 50 nat of the best
TOL_FAR = 1e-3    # nat, plus 1e-5 |lnL|, every draw
TOL_Z = 1e-5      # nat
EIG_TOL = 1e-14
# (near, far) for the stress-rate Path B fixture
TOL_CASE = {(WC.ROTATION, 1): (1e-3, 1e-2)}
TOL_G = 1e-4     # gradient, relative to |g| + RMS g over the draws


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


CASES = [(WC.ROTATION, 0), (WC.ROTATION, 1), (WC.FINITE_ARM, 0), (WC.FINITE_ARM, 3),
         (WC.FINITE_ARM, 6)]
_cache = {}


def rounded(draws):
    """The draws as the mixed kernels see them: float32 values, as float64."""
    return {p: np.asarray(draws[p], dtype=np.float32).astype(np.float64) for p in W.PARAMS}


def fixture(kind, p_max, n_draws=1500):
    key = (kind, p_max, n_draws)
    if key not in _cache:
        point, exact, info, draws, logw = WC.comp_small(kind, p_max, n_draws=n_draws)
        draws = rounded(draws)
        ref = OC.lnL(OC.CompPoint(point), draws)
        _cache[key] = (point, draws, logw, ref)
    return _cache[key]


def check_close(got, ref, tol_near=TOL_NEAR, tol_far=TOL_FAR):
    near = ref > np.max(ref) - 50.0
    err = np.abs(got - ref)
    assert np.max(err[near]) <= tol_near, np.max(err[near])
    assert np.all(err <= tol_far + 1e-5 * np.abs(ref)), np.max(err - 1e-5 * np.abs(ref))


@pytest.mark.parametrize("kind,p_max", CASES)
def test_mixed_lnl_and_lnz_match_oracle(R, kind, p_max):
    point, draws, logw, ref = fixture(kind, p_max)
    cp = R.CompPoint(point)
    info = R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    assert info[0] >= info[1] >= 1 and info[0] % 2 == 0 and info[3] in (32, 64, 128)
    d = R.Draws(draws, logw)
    got = R.rift_ile_comp_lnL_mixed(cp, d).cpu().numpy()
    check_close(got, ref, *TOL_CASE.get((kind, p_max), (TOL_NEAR, TOL_FAR)))
    z = R.rift_ile_comp_lnZ_mixed(cp, d)
    zr = O.lnZ(ref, logw)
    assert abs(z[0] - zr[0]) <= TOL_Z
    assert abs(z[2] - zr[2]) <= 1e-3 * zr[2]
    st = R.rift_ile_comp_lnZ_state_mixed_async(cp, d).cpu().numpy()
    assert np.array_equal(st, np.array(R.rift_ile_comp_lnZ_state_mixed(cp, d)))


@pytest.mark.parametrize("kind,p_max", CASES)
def test_mixed_gradient_matches_oracle(R, kind, p_max):
    point, draws, logw, ref = fixture(kind, p_max)
    n = 160
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    lnl, g = R.rift_ile_comp_lnL_grad_mixed(cp, R.Draws(sub))
    lnl, g = lnl.cpu().numpy(), g.cpu().numpy()
    fwd = R.rift_ile_comp_lnL_mixed(cp, R.Draws(sub)).cpu().numpy()
    assert np.max(np.abs(lnl - fwd)) <= 1e-12 * np.max(np.abs(fwd))
    ref_l, ref_g = OC.lnL_grad(OC.CompPoint(point), sub)
    for j, p in enumerate(W.PARAMS):
        s = np.abs(ref_g[:, j]) + np.sqrt(np.mean(ref_g[:, j] ** 2))
        err = np.max(np.abs(g[j] - ref_g[:, j]) / s)
        assert err <= TOL_G, (p, err)


def test_autograd_uses_the_mixed_form_once_built(R):
    """torch.autograd through a CompPoint: FP64 until the mixed form is built,
    then (precision FP32_MIXED) the mixed adjoint, bit for bit; FP64 asked for
    explicitly stays FP64."""
    point, draws, logw, ref = fixture(WC.ROTATION, 0)
    cp = R.CompPoint(point)
    n = 48
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    wts = torch.linspace(-1.0, 2.0, n, dtype=torch.float64, device="cuda")

    def grads(precision):
        th = [torch.tensor(sub[p], dtype=torch.float64, device="cuda", requires_grad=True)
              for p in W.PARAMS]
        lnl = R.lnL(cp, *th, precision=precision)
        (lnl * wts).sum().backward()
        return lnl.detach(), [t.grad for t in th]

    l64, g64 = grads(R.FP32_MIXED)
    rl, rg = R.rift_ile_comp_lnL_grad(cp, R.Draws(sub))
    assert torch.equal(l64, rl) and all(torch.equal(g64[j], rg[j] * wts) for j in range(7))
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    lm, gm = grads(R.FP32_MIXED)
    rl, rg = R.rift_ile_comp_lnL_grad_mixed(cp, R.Draws(sub))
    assert torch.equal(lm, rl) and all(torch.equal(gm[j], rg[j] * wts) for j in range(7))
    lf, gf = grads(R.FP64)
    assert torch.equal(lf, l64)


def test_mixed_gradient_nonfinite_empty_and_errors(R):
    point, draws, logw, ref = fixture(WC.FINITE_ARM, 3)
    cp = R.CompPoint(point)
    bad = {p: np.asarray(draws[p])[:8].copy() for p in W.PARAMS}
    bad["t"][3] = np.nan
    with pytest.raises(R.RiftError):
        R.rift_ile_comp_lnL_grad_mixed(cp, R.Draws(bad))
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    lnl, g = R.rift_ile_comp_lnL_grad_mixed(cp, R.Draws(bad))
    lnl, g = lnl.cpu().numpy(), g.cpu().numpy()
    assert np.isnan(lnl[3]) and np.all(np.isnan(g[:, 3]))
    assert np.all(np.isfinite(np.delete(lnl, 3))) and np.all(np.isfinite(np.delete(g, 3, axis=1)))
    empty = {p: np.zeros(0) for p in W.PARAMS}
    lnl, g = R.rift_ile_comp_lnL_grad_mixed(cp, R.Draws(empty))
    assert lnl.numel() == 0 and tuple(g.shape) == (7, 0)


def test_width_follows_tol_and_rebuild(R):
    point, draws, logw, ref = fixture(WC.ROTATION, 1)
    cp = R.CompPoint(point)
    assert R.rift_ile_comp_mixed_info(cp) == (0, 0, 0, 0)
    wide = R.rift_ile_comp_mixed_build(cp, 1e-15)
    narrow = R.rift_ile_comp_mixed_build(cp, 1e-6)
    assert narrow[1] < wide[1]
    assert R.rift_ile_comp_mixed_info(cp) == narrow
    d = R.Draws(draws, logw)
    coarse = R.rift_ile_comp_lnL_mixed(cp, d).cpu().numpy()
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    fine = R.rift_ile_comp_lnL_mixed(cp, d).cpu().numpy()
    check_close(fine, ref, *TOL_CASE[(WC.ROTATION, 1)])
    # what the coarse whitening drops is visible at the peak
    near = ref > np.max(ref) - 50.0
    assert np.max(np.abs(coarse - ref)[near]) > np.max(np.abs(fine - ref)[near])


def test_errors_before_build_and_bad_tol(R):
    point, draws, logw, ref = fixture(WC.ROTATION, 0)
    cp = R.CompPoint(point)
    d = R.Draws(draws, logw)
    with pytest.raises(R.RiftError):
        R.rift_ile_comp_lnL_mixed(cp, d)
    with pytest.raises(R.RiftError):
        R.rift_ile_comp_lnZ_state_mixed(cp, d)
    for tol in (0.0, 1.0, -1e-3, float("nan")):
        with pytest.raises(R.RiftError):
            R.rift_ile_comp_mixed_build(cp, tol)
    assert R.rift_ile_comp_mixed_info(cp) == (0, 0, 0, 0)


@pytest.mark.parametrize("n", [1, 127, 129, 1000])
def test_ragged_counts_and_float32_draws(R, n):
    """Ragged counts, with the draws passed as float64 and as float32 (the
    same values): the two calls agree bit for bit and match the oracle."""
    point, draws, logw, ref = fixture(WC.ROTATION, 0)
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    got = R.rift_ile_comp_lnL_mixed(cp, R.Draws(sub)).cpu().numpy()
    sub32 = {p: np.asarray(sub[p], dtype=np.float32) for p in W.PARAMS}
    got32 = R.rift_ile_comp_lnL_mixed(cp, R.Draws(sub32)).cpu().numpy()
    assert np.array_equal(got, got32)
    err = np.abs(got - ref[:n])
    assert np.all(err <= TOL_FAR + 1e-5 * np.abs(ref[:n]))
    near = ref[:n] > np.max(ref) - 50.0
    if near.any():
        assert np.max(err[near]) <= TOL_NEAR


def test_out_of_table_nonfinite_and_empty(R):
    point, draws, logw, ref = fixture(WC.FINITE_ARM, 3)
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    far = {p: np.asarray(draws[p])[:64].copy() for p in W.PARAMS}
    far["t"] = far["t"] + np.linspace(-0.05, 0.05, 64)   # beyond the +-25 ms tables
    got = R.rift_ile_comp_lnL_mixed(cp, R.Draws(far)).cpu().numpy()
    ref_far, td, tq, oob = OC.lnL(OC.CompPoint(point), far, terms=True)
    assert oob > 0
    assert np.all(np.abs(got - ref_far) <= TOL_FAR + 1e-5 * np.abs(ref_far))
    R.rift_ile_comp_lnZ_state_mixed(cp, R.Draws(far))
    assert R.rift_ile_last_oob() == oob
    bad = {p: np.asarray(draws[p])[:8].copy() for p in W.PARAMS}
    bad["t"][3] = np.inf
    got = R.rift_ile_comp_lnL_mixed(cp, R.Draws(bad)).cpu().numpy()
    assert np.isnan(got[3]) and np.all(np.isfinite(np.delete(got, 3)))
    empty = {p: np.zeros(0) for p in W.PARAMS}
    st = R.rift_ile_comp_lnZ_state_mixed(cp, R.Draws(empty))
    assert st[0] == -math.inf and st[1] == 0.0 and st[3] == 0.0
    assert R.rift_ile_comp_lnL_mixed(cp, R.Draws(empty)).numel() == 0


@pytest.fixture(scope="module")
def big():
    return WC.comp_3g(WC.ROTATION, 0, n_draws=1 << 22)


def test_full_size_path_a_sampled(R, big):
    """3G network, ten modes, Path A, 2^22 float32 draws in one launch (the
    bench's configuration): the 256 best and 256 strided draws against the
    oracle, and the fused lnZ against the FP64 path's."""
    point, exact, info, draws, logw = big   # float32 draws
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    d = R.Draws(draws, logw)
    lnl = R.rift_ile_comp_lnL_mixed(cp, d)
    idx = np.concatenate([torch.topk(lnl, 256).indices.cpu().numpy(),
                          np.arange(0, d.n, d.n // 256)])
    sub = {p: np.asarray(draws[p])[idx].astype(np.float64) for p in W.PARAMS}
    ref = OC.lnL(OC.CompPoint(point), sub)
    got = lnl.cpu().numpy()[idx]
    err = np.abs(got - ref)
    assert np.max(err[:256]) <= TOL_NEAR, np.max(err[:256])
    assert np.all(err <= TOL_FAR + 1e-5 * np.abs(ref)), np.max(err - 1e-5 * np.abs(ref))
    zm = R.rift_ile_comp_lnZ_mixed(cp, d)
    zf = R.rift_ile_comp_lnZ(cp, d)
    assert abs(zm[0] - zf[0]) <= TOL_Z


def test_full_size_path_a_gradient_vs_fp64(R, big):
    """3G network, ten modes, Path A: the adjoint of the first 2^20 draws
    against the FP64 adjoint (itself pinned to the oracle), every component
    within TOL_G of |g| + RMS g for the draws within 50 nat of the best."""
    point, exact, info, draws, logw = big
    n = 1 << 20
    sub = {p: np.asarray(draws[p])[:n] for p in W.PARAMS}
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    d = R.Draws(sub)
    lm, gm = R.rift_ile_comp_lnL_grad_mixed(cp, d)
    lf, gf = R.rift_ile_comp_lnL_grad(cp, d)
    near = lf > lf.max() - 50.0
    assert int(near.sum()) > 100
    for j, p in enumerate(W.PARAMS):
        s = gf[j].abs() + gf[j][near].pow(2).mean().sqrt()
        err = float(((gm[j] - gf[j]).abs() / s)[near].max())
        assert err <= TOL_G, (p, err)


@pytest.mark.parametrize("kind,p_max", [(WC.ROTATION, 1), (WC.FINITE_ARM, 3)])
def test_full_size_paths_b_and_d_gradient_vs_fp64(R, kind, p_max):
    """3G network, Paths B and D, 2^18 float32 draws: the mixed adjoint
    against the FP64 adjoint within TOL_G of |g| + RMS g within 50 nat."""
    point, exact, info, draws, logw = WC.comp_3g(kind, p_max, n_draws=1 << 18)
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    d = R.Draws(draws)
    lm, gm = R.rift_ile_comp_lnL_grad_mixed(cp, d)
    lf, gf = R.rift_ile_comp_lnL_grad(cp, d)
    near = lf > lf.max() - 50.0
    assert int(near.sum()) > 100
    for j, p in enumerate(W.PARAMS):
        s = gf[j].abs() + gf[j][near].pow(2).mean().sqrt()
        err = float(((gm[j] - gf[j]).abs() / s)[near].max())
        assert err <= TOL_G, (p, err)


@pytest.mark.parametrize("kind,p_max,tol_near", [(WC.ROTATION, 1, 5e-4), (WC.FINITE_ARM, 3, 1e-4)])
def test_full_size_paths_b_and_d_vs_fp64(R, kind, p_max, tol_near):
    """3G network, Path B (p_max 1) and Path D (p_max 3), 2^20 float32 draws:
    every draw within 50 nat of the best against the FP64 path (itself pinned
    to the oracle), and the fused lnZ."""
    point, exact, info, draws, logw = WC.comp_3g(kind, p_max, n_draws=1 << 20)
    cp = R.CompPoint(point)
    R.rift_ile_comp_mixed_build(cp, EIG_TOL)
    d = R.Draws(draws, logw)
    lm = R.rift_ile_comp_lnL_mixed(cp, d)
    lf = R.rift_ile_comp_lnL(cp, d)
    near = lf > lf.max() - 50.0
    assert int(near.sum()) > 1000
    assert float((lm - lf).abs()[near].max()) <= tol_near
    assert abs(R.rift_ile_comp_lnZ_mixed(cp, d)[0] - R.rift_ile_comp_lnZ(cp, d)[0]) <= TOL_Z
