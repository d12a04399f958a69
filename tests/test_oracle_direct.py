"""Pins of the direct-marginalisation oracle (ERAI over (phi, psi), adaptive
Gauss-Hermite in distance), against things other than itself:

* the reconstructed harmonic model equals the static oracle's data and norm
  terms at off-grid (phi, psi) (eq. ap:angleharm is exact at fixed time);
* the Gauss-Hermite distance integral equals adaptive quadrature of the same
  integrand over the prior range when the peak is inside it;
* the marginal equals a brute-force quadrature (static oracle on a fine
  (phi, psi) grid, distance by adaptive quadrature) on the two-detector
  workload, and changes little when the angle grid is refined;
* planted mistakes (a too-small phase grid, a lost sqrt(2), the wrong
  distance prior power) each fail one of these;
* the band-limited time rule (eq. ap:tband): its sinc reconstruction of the
  data coefficients converges to the coefficients evaluated at the fine
  times as the window widens, the rule agrees with the fixed-spacing rule
  evaluated directly on the same fine nodes, and fine nodes misplaced by half
  an interval are caught.
"""
import importlib.util
import math
import os
import sys
import tempfile

import numpy as np
import pytest
import scipy.integrate

import oracle as O
import oracle.direct as OD
import workload as W

FIX = W.config0(n_draws=8)


def _truth_like(info, k=0):
    tr = dict(info["truth"])
    return tr


def _general_point():
    """The two-detector point with a generic symmetric V added, so that the
    model norm carries phase harmonics up to 2 m_max (as a precessing source's
    would); the reconstruction must still be exact."""
    point, exact, info, draws, logw = FIX
    p = dict(point)
    rng = np.random.default_rng(3)
    M = int(p["M"])
    E = rng.normal(size=(p["K"], M, M)) + 1j * rng.normal(size=(p["K"], M, M))
    p["V"] = np.asarray(p["V"]) + 0.1 * np.max(np.abs(p["U"])) * (E + np.transpose(E, (0, 2, 1)))
    return p


GENERAL = _general_point()


def _battery(mod):
    fails = []
    _, exact, info, draws, logw = FIX
    point = GENERAL
    pt = O.OraclePoint(point)
    tr = info["truth"]
    cK, cR, _ = mod.reconstruct(pt, point, tr["ra"], tr["dec"], tr["incl"], tr["t"])
    rng = np.random.default_rng(1)
    ps, ph = rng.uniform(0, np.pi, 6), rng.uniform(0, 2 * np.pi, 6)
    th = {"ra": np.full(6, tr["ra"]), "dec": np.full(6, tr["dec"]), "psi": ps,
          "incl": np.full(6, tr["incl"]), "phase": ph, "lnD": np.full(6, math.log(point["d_ref"])),
          "t": np.full(6, tr["t"])}
    _, Td, Tq, _ = O.lnL(pt, th, terms=True, threads=1)
    if (np.max(np.abs(mod.evaluate(cK, ps, ph) - Td)) > 1e-9 * np.max(np.abs(Td))
            or np.max(np.abs(mod.evaluate(cR, ps, ph) - 2 * Tq)) > 1e-9 * np.max(np.abs(Tq))):
        fails.append("reconstruction")
    # Gauss-Hermite against quadrature: peak well inside [d_ref/d_max, d_ref/d_min]
    d_ref, d_min, d_max = 100.0, 50.0, 200.0
    for K, R in ((400.0, 400.0), (300.0, 350.0), (150.0, 125.0)):
        lo, hi = d_ref / d_max, d_ref / d_min
        norm = 3.0 * d_ref ** 3 / (d_max ** 3 - d_min ** 3)
        peak = K * K / (2 * R)
        val, _ = scipy.integrate.quad(lambda x: norm * x ** -4 * math.exp(K * x - 0.5 * R * x * x - peak),
                                      lo, hi, epsabs=0, epsrel=1e-13, limit=200)
        got = mod.distance_gh(np.array(K), np.array(R), d_ref, d_min, d_max, 40)
        if abs(float(got) - (peak + math.log(val))) > 1e-7:
            fails.append("gauss_hermite")
            break
    return fails


def test_unmodified_passes_battery():
    assert _battery(OD) == []


def test_marginal_against_brute_force():
    point, exact, info, draws, logw = FIX
    pt = O.OraclePoint(point)
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    d["ra"] = d["ra"] + 0.01
    n_phi, n_psi = 48, 24
    got = OD.lnL_direct(point, d, n_phi, n_psi, 40, 50.0, 200.0)[0]
    # the angle grid resolves the peak (width ~1/(2 rho) in phase at SNR 20)
    coarse = OD.lnL_direct(point, d, 256, 128, 40, 50.0, 200.0)[0]
    finer = OD.lnL_direct(point, d, 512, 256, 40, 50.0, 200.0)[0]
    # brute force: static oracle on the grid, distance by adaptive quadrature
    psis = np.pi * np.arange(n_psi) / n_psi
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    K, R = OD._terms_on_grid(pt, point["d_ref"], d["ra"][0], d["dec"][0], d["incl"][0],
                             d["t"][0], phis, psis)
    lo, hi = point["d_ref"] / 200.0, point["d_ref"] / 50.0
    norm = 3.0 * point["d_ref"] ** 3 / (200.0 ** 3 - 50.0 ** 3)
    vals = []
    ref = float(np.max(K * K / (2 * R)))
    for k_, r_ in zip(K.ravel(), R.ravel()):
        v, _ = scipy.integrate.quad(lambda x: norm * x ** -4 * math.exp(k_ * x - 0.5 * r_ * x * x - ref),
                                    lo, hi, epsabs=0, epsrel=1e-12, limit=200)
        vals.append(v)
    brute = ref + math.log(np.mean(vals))
    assert abs(got - brute) <= 1e-6, (got, brute)
    assert abs(finer - coarse) <= 1e-6, (finer, coarse)


SRC = os.path.join(os.path.dirname(OD.__file__), "direct.py")
MUTATIONS = {
    "nyquist_too_small": ("n_psi, n_phi = 5, 4 * m_max + 1", "n_psi, n_phi = 5, 2 * m_max + 1"),
    "gh_no_sqrt2": ("x = xs[..., None] + math.sqrt(2.0) * sig[..., None] * xi",
                    "x = xs[..., None] + sig[..., None] * xi"),
    "prior_power": ("norm * np.abs(x) ** -4.0", "norm * np.abs(x) ** -2.0"),
    "norm_scale": ("np.fft.fft2(R) / R.size", "np.fft.fft2(R) / K.shape[0]"),
}


def _load(text, tag):
    d = tempfile.mkdtemp()
    path = os.path.join(d, f"direct_{tag}.py")
    with open(path, "w") as f:
        f.write(text)
    spec = importlib.util.spec_from_file_location(f"oracle._direct_{tag}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1
    assert _battery(_load(text.replace(old, new), name)), name


def test_time_rule_converges_and_reduces():
    """The time-marginalised value converges as the node count doubles, and a
    single node reproduces the fixed-time value at that node."""
    point, exact, info, draws, logw = FIX
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    fixed = OD.lnL_direct(point, d, 64, 32, 24, 50.0, 200.0)[0]
    one = OD.lnL_direct(point, d, 64, 32, 24, 50.0, 200.0, 1, tr["t"] - 1e-4, tr["t"] + 1e-4)[0]
    assert abs(one - fixed) <= 1e-12 * abs(fixed)
    # SNR 20: sigma_t ~ 1/(2 pi rho sigma_f) ~ 1e-4 s; a +-1 ms window
    vals = [OD.lnL_direct(point, d, 64, 32, 24, 50.0, 200.0, n, tr["t"] - 1e-3, tr["t"] + 1e-3)[0]
            for n in (40, 80, 160)]
    # the table cubic is only C^1-piecewise in t, so the rule converges
    # algebraically: each doubling cuts the change by more than 4
    d1, d2 = abs(vals[1] - vals[0]), abs(vals[2] - vals[1])
    assert d2 <= 0.25 * d1 and d2 <= 5e-4, vals


def _fine_table_point():
    """Noise-free two-detector point whose Q table is sampled at 16 384 Hz
    (band limit 512 Hz), so that the table cubic is exact to ~1e-5 and the
    data coefficients reconstructed at any time stand in for the band-limited
    correlation itself."""
    rng = np.random.default_rng(41)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:4], f_low=20.0, f_max=512.0, df=0.5, rate=16384.0,
        half_window=0.03, snr=20.0, truth=truth, gmst=0.4, d_ref=100.0, rng=rng, noise=False,
        q_dtype=np.complex128)
    return point, info


def _tband_error(mod, half):
    """Largest error, relative to the largest coefficient, of the sinc
    reconstruction (coarse spacing h = 1/2048 s, 4 fine nodes per interval)
    against the directly reconstructed data coefficients at the fine nodes of
    the two central coarse intervals, for a window of `half` coarse samples on
    each side of the peak."""
    point, info = _fine_table_point()
    pt = O.OraclePoint(point)
    tr = info["truth"]
    h, M = 1.0 / 2048, 4
    t_lo = tr["t"] - half * h
    times = t_lo + (np.arange(2 * half) + 0.5) * h
    cK = np.stack([mod.reconstruct(pt, point, tr["ra"], tr["dec"], tr["incl"], t)[0]
                   for t in times])
    up = mod.sinc_upsample(cK, M)
    mid = np.arange(half * M - 2 * M, half * M + 2 * M)
    direct = np.stack([mod.reconstruct(pt, point, tr["ra"], tr["dec"], tr["incl"],
                                       t_lo + (f + 0.5) * h / M)[0] for f in mid])
    return np.max(np.abs(up[mid] - direct)) / np.max(np.abs(direct))


def test_band_limited_reconstruction_converges_to_the_correlation():
    """eq. ap:tband: the sinc-interpolated data coefficients approach the
    correlation evaluated at the fine times as the window widens (the
    truncated stencil is the only error: the coefficients are linear in the
    band-limited Q); at t_up = 1 the upsampling is the identity."""
    errs = [_tband_error(OD, half) for half in (8, 16, 32)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= 1e-4, errs
    x = np.random.default_rng(2).normal(size=(7, 3))
    assert np.max(np.abs(OD.sinc_upsample(x, 1) - x)) <= 1e-15


def test_band_limited_rule_matches_the_fine_fixed_rule():
    """With the peak well inside the window, the band-limited rule on n_t
    coarse nodes x t_up equals the fixed-spacing rule evaluated directly at
    the same n_t t_up fine nodes (same weights), up to the reconstruction
    error; t_up = 1 is the fixed-spacing rule itself."""
    point, info = _fine_table_point()
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    h, half = 1.0 / 2048, 32
    lo, hi = tr["t"] - half * h, tr["t"] + half * h
    band = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)[0]
    fine = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 8 * half, lo, hi)[0]
    coarse = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi)[0]
    same = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 1)[0]
    # the truncated stencil leaves ~4e-6 of K at the peak (K ~ 370 at x = 1)
    assert abs(band - fine) <= 2.5e-3, (band, fine)
    assert abs(same - coarse) == 0.0
    assert abs(band - coarse) > 10 * abs(band - fine)  # the coarse rule alone is not enough


def test_band_limited_offset_mistake_is_caught():
    """Planted: fine nodes placed at the interval starts instead of their
    midpoints."""
    with open(SRC) as f:
        text = f.read()
    old = "tf = (np.arange(n * t_up) + 0.5) / t_up"
    assert text.count(old) == 1
    mod = _load(text.replace(old, "tf = np.arange(n * t_up) / t_up"), "tband_offset")
    assert _tband_error(mod, 32) > 1e-2


# ------------------------------------------------------------- peak-local rule

def _two_injection_point(shift):
    """The noise-free fine-table point, and the same point whose correlation
    tables also hold a second, identical signal `shift` table samples later
    (the tables add as the data do; U and V do not depend on the data)."""
    point, info = _fine_table_point()
    Q = np.asarray(point["Q"])
    Q2 = np.zeros_like(Q)
    Q2[:, shift:, :] = Q[:, :-shift, :]
    both = dict(point)
    both["Q"] = Q + Q2
    return point, both, info


def test_projection_bound_is_attained_at_the_injection_and_bounds_every_template():
    """The peak-local rule's envelope: U(t) = (1/2) sum_k q_k^T G_k^+ q_k is
    rho^2/2 at a noise-free injection (the data lie in the template span), and
    lies above lnL at any (phi, psi, x) and above the angular-and-distance
    marginal at that time."""
    point, info = _fine_table_point()
    tr = info["truth"]
    B = OD.ProjectionBound(point)
    assert abs(B(tr["ra"], tr["dec"], tr["t"]) - info["rho2"] / 2) <= 1e-5 * info["rho2"]
    pt = O.OraclePoint(point)
    rng = np.random.default_rng(9)
    for _ in range(4):
        t = tr["t"] + rng.uniform(-2e-3, 2e-3)
        U = B(tr["ra"], tr["dec"], t)
        th = {p: np.full(300, tr[p]) for p in W.PARAMS}
        th["t"][:] = t
        th["phase"] = rng.uniform(0, 2 * np.pi, 300)
        th["psi"] = rng.uniform(0, np.pi, 300)
        th["lnD"] = np.log(100.0) + rng.normal(0, 0.2, 300)
        assert np.max(O.lnL(pt, th)) <= U + 1e-6 * abs(U)
        d1 = {p: np.array([tr[p]]) for p in W.PARAMS}
        one = OD.lnL_direct(point, d1, 32, 16, 16, 50.0, 200.0, 1, t - 1e-7, t + 1e-7)[0]
        assert one <= U


def test_peak_local_rule_matches_the_band_limited_rule():
    """eq. ap:tlocal on the fine nodes of eq. ap:tband: with the peak well
    inside a +-32 coarse-sample window, the neighbourhood of +-16 sigma_t keeps
    under a third of the nodes, the remainder bound is below the tolerance,
    and the value equals the full band-limited rule within that bound."""
    point, info = _fine_table_point()
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    h, half = 1.0 / 2048, 32
    lo, hi = tr["t"] - half * h, tr["t"] + half * h
    full = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)[0]
    diag = []
    loc = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4, t_local=True,
                        diag=diag)[0]
    g = diag[0]
    assert not g["fallback"] and g["gap"] < math.log(1e-10)
    assert 0.05 < g["kept"].mean() < 0.33
    # the width against a least-squares parabola through the envelope's seven
    # nodes about the maximum (U ~ U0 - (t - t0)^2 / (2 sigma_t^2))
    B = OD.ProjectionBound(point)
    hf = h / 4
    f0 = g["maxima"][int(np.argmax([B(tr["ra"], tr["dec"], lo + (f + 0.5) * hf)
                                    for f in g["maxima"]]))]
    fs = np.arange(f0 - 3, f0 + 4)
    Us = [B(tr["ra"], tr["dec"], lo + (f + 0.5) * hf) for f in fs]
    a = np.polyfit((fs - f0) * hf, Us, 2)[0]
    sig_fit = 1.0 / math.sqrt(-2.0 * a)
    sig_rule = g["widths"][g["maxima"].index(f0)]
    assert abs(sig_rule / sig_fit - 1.0) < 0.1, (sig_rule, sig_fit)
    assert abs(loc - full) <= 2 * math.exp(g["gap"]) + 1e-13 * abs(full)
    # the neighbourhood holds the injection's node
    tf = lo + (np.arange(8 * half) + 0.5) * h / 4
    assert g["kept"][np.argmin(np.abs(tf - tr["t"]))]
    # a tolerance no bound can meet falls back to the band-limited rule itself
    diag = []
    fb = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4, t_local=True,
                       t_tol=1e-300, diag=diag)[0]
    assert diag[0]["fallback"] and fb == full


def test_peak_local_rule_keeps_both_peaks_of_two_injections():
    """Two identical signals 300 table samples (18.3 ms) apart: the envelope
    has two maxima of equal height, both neighbourhoods are kept and the
    stretch between them is not, and (at a tolerance of 1e-8) the value equals
    the band-limited rule within the remainder bound."""
    shift = 300
    dts = shift * float(np.asarray(_fine_table_point()[0]["q_dt"]))
    point, both, info = _two_injection_point(shift)
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    h, half = 1.0 / 2048, 48
    lo, hi = tr["t"] - half * h + dts / 2, tr["t"] + half * h + dts / 2
    full = OD.lnL_direct(both, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4)[0]
    diag = []
    loc = OD.lnL_direct(both, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4, t_local=True,
                        t_tol=1e-8, diag=diag)[0]
    g = diag[0]
    tf = lo + (np.arange(8 * half) + 0.5) * h / 4
    for t_inj in (tr["t"], tr["t"] + dts):
        assert g["kept"][np.argmin(np.abs(tf - t_inj))]
    assert len(g["maxima"]) >= 2
    assert not g["kept"][np.argmin(np.abs(tf - (tr["t"] + dts / 2)))]
    assert not g["fallback"] and g["kept"].mean() < 0.35
    assert abs(loc - full) <= 2 * math.exp(g["gap"]) + 1e-13 * abs(full)


@pytest.mark.parametrize("name,old,new", [
    ("bound_half_dropped", "total += 0.5 * float(q @ self.Ginv[k] @ q)",
     "total += float(q @ self.Ginv[k] @ q)"),
    ("width_without_root", "sig = h / math.sqrt(curv)", "sig = h / curv"),
    ("neighbourhood_one_sided", "keep |= np.abs(tf - tf[f]) <= c * sig",
     "keep |= (tf - tf[f] >= 0) & (tf - tf[f] <= c * sig)"),
])
def test_peak_local_planted_mistakes_are_caught(name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, name
    mod = _load(text.replace(old, new), "tlocal_" + name)
    failed = False
    try:
        point, info = _fine_table_point()
        tr = info["truth"]
        B = mod.ProjectionBound(point)
        if abs(B(tr["ra"], tr["dec"], tr["t"]) - info["rho2"] / 2) > 1e-5 * info["rho2"]:
            failed = True
        d = {p: np.array([tr[p]]) for p in W.PARAMS}
        h, half = 1.0 / 2048, 32
        lo, hi = tr["t"] - half * h, tr["t"] + half * h
        diag = []
        mod.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4, t_local=True,
                       diag=diag)
        g = diag[0]
        tf = lo + (np.arange(8 * half) + 0.5) * h / 4
        if g["fallback"] or not (0.05 < g["kept"].mean() < 0.33):
            failed = True
        else:  # the width against a parabola fit of the correct envelope
            Bc = OD.ProjectionBound(point)
            f0 = g["maxima"][0]
            fs = np.arange(f0 - 3, f0 + 4)
            Us = [Bc(tr["ra"], tr["dec"], lo + (f + 0.5) * h / 4) for f in fs]
            sig_fit = 1.0 / math.sqrt(-2.0 * np.polyfit((fs - f0) * h / 4, Us, 2)[0])
            if abs(g["widths"][0] / sig_fit - 1.0) >= 0.1:
                failed = True
            # the neighbourhood must reach 4 coarse samples before the peak
            if not g["kept"][np.argmin(np.abs(tf - (tr["t"] - 4 * h)))]:
                failed = True
    except Exception:
        failed = True
    assert failed, f"planted mistake {name} passed every pin"


# ------------------------------------------- mirrored band-limited reconstruction

def test_mirrored_reconstruction_is_exact_on_the_reflection_basis_and_equals_the_pregrid():
    """The mirrored series' trigonometric interpolant reproduces, at every
    fine midpoint, the series the reflection continues smoothly (sums of
    cos(pi k (x + 1/2)/n) sampled at the coarse midpoints, k < n), where the
    truncated sinc sum errs at the window's ends; and it equals the pregrid's
    FFT route (reflect, zero-pad, invert) at the common points."""
    import oracle.precompute as OP
    rng = np.random.default_rng(1)
    for n, tu in ((12, 4), (33, 2), (7, 8)):
        a = rng.normal(size=n) + 1j * rng.normal(size=n)
        ks = np.arange(n)
        coarse = np.cos(np.pi * np.outer(np.arange(n) + 0.5, ks) / n) @ a
        tf = (np.arange(n * tu) + 0.5) / tu
        exact = np.cos(np.pi * np.outer(tf, ks) / n) @ a
        m = OD.mirrored_upsample(coarse, tu)
        assert np.max(np.abs(m - exact)) <= 1e-12 * np.sum(np.abs(a))
        assert np.max(np.abs(OD.sinc_upsample(coarse, tu) - exact)) > 1e-3
        pg = OP.q_pregrid(coarse[None, :, None], 2 * tu)[0, :, 0]
        idx = 2 * np.arange(n * tu) + 1 - tu   # offsets from the first sample in h / (2 tu)
        ok = (idx >= 0) & (idx < pg.shape[0])
        assert np.max(np.abs(m[ok] - pg[idx[ok]])) <= 1e-12 * np.sum(np.abs(a))


def test_mirrored_rule_matches_the_fine_fixed_rule():
    """With the peak well inside the window, the mirrored band-limited rule
    agrees with the fixed-spacing rule evaluated directly on its fine nodes,
    as the truncated one does."""
    point, info = _fine_table_point()
    tr = info["truth"]
    d = {p: np.array([tr[p]]) for p in W.PARAMS}
    h, half = 1.0 / 2048, 32
    lo, hi = tr["t"] - half * h, tr["t"] + half * h
    mir = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 2 * half, lo, hi, 4, t_mirror=True)[0]
    fine = OD.lnL_direct(point, d, 48, 24, 16, 50.0, 200.0, 8 * half, lo, hi)[0]
    assert abs(mir - fine) <= 2.5e-3, (mir, fine)


def test_mirrored_reconstruction_misplaced_mirror_is_caught():
    with open(SRC) as f:
        text = f.read()
    old = "mirrored_kernel(np.add.outer(tf, tj), n)"
    assert text.count(old) == 1
    mod = _load(text.replace(old, "mirrored_kernel(np.add.outer(tf, tj - 0.5), n)"), "mirror_shift")
    n, tu = 12, 4
    a = np.random.default_rng(2).normal(size=n)
    coarse = np.cos(np.pi * np.outer(np.arange(n) + 0.5, np.arange(n)) / n) @ a
    exact = np.cos(np.pi * np.outer((np.arange(n * tu) + 0.5) / tu, np.arange(n)) / n) @ a
    assert np.max(np.abs(mod.mirrored_upsample(coarse, tu) - exact)) > 1e-3
