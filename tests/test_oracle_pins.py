"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
independent injection of the workload generator (tensor projection,
Wigner-d harmonics), closed forms, invariances stated in the paper, library
quadrature, or brute-force sums.  A dropped term, a wrong sign, a wrong index
or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle as O
import workload as W


def small_point(modes=((2, 2), (2, -2)), noise=False, snr=20.0, ndet=2, seed=11, rate=4096.0,
                half_window=0.05, f_low=20.0, f_max=512.0, df=0.5, dets=None, truth=None,
                q_dtype=np.complex128):
    rng = np.random.default_rng(seed)
    dets = dets if dets is not None else W.random_l_detectors(rng, ndet)
    truth = truth if truth is not None else W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=list(modes), f_low=f_low, f_max=f_max, df=df, rate=rate,
        half_window=half_window, snr=snr, truth=truth, gmst=0.7, d_ref=100.0, rng=rng,
        noise=noise, q_dtype=q_dtype)
    return point, exact, info, O.OraclePoint(point, exact)


def one(truth, **over):
    th = dict(truth)
    th.update(over)
    return {p: np.array([th[p]], dtype=np.float64) for p in W.PARAMS}


def rand_draws(rng, n, truth=None, spread=None):
    pri = W.Prior(50.0, 200.0, 0.01).sample(rng, n)
    if truth is not None:
        for p in W.PARAMS:
            pri[p] = truth[p] + spread[p] * rng.standard_normal(n)
    return {p: np.asarray(pri[p], dtype=np.float64) for p in W.PARAMS}


def half_dd(exact):
    return 0.5 * float(np.sum(exact["wgt"] * np.abs(exact["dk"]) ** 2))


# --------------------------------------------------------------- whole lnL

@pytest.mark.parametrize("modes", [((2, 2), (2, -2)), tuple(W.MODES10)])
def test_truth_gives_half_rho2(modes):
    """Noise-free injection at the true parameters, exact Q:
    lnL = <h|d> - <h|h>/2 with d = h gives rho^2/2 (Sec. III, static case)."""
    point, exact, info, pt = small_point(modes=modes, snr=37.0)
    lnl, td, tq, oob = O.lnL(pt, one(info["truth"]), exact_q=True, terms=True)
    rho2 = info["rho2"]
    assert oob == 0
    assert abs(lnl[0] - rho2 / 2) < 1e-10 * rho2
    assert abs(td[0] - rho2) < 1e-10 * rho2
    assert abs(tq[0] - rho2 / 2) < 1e-10 * rho2


def test_lnl_equals_direct_inner_products_at_arbitrary_draws():
    """At any draw, lnL(exact Q) = <h(theta)|d> - <h(theta)|h(theta)>/2 with
    the template h(theta) built by the generator's independent injection and
    the inner product 2 df sum conj(a) b / S taken directly."""
    point, exact, info, pt = small_point(modes=W.MODES10[:6], noise=True, snr=15.0)
    rng = np.random.default_rng(3)
    draws = rand_draws(rng, 12)
    lnl = O.lnL(pt, draws, exact_q=True)
    rng2 = np.random.default_rng(0)
    hlm_unit = exact["hlm"]
    rng_det = np.random.default_rng(11)
    dets = W.random_l_detectors(rng_det, 2)
    for i in range(12):
        th = {p: float(draws[p][i]) for p in W.PARAMS}
        hk, _ = W.inject(dets, W.MODES10[:6], hlm_unit, exact["freq"], th, point["gmst"],
                         point["d_ref"])
        dh = float(np.sum(exact["wgt"] * np.real(np.conj(hk) * exact["dk"])))
        hh = float(np.sum(exact["wgt"] * np.abs(hk) ** 2))
        assert abs(lnl[i] - (dh - 0.5 * hh)) < 1e-9 * max(1.0, abs(dh) + hh)
    del rng2


def test_cauchy_schwarz_bound_every_draw():
    """lnL <= <d|d>/2 for every draw (App. A): exact in exact-Q mode; with the
    table + cubic the bound holds up to the interpolation error."""
    point, exact, info, pt = small_point(modes=W.MODES10[:4], noise=True, snr=25.0)
    rng = np.random.default_rng(4)
    truth = info["truth"]
    spread = {"ra": 0.02, "dec": 0.02, "psi": 0.05, "incl": 0.05, "phase": 0.05, "lnD": 0.05,
              "t": 2e-4}
    draws = rand_draws(rng, 400, truth, spread)
    bound = half_dd(exact)
    lnl_ex = O.lnL(pt, draws, exact_q=True)
    assert np.all(lnl_ex <= bound * (1 + 1e-12))
    lnl_tab = O.lnL(pt, draws)
    assert np.all(lnl_tab <= bound + 0.05 * math.sqrt(2 * bound))


def test_quadratic_term_is_half_template_norm_and_nonnegative():
    point, exact, info, pt = small_point(modes=W.MODES10[:6])
    rng = np.random.default_rng(5)
    draws = rand_draws(rng, 50)
    _, td, tq, _ = O.lnL(pt, draws, exact_q=True, terms=True)
    assert np.all(tq >= 0)
    dets = W.random_l_detectors(np.random.default_rng(11), 2)
    for i in range(0, 50, 7):
        th = {p: float(draws[p][i]) for p in W.PARAMS}
        hk, _ = W.inject(dets, W.MODES10[:6], exact["hlm"], exact["freq"], th, point["gmst"],
                         point["d_ref"])
        hh = float(np.sum(exact["wgt"] * np.abs(hk) ** 2))
        assert abs(tq[i] - 0.5 * hh) < 1e-10 * max(hh, 1e-30)


# ------------------------------------------------------- antenna and delays

def test_antenna_psi_structure_and_bounds():
    rng = np.random.default_rng(6)
    for _ in range(20):
        pos, resp = W.detector(rng.uniform(-1, 1), rng.uniform(-3, 3), rng.uniform(0, 3))
        ra, dec, psi, g = rng.uniform(0, 6.28), rng.uniform(-1.5, 1.5), rng.uniform(0, 3), 0.4
        F0 = O.antenna(resp, ra, dec, 0.0, g)
        F = O.antenna(resp, ra, dec, psi, g)
        # F(psi) = exp(2 i psi) F(0): the antenna factor carries e^{2 i psi} (App. E)
        assert abs(F - np.exp(2j * psi) * F0) < 1e-13
        assert abs(O.antenna(resp, ra, dec, psi + math.pi, g) - F) < 1e-13
        assert abs(O.antenna(resp, ra, dec, psi + math.pi / 2, g) + F) < 1e-13
        assert abs(F.real) <= 1 + 1e-12 and abs(F.imag) <= 1 + 1e-12


def test_antenna_closed_form_overhead_source():
    """Source at the zenith of an L detector with arms along east/north:
    F_+ = cos 2 psi, F_x = -sin 2 psi in this basis (F = e^{2 i psi})."""
    lat, lon = 0.3, 1.1
    pos, resp = W.detector(lat, lon, 0.0)
    for psi in (0.0, 0.3, 1.0):
        F = O.antenna(resp, lon + 0.25, lat, psi, 0.25)
        assert abs(F - np.exp(2j * psi)) < 1e-12


def test_et_null_stream():
    """Sum of the antenna factors of the co-located 60-degree triangle is zero
    for every source direction and polarisation."""
    dets = W.et_triangle(0.7, 0.16, 0.35)
    rng = np.random.default_rng(7)
    for _ in range(30):
        ra, dec, psi = rng.uniform(0, 6.28), rng.uniform(-1.5, 1.5), rng.uniform(0, 3.14)
        s = sum(O.antenna(r, ra, dec, psi, 1.3) for _, r in dets)
        assert abs(s) < 1e-14


def test_delay_sign_and_magnitude():
    """A source straight above a detector reaches it |x_k| earlier than the
    geocentre: t_k = t_c - |x_k| (s points to the source)."""
    lat, lon, gmst = 0.5, -1.2, 2.0
    pos, _ = W.detector(lat, lon, 0.3)
    tk = O.delay(pos, lon + gmst, lat, gmst, 0.001)
    assert abs(tk - (0.001 - np.linalg.norm(pos))) < 1e-15
    tk2 = O.delay(pos, lon + gmst + math.pi, -lat, gmst, 0.0)
    assert abs(tk2 - np.linalg.norm(pos)) < 1e-15


def test_sky_basis_orthonormal():
    s, e1, e2 = O.sky_basis(1.0, 0.3, 0.2)
    B = np.stack([s, e1, e2])
    assert np.allclose(B @ B.T, np.eye(3), atol=1e-15)


# --------------------------------------------------------------- harmonics

def test_sylm_closed_forms():
    for th in (0.0, 0.4, 1.3, 2.5, math.pi):
        for ph in (0.0, 0.9):
            c = math.cos(th)
            forms = {
                2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
                -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2,
                1: math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 + c),
                -1: math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 - c),
                0: math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2,
            }
            for m, v in forms.items():
                y = O.sylm(-2, 2, m, th, ph)
                assert abs(y - v * np.exp(1j * m * ph)) < 1e-14


def _wigner_expm(l, beta):
    """d^l(beta) = exp(-i beta J_y), J_y from the ladder operators (library expm)."""
    ms = np.arange(l, -l - 1, -1)
    Jp = np.zeros((2 * l + 1, 2 * l + 1))
    for a, m in enumerate(ms):
        if m + 1 <= l:
            Jp[a - 1, a] = math.sqrt(l * (l + 1) - m * (m + 1))
    Jy = (Jp - Jp.T) / 2j
    return scipy.linalg.expm(-1j * beta * Jy), ms


@pytest.mark.parametrize("l", [2, 3, 4, 5, 8])
def test_sylm_against_matrix_exponential_wigner_d(l):
    """-2Y_lm = sqrt((2l+1)/4pi) d^l_{m,2}(theta) e^{i m phi} with d^l from
    the matrix exponential of the angular-momentum generator."""
    for th in (0.2, 1.1, 2.9):
        d, ms = _wigner_expm(l, th)
        col = list(ms).index(2)
        for row, m in enumerate(ms):
            ref = math.sqrt((2 * l + 1) / (4 * math.pi)) * d[row, col].real * np.exp(1j * m * 0.6)
            assert abs(O.sylm(-2, l, int(m), th, 0.6) - ref) < 1e-12


@pytest.mark.parametrize("l", [2, 3, 4, 6, 8])
def test_sylm_addition_theorem(l):
    for th in (0.3, 1.7, 2.8):
        tot = sum(abs(O.sylm(-2, l, m, th, 0.2)) ** 2 for m in range(-l, l + 1))
        assert abs(tot - (2 * l + 1) / (4 * math.pi)) < 1e-13


def test_sylm_orthonormal_by_quadrature():
    nodes, weights = np.polynomial.legendre.leggauss(40)
    lm = [(2, 2), (3, 2), (4, 2), (2, 1), (3, 1)]
    for a in lm:
        for b in lm:
            if a[1] != b[1]:
                continue  # e^{i(m-m')phi} integrates to zero over phi
            val = 2 * math.pi * sum(
                w * (np.conj(O.sylm(-2, a[0], a[1], math.acos(x), 0.0)) *
                     O.sylm(-2, b[0], b[1], math.acos(x), 0.0)).real for x, w in zip(nodes, weights))
            assert abs(val - (1.0 if a == b else 0.0)) < 1e-12


def test_sylm_dtheta_matches_finite_difference():
    for l, m in [(2, 2), (3, -1), (4, 4), (5, 2)]:
        for th in (0.3, 1.4, 2.6):
            h = 1e-6
            fd = (O.sylm(-2, l, m, th + h, 0.3) - O.sylm(-2, l, m, th - h, 0.3)) / (2 * h)
            assert abs(O.sylm(-2, l, m, th, 0.3, dtheta=True) - fd) < 1e-8


# ----------------------------------------------------- invariances of lnL

def test_psi_plus_pi_invariance():
    point, exact, info, pt = small_point(modes=W.MODES10[:6], noise=True)
    rng = np.random.default_rng(8)
    d = rand_draws(rng, 100)
    d2 = dict(d)
    d2["psi"] = d["psi"] + math.pi
    a, b = O.lnL(pt, d), O.lnL(pt, d2)
    assert np.max(np.abs(a - b)) < 1e-10 * max(1.0, np.max(np.abs(a)))


def test_phase_psi_degeneracy_22_only():
    """(2,+-2) modes only: lnL(phi + pi/2, psi + pi/2) = lnL(phi, psi)."""
    point, exact, info, pt = small_point(noise=True)
    rng = np.random.default_rng(9)
    d = rand_draws(rng, 100)
    d2 = dict(d)
    d2["phase"] = d["phase"] + math.pi / 2
    d2["psi"] = d["psi"] + math.pi / 2
    a, b = O.lnL(pt, d), O.lnL(pt, d2)
    assert np.max(np.abs(a - b)) < 1e-10 * max(1.0, np.max(np.abs(a)))


def test_face_on_depends_only_on_psi_plus_phase():
    """iota = 0: only m = +2 survives, so lnL depends on (phi, psi) only through
    phi + psi (the phi_+ coordinate)."""
    point, exact, info, pt = small_point(modes=W.MODES10[:6], noise=True)
    rng = np.random.default_rng(10)
    d = rand_draws(rng, 60)
    d["incl"] = np.zeros(60)
    d2 = dict(d)
    shift = rng.uniform(-1, 1, 60)
    d2["phase"] = d["phase"] + shift
    d2["psi"] = d["psi"] - shift
    a, b = O.lnL(pt, d), O.lnL(pt, d2)
    assert np.max(np.abs(a - b)) < 1e-10 * max(1.0, np.max(np.abs(a)))


def test_angular_harmonic_content():
    """At fixed time, lnL(phi, psi) has Fourier content only for |q| <= 2 m_max
    in phi and |2p| <= 4 in psi (eq. ap:angleharm)."""
    modes = W.MODES10[:8]
    point, exact, info, pt = small_point(modes=modes, noise=True)
    mmax = max(abs(m) for _, m in modes)
    n_phi, n_psi = 32, 16
    phis = 2 * math.pi * np.arange(n_phi) / n_phi
    psis = math.pi * np.arange(n_psi) / n_psi
    base = {p: info["truth"][p] for p in W.PARAMS}
    P, S = np.meshgrid(phis, psis, indexing="ij")
    d = {p: np.full(P.size, base[p]) for p in W.PARAMS}
    d["phase"], d["psi"] = P.ravel(), S.ravel()
    grid = O.lnL(pt, d).reshape(n_phi, n_psi)
    spec = np.abs(np.fft.fft2(grid)) / grid.size
    qs = np.fft.fftfreq(n_phi, 1.0 / n_phi)
    ps = np.fft.fftfreq(n_psi, 1.0 / n_psi)  # frequency in units of 2 psi
    mask = (np.abs(qs)[:, None] > 2 * mmax) | (np.abs(ps)[None, :] > 2)
    assert spec[mask].max() < 1e-11 * spec.max()
    assert spec[~mask].max() > 0


# ---------------------------------------------------------------- distance

def test_distance_scaling_exact_quadratic():
    """T_d ~ 1/D and T_q ~ 1/D^2: lnL(x) = K x - R x^2/2 exactly (eq. ap:dexp),
    and at the noise-free truth with D_ref = D_true, x* = K/R = 1 (eq. ap:dpeak)."""
    point, exact, info, pt = small_point(modes=W.MODES10[:6])
    truth = info["truth"]
    xs = np.array([0.5, 0.8, 1.0, 1.3, 2.0])
    d = {p: np.full(5, truth[p]) for p in W.PARAMS}
    d["lnD"] = np.log(100.0 / xs)
    lnl, td, tq, _ = O.lnL(pt, d, exact_q=True, terms=True)
    K = td / xs
    R = 2 * tq / xs ** 2
    assert np.ptp(K) < 1e-12 * abs(K[0]) and np.ptp(R) < 1e-12 * abs(R[0])
    assert abs(K[0] / R[0] - 1.0) < 1e-12


def test_dist_nodes_rule_and_prior_normalisation():
    """Spacing c(tol)/rho_max with c = pi sqrt(2/ln(2/tol)) (eq. ap:dlog); the
    weights integrate the normalised D^2 prior to one."""
    x, lnw = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)
    c = math.pi * math.sqrt(2 / math.log(2 / 1e-4))
    lnd = np.log(100.0 / x)
    assert np.max(np.diff(lnd)) <= c / 1000.0 * (1 + 1e-12)
    # trapezoid in ln d on the smooth density 3 D^3/(Dmax^3 - Dmin^3): its error
    # is (h^2/12) int f'' = (3/4) h^2 relative, h the spacing
    h = np.max(np.diff(lnd))
    assert abs(np.exp(lnw).sum() - 1.0) < 0.76 * h * h


def test_distance_marginal_against_adaptive_quadrature():
    """LSE over the node table = ln int p(D) exp(lnL(D)) dD, checked against
    scipy's adaptive quadrature, and converging as the spacing halves."""
    point, exact, info, pt = small_point(modes=W.MODES10[:4], snr=60.0, noise=True)
    rng = np.random.default_rng(12)
    truth = info["truth"]
    spread = {"ra": 0.01, "dec": 0.01, "psi": 0.03, "incl": 0.03, "phase": 0.03, "lnD": 0.0,
              "t": 1e-4}
    d = rand_draws(rng, 4, truth, spread)
    _, td1, tq1, _ = O.lnL(pt, {**d, "lnD": np.full(4, math.log(100.0))}, terms=True)
    errs = []
    for rho_max in (60.0, 120.0, 240.0):
        x, lnw = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, rho_max)
        marg = O.lnL_distmarg(pt, d, x, lnw)
        for i in range(4):
            K, R = td1[i], 2 * tq1[i]
            f = lambda D: 3 * D ** 2 / (200.0 ** 3 - 50.0 ** 3) * math.exp(
                K * 100.0 / D - 0.5 * R * (100.0 / D) ** 2 - (K * K / (2 * R)))
            val, _ = scipy.integrate.quad(f, 50.0, 200.0, epsabs=0, epsrel=1e-13, limit=400,
                                          points=[100.0 * R / K] if 50 < 100.0 * R / K < 200 else None)
            ref = math.log(val) + K * K / (2 * R)
            errs.append((rho_max, abs(marg[i] - ref)))
    worst = {r: max(e for rr, e in errs if rr == r) for r in (60.0, 120.0, 240.0)}
    assert worst[240.0] < 1e-6
    assert worst[240.0] <= worst[60.0]


def dist_marginal_fd_errors(pt, d, x, lnw):
    """Per component, |analytic - central difference| / max(1, |analytic|) of
    the distance-marginalised gradient.  The node sum is a smooth function of
    K and R whatever the table, so its derivative is E[x] dK - E[x^2] dR/2
    over the node posterior exactly (eq. ap:dexp, eq. ap:dlog)."""
    _, g = O.lnL_distmarg(pt, d, x, lnw, grad=True)
    th = np.stack([d[p] for p in W.PARAMS], axis=1)
    errs = {}
    for j in range(7):
        step = 1e-6 * (1e-3 if j == 6 else 1.0)  # t in seconds
        tp, tm = th.copy(), th.copy()
        tp[:, j] += step
        tm[:, j] -= step
        fd = (O.lnL_distmarg(pt, tp, x, lnw) - O.lnL_distmarg(pt, tm, x, lnw)) / (2 * step)
        errs[j] = np.abs(g[:, j] - fd) / np.maximum(1.0, np.abs(g[:, j]))
    return g, errs


def test_distance_marginal_gradient_matches_central_differences():
    """The distance-marginalised gradient against central differences of the
    distance-marginalised lnL in ra, dec, psi, iota, phi_ref and t_c, on draws
    near the peak where the node posterior is narrow and E[x^2] - E[x]^2 is
    small but not negligible; the draw's own lnD is ignored, so its slot and its
    central difference are both zero.  A dropped 1/2 on dR or E[x]^2 in place
    of E[x^2] moves every component by ~T_q-sized amounts."""
    point, exact, info, pt = small_point(modes=W.MODES10[:6], noise=True, snr=30.0,
                                         rate=16384.0)
    rng = np.random.default_rng(21)
    truth = info["truth"]
    spread = {"ra": 0.02, "dec": 0.02, "psi": 0.1, "incl": 0.1, "phase": 0.1, "lnD": 0.3,
              "t": 3e-4}
    d = rand_draws(rng, 64, truth, spread)
    x, lnw = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, 60.0)
    g, errs = dist_marginal_fd_errors(pt, d, x, lnw)
    assert np.all(g[:, 5] == 0.0)
    for j in (0, 1, 2, 3, 4, 6):
        # the cubic's slope is only C0 at knots (t, and ra/dec through t_k)
        assert np.median(errs[j]) < 1e-5, (j, np.median(errs[j]))
        assert np.mean(errs[j] < 1e-4) > 0.9, j
    assert np.max(errs[5]) < 1e-12
    # the node posterior really is spread: E[x^2] differs from E[x]^2, so the
    # check separates the two moments
    assert np.max(np.abs(g[:, :5])) > 10.0


# ------------------------------------------------------------ interpolation

def test_cubic_interpolant_exact_for_cubics():
    t0, dt, n = -0.01, 1e-4, 200
    tj = t0 + dt * np.arange(n)
    coeffs = np.array([0.3 + 0.1j, -2.0, 5.0 + 1j, 40.0])
    poly = lambda t: coeffs[0] + coeffs[1] * t * 100 + coeffs[2] * (t * 100) ** 2 + coeffs[3] * (t * 100) ** 3
    q = poly(tj)[:, None]
    for t in np.linspace(t0 + 2 * dt, t0 + (n - 3) * dt, 37):
        v, dv, oob = O.qinterp(q, t0, dt, t)
        assert oob == 0
        assert abs(v[0] - poly(t)) < 1e-9 * abs(poly(t)) + 1e-12
        dpoly = 100 * (coeffs[1] + 2 * coeffs[2] * (t * 100) + 3 * coeffs[3] * (t * 100) ** 2)
        assert abs(dv[0] - dpoly) < 1e-7 * abs(dpoly)


def test_cubic_taps_outside_table_read_zero_and_count():
    q = np.ones((10, 1), dtype=np.complex128)
    v, _, oob = O.qinterp(q, 0.0, 1.0, 0.5)
    assert oob == 1  # tap j-1 = -1
    v2, _, oob2 = O.qinterp(q, 0.0, 1.0, 20.0)
    assert oob2 == 4 and v2[0] == 0


def test_interpolation_error_falls_16x_per_doubling():
    """The four-point cubic's error against exact Q falls ~16x when the table
    rate doubles (eq. ap:q-pregrid-accuracy)."""
    rng = np.random.default_rng(13)
    errs = []
    for rate in (2048.0, 4096.0, 8192.0):
        point, exact, info, pt = small_point(modes=((2, 2), (2, -2)), rate=rate, snr=50.0,
                                             seed=14)
        truth = info["truth"]
        spread = {"ra": 0.01, "dec": 0.01, "psi": 0.03, "incl": 0.03, "phase": 0.03,
                  "lnD": 0.02, "t": 3e-4}
        d = rand_draws(np.random.default_rng(15), 200, truth, spread)
        errs.append(np.max(np.abs(O.lnL(pt, d) - O.lnL(pt, d, exact_q=True))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 8 < r1 < 32 and 8 < r2 < 32


# --------------------------------------------------------------------- lnZ

def test_lnz_closed_forms():
    lnZ, sig, neff = O.lnZ(np.full(1000, -3.25))
    assert abs(lnZ + 3.25) < 1e-14 and sig < 1e-7 and abs(neff - 1000) < 1e-9
    v = np.array([0.0] * 3 + [math.log(2.0)])
    lnZ, sig, neff = O.lnZ(v)
    assert abs(lnZ - math.log(5.0 / 4)) < 1e-15
    assert abs(neff - 2.5) < 1e-15
    assert abs(sig - math.sqrt(7 / 25 - 1 / 4)) < 1e-15
    lnZ, sig, neff = O.lnZ(np.zeros(4), np.log(np.array([1, 1, 1, 2.0])))
    assert abs(lnZ - math.log(5.0 / 4)) < 1e-15


def test_lnz_large_offsets_against_fsum():
    rng = np.random.default_rng(16)
    v = 5e5 + rng.normal(0, 20, 5000)
    w = rng.normal(0, 3, 5000)
    m = np.max(v + w)
    ref = m + math.log(math.fsum(np.exp(v + w - m))) - math.log(5000)
    assert abs(O.lnZ(v, w)[0] - ref) < 1e-9


def test_lnz_matches_brute_force_time_phase_quadrature():
    """Tiny case, sky/psi/iota/D fixed: lnZ over (t, phi) draws equals a brute
    2-D quadrature of exp(lnL) (periodic trapezoid in phi, Simpson in t) when
    the quadrature nodes are fed as draws with their weights, and Monte Carlo
    prior draws agree with it within 3 sigma."""
    point, exact, info, pt = small_point(snr=8.0, noise=True, f_max=256.0)
    truth = info["truth"]
    n_phi, n_t = 24, 801
    t_half = 2e-3
    phis = 2 * math.pi * np.arange(n_phi) / n_phi
    ts = np.linspace(-t_half, t_half, n_t)
    simpson = np.ones(n_t)
    simpson[1:-1:2], simpson[2:-1:2] = 4.0, 2.0
    simpson *= (ts[1] - ts[0]) / 3
    P, T = np.meshgrid(phis, ts, indexing="ij")
    d = {p: np.full(P.size, truth[p]) for p in W.PARAMS}
    d["phase"], d["t"] = P.ravel(), T.ravel()
    lnl = O.lnL(pt, d, exact_q=True).reshape(n_phi, n_t)
    wq = (np.full(n_phi, 1.0 / n_phi)[:, None] * simpson[None, :] / (2 * t_half))
    m = lnl.max()
    quad = m + math.log(math.fsum((wq * np.exp(lnl - m)).ravel()))
    logw = np.log(wq.ravel() * P.size)
    assert abs(O.lnZ(lnl.ravel(), logw)[0] - quad) < 1e-12 * max(1, abs(quad))
    rng = np.random.default_rng(17)
    nmc = 20000
    dm = {p: np.full(nmc, truth[p]) for p in W.PARAMS}
    dm["phase"] = rng.uniform(0, 2 * math.pi, nmc)
    dm["t"] = rng.uniform(-t_half, t_half, nmc)
    lz, sig, neff = O.lnZ(O.lnL(pt, dm, exact_q=True))
    assert abs(lz - quad) < 3 * sig + 1e-9


# --------------------------------------------------------------- gradients

def test_gradient_matches_central_differences():
    point, exact, info, pt = small_point(modes=W.MODES10[:6], noise=True, snr=30.0,
                                         rate=16384.0)
    rng = np.random.default_rng(18)
    truth = info["truth"]
    spread = {"ra": 0.05, "dec": 0.05, "psi": 0.2, "incl": 0.2, "phase": 0.2, "lnD": 0.1,
              "t": 1e-3}
    d = rand_draws(rng, 40, truth, spread)
    _, g = O.lnL_grad(pt, d)
    h = 1e-6
    th = np.stack([d[p] for p in W.PARAMS], axis=1)
    for j in range(7):
        step = h * (1e-3 if j == 6 else 1.0)  # t in seconds
        tp, tm = th.copy(), th.copy()
        tp[:, j] += step
        tm[:, j] -= step
        fd = (O.lnL(pt, tp) - O.lnL(pt, tm)) / (2 * step)
        # the cubic's slope is only C0 at knots: accept one-sided agreement there
        err = np.abs(g[:, j] - fd)
        scale = np.maximum(1.0, np.abs(g[:, j]))
        assert np.median(err / scale) < 1e-5, (j, np.median(err / scale))
        assert np.mean(err / scale < 1e-4) > 0.9


def test_gradient_exact_q_matches_central_differences_everywhere():
    point, exact, info, pt = small_point(modes=W.MODES10[:4], noise=True, snr=30.0)
    rng = np.random.default_rng(19)
    d = rand_draws(rng, 10)
    _, g = O.lnL_grad(pt, d, exact_q=True)
    th = np.stack([d[p] for p in W.PARAMS], axis=1)
    for j in range(7):
        step = 1e-6 * (1e-3 if j == 6 else 1.0)
        tp, tm = th.copy(), th.copy()
        tp[:, j] += step
        tm[:, j] -= step
        fd = (O.lnL(pt, tp, exact_q=True) - O.lnL(pt, tm, exact_q=True)) / (2 * step)
        assert np.all(np.abs(g[:, j] - fd) < 1e-5 * np.maximum(1.0, np.abs(g[:, j]))), j


def test_fisher_closed_form_single_detector_single_mode():
    """One detector, one (2,2) mode, exact Q, zero noise: -Hessian of lnL in
    (lnD, phi_ref, t_c) at the truth equals
    rho^2 [[1,0,0],[0,4,4 pi <f>],[0,4 pi <f>,4 pi^2 <f^2>]] (eq. ap:fisher3)
    with the moments of eq. ap:fmoments (lnD = -lnA)."""
    rng = np.random.default_rng(20)
    dets = W.random_l_detectors(rng, 1)
    point, exact, info, pt = small_point(modes=((2, 2),), dets=dets, snr=30.0, f_max=256.0)
    truth = info["truth"]
    idx = [5, 4, 6]  # lnD, phase, t
    th0 = np.array([[truth[p] for p in W.PARAMS]])
    H = np.zeros((3, 3))
    for a, j in enumerate(idx):
        step = 1e-5 * (1e-3 if j == 6 else 1.0)
        tp, tm = th0.copy(), th0.copy()
        tp[0, j] += step
        tm[0, j] -= step
        gp = O.lnL_grad(pt, tp, exact_q=True)[1][0]
        gm = O.lnL_grad(pt, tm, exact_q=True)[1][0]
        H[a] = (gp[idx] - gm[idx]) / (2 * step)
    Gamma = -0.5 * (H + H.T)
    mom = W.noise_moments(exact["freq"], exact["wgt"][0], info["hk"][0])
    rho2 = info["rho2"]
    ref = rho2 * np.array([[1, 0, 0], [0, 4, 4 * math.pi * mom[1]],
                           [0, 4 * math.pi * mom[1], 4 * math.pi ** 2 * mom[2]]])
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.max(np.abs(Gamma - ref) / scale) < 1e-4


# ------------------------------------------------------------ input checks

def test_fixture_u_hermitian_v_symmetric():
    point, exact, info, pt = small_point(modes=W.MODES10)
    U, V = point["U"], point["V"]
    assert np.allclose(U, np.conj(np.transpose(U, (0, 2, 1))), rtol=0, atol=1e-12 * np.abs(U).max())
    assert np.allclose(V, np.transpose(V, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(V).max())
