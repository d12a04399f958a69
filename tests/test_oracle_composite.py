"""Pins of the composite-index oracle (Sec. III: Earth rotation, Paths A/B;
finite arms, Path D), each against something other than the oracle itself:

* Path A carries the antenna drift exactly, so with data injected as
  F_k(t) h_Y(t - t_k) (placed, then modulated) the likelihood at the
  injection equals <d|d>/2, and no draw exceeds it (Cauchy-Schwarz,
  Appendix A), only if the arrival-time post-phase is applied;
* the rotation coefficients satisfy sum_n C_(p,n) e^{i n theta} =
  F_k(gmst + theta) (-dt_k(theta))^p / p! at sidereal angles off the DFT grid
  (eq. slowrot:master), and a source at a celestial pole sees one harmonic;
* Omega -> 0 collapses the rotation likelihood to the static one, and
  p_max = 0 of the finite-arm expansion is the static antenna factor;
* the finite-arm expansion converges to the full two-arm transfer function
  (eq. fsize:FA) and the likelihood at the injection to <d|d>/2 as p_max grows;
* planted mistakes (post-phase dropped or flipped, DFT sign, drift sign,
  factorial, arm power, polarisation conjugate, composite order) each fail
  one of these pins.
"""
import importlib.util
import math
import os
import sys
import tempfile

import numpy as np
import pytest

import oracle as O
import oracle.composite as OC
import workload as W
import workload.composite as WC


@pytest.fixture(scope="module")
def rot0():
    return WC.comp_small(WC.ROTATION, 0, n_draws=384)


@pytest.fixture(scope="module")
def arm6():
    return WC.comp_small(WC.FINITE_ARM, 6, n_draws=256)


def truth_draw(info):
    return {p: np.array([info["truth"][p]]) for p in W.PARAMS}


def test_n_index():
    assert [OC.n_index(OC.ROTATION, p) for p in range(4)] == [5, 12, 21, 32]
    assert [OC.n_index(OC.FINITE_ARM, p) for p in range(4)] == [1, 2, 3, 4]


def test_path_a_saturates_cauchy_schwarz(rot0):
    point, exact, info, draws, logw = rot0
    pt = OC.CompPoint(point)
    half_dd = 0.5 * info["rho2"]
    lt = OC.lnL(pt, truth_draw(info))[0]
    assert abs(lt - half_dd) <= 1e-9 * half_dd, (lt, half_dd)
    lnl = OC.lnL(pt, draws)
    assert np.all(lnl <= half_dd * (1 + 1e-9)), lnl.max() - half_dd


@pytest.mark.parametrize("p_max", [0, 1, 2])
def test_rotation_coefficient_identity(p_max):
    rng = np.random.default_rng(5)
    dets = WC.random_detectors_arms(rng, 3, 4.0e3)
    omega = 0.7
    for trial in range(4):
        ra, dec, psi = rng.uniform(0, 2 * math.pi), rng.uniform(-1.4, 1.4), rng.uniform(0, math.pi)
        gmst, tc = rng.uniform(0, 2 * math.pi), rng.uniform(-0.01, 0.01)
        for d in dets:
            C = OC.rotation_coeffs(d["resp"], d["pos"], omega, p_max, ra, dec, psi, gmst, tc)
            tk = O.delay(d["pos"], ra, dec, gmst, tc)
            off = 0
            for p in range(p_max + 1):
                n = np.arange(-(2 + p), 3 + p)
                Cp = C[off:off + len(n)] * np.exp(-1j * n * omega * tk)   # undo the post-phase
                off += len(n)
                for theta in rng.uniform(0, 2 * math.pi, 3):
                    lhs = np.sum(Cp * np.exp(1j * n * theta))
                    F = O.antenna(d["resp"], ra, dec, psi, gmst + theta)
                    mdt = -(O.delay(d["pos"], ra, dec, gmst + theta, tc) - tk)
                    rhs = F * mdt ** p / math.factorial(p)
                    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(F)) * 0.03 ** p, (p, lhs, rhs)
            assert off == len(C)


def test_pole_sees_one_harmonic():
    """Source on the celestial axis: the antenna factor rotates rigidly, so
    only e^{-2 i theta} (north) or e^{+2 i theta} (south) survives."""
    rng = np.random.default_rng(6)
    d = WC.random_detectors_arms(rng, 1, 4.0e3)[0]
    for dec, keep in ((math.pi / 2, -2), (-math.pi / 2, 2)):
        C = OC.rotation_coeffs(d["resp"], d["pos"], 0.0, 0, 0.4, dec, 0.3, 1.1, 0.0)
        for j, n in enumerate(range(-2, 3)):
            if n == keep:
                assert abs(C[j]) > 0.1
            else:
                assert abs(C[j]) < 1e-12, (dec, n, C)


def _static_from_block(point, a):
    """Static point whose tables are block a of a composite point."""
    M = int(point["M"])
    sl = slice(a * M, (a + 1) * M)
    return {"K": point["K"], "M": M, "ell": point["ell"], "em": point["em"],
            "Q": np.ascontiguousarray(np.asarray(point["Q"])[:, :, sl]),
            "q_t0": point["q_t0"], "q_dt": point["q_dt"],
            "U": np.ascontiguousarray(point["U"][:, sl, sl]),
            "V": np.ascontiguousarray(point["V"][:, sl, sl]),
            "det_pos": point["det_pos"], "det_resp": point["det_resp"],
            "gmst": point["gmst"], "d_ref": point["d_ref"]}


@pytest.mark.parametrize("p_max", [0, 2])
def test_rotation_omega_zero_is_static(p_max):
    point, exact, info, draws, logw = WC.comp_small(WC.ROTATION, p_max, n_draws=128, omega=0.0)
    pt = OC.CompPoint(point)
    comp = OC.lnL(pt, draws)
    static = O.lnL(O.OraclePoint(_static_from_block(point, 2)), draws, threads=1)  # (p, n) = (0, 0)
    assert np.max(np.abs(comp - static)) <= 1e-10 * np.max(np.abs(static))


def test_arm_p0_is_static_antenna():
    rng = np.random.default_rng(7)
    for d in WC.random_detectors_arms(rng, 3, 4.0e4):
        for _ in range(5):
            ra, dec, psi, gmst = rng.uniform(0, 6.2), rng.uniform(-1.5, 1.5), rng.uniform(0, 3.1), 0.9
            b = OC.arm_coeffs(d["arm_x"], d["arm_y"], 3, ra, dec, psi, gmst)
            F = O.antenna(d["resp"], ra, dec, psi, gmst)
            assert abs(b[0] - F) <= 1e-14


def test_arm_expansion_matches_transfer_function():
    """sum_p b_p W_p(pi f T) = e^{2 pi i f T} F_k(f) of eq. fsize:FA, where the
    right side is built from the two legs' sinc transfer functions."""
    rng = np.random.default_rng(8)
    d = WC.random_detectors_arms(rng, 1, 4.0e4)[0]
    f = np.linspace(-2048.0, 2048.0, 41)
    x = math.pi * f * d["T"]
    W18 = WC.arm_weights(x, 18)
    for _ in range(4):
        ra, dec, psi, gmst = rng.uniform(0, 6.2), rng.uniform(-1.5, 1.5), rng.uniform(0, 3.1), 0.3
        b = OC.arm_coeffs(d["arm_x"], d["arm_y"], 18, ra, dec, psi, gmst)
        s, e1, e2 = O.sky_basis(ra, dec, gmst)
        p = math.cos(psi) * e1 + math.sin(psi) * e2
        q = -math.sin(psi) * e1 + math.cos(psi) * e2
        m = p - 1j * q
        ex, ey = (m @ d["arm_x"]) ** 2, (m @ d["arm_y"]) ** 2
        full = 0.5 * (WC.dhat(d["arm_x"] @ s, x) * ex - WC.dhat(d["arm_y"] @ s, x) * ey)
        assert np.max(np.abs(b @ W18 - full)) <= 1e-13
        # p_max = 0 misses the direction dependence by O(x) at the band edge
        assert np.max(np.abs(b[0] * W18[0] - full)) > 1e-3


def test_path_d_converges_to_saturation(arm6):
    point, exact, info, draws, logw = arm6
    half_dd = 0.5 * info["rho2"]
    gaps = []
    for p_max in (0, 2, 4, 6):
        pt_p = WC.comp_small(WC.FINITE_ARM, p_max, n_draws=8)[0]
        gaps.append(half_dd - OC.lnL(OC.CompPoint(pt_p), truth_draw(info))[0])
    assert gaps[0] > 1e-3 * half_dd * 1e-2
    assert all(g >= -1e-9 * half_dd for g in gaps)
    assert all(gaps[i + 1] < 0.1 * gaps[i] for i in range(3)), gaps
    assert gaps[-1] <= 1e-9 * half_dd
    lnl = OC.lnL(OC.CompPoint(point), draws)
    assert np.all(lnl <= half_dd * (1 + 1e-9))


# ------------------------------------------------------------ planted mistakes

SRC = os.path.join(os.path.dirname(OC.__file__), "composite.py")
MUTATIONS = {
    "no_postphase": ("out.append(Cp * np.exp(1j * n * omega * tk))", "out.append(Cp)"),
    "postphase_sign": ("out.append(Cp * np.exp(1j * n * omega * tk))",
                       "out.append(Cp * np.exp(-1j * n * omega * tk))"),
    "dft_sign": ("C0 = np.array([np.mean(F * np.exp(-1j * n * th))",
                 "C0 = np.array([np.mean(F * np.exp(1j * n * th))"),
    "drift_sign": ("mdt = np.array([-(delay(pos", "mdt = np.array([(delay(pos"),
    "factorial": ("np.convolve(C0, P) / math.factorial(p)",
                  "np.convolve(C0, P) / math.factorial(p + 1)"),
    "arm_power": ("0.5 * (ux ** j * ex - uy ** j * ey)", "0.5 * (ux ** (j + 1) * ex - uy ** (j + 1) * ey)"),
    "eps_conj": ("- 1j * (np.outer(p, q) + np.outer(q, p))", "+ 1j * (np.outer(p, q) + np.outer(q, p))"),
    "kron_order": ("c = np.kron(pt.coeffs(k, ra, dec, psi, tc), Y)",
                   "c = np.kron(Y, pt.coeffs(k, ra, dec, psi, tc))"),
}


def _load_variant(src_text, tag):
    d = tempfile.mkdtemp()
    path = os.path.join(d, f"composite_{tag}.py")
    with open(path, "w") as f:
        f.write(src_text)
    spec = importlib.util.spec_from_file_location(f"oracle._composite_{tag}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def _battery(mod):
    fails = []
    point, exact, info, draws, logw = WC.comp_small(WC.ROTATION, 0, n_draws=32)
    half_dd = 0.5 * info["rho2"]
    lt = mod.lnL(mod.CompPoint(point), truth_draw(info))[0]
    if abs(lt - half_dd) > 1e-9 * half_dd:
        fails.append("path_a_truth")
    d = WC.random_detectors_arms(np.random.default_rng(9), 1, 4.0e3)[0]
    ra, dec, psi, gmst, tc, om = 1.0, 0.4, 0.6, 2.0, 0.003, 0.7
    C = mod.rotation_coeffs(d["resp"], d["pos"], om, 2, ra, dec, psi, gmst, tc)
    tk = O.delay(d["pos"], ra, dec, gmst, tc)
    off = 0
    for p in range(3):
        n = np.arange(-(2 + p), 3 + p)
        Cp = C[off:off + len(n)] * np.exp(-1j * n * om * tk)
        off += len(n)
        th = 0.37
        F = O.antenna(d["resp"], ra, dec, psi, gmst + th)
        mdt = -(O.delay(d["pos"], ra, dec, gmst + th, tc) - tk)
        if abs(np.sum(Cp * np.exp(1j * n * th)) - F * mdt ** p / math.factorial(p)) > 1e-12 * 0.03 ** p:
            fails.append("identity")
            break
    b = mod.arm_coeffs(d["arm_x"], d["arm_y"], 2, ra, dec, psi, gmst)
    if abs(b[0] - O.antenna(d["resp"], ra, dec, psi, gmst)) > 1e-14:
        fails.append("arm_b0")
    pa = WC.comp_small(WC.FINITE_ARM, 6, n_draws=4)
    la = mod.lnL(mod.CompPoint(pa[0]), truth_draw(pa[2]))[0]
    if abs(la - 0.5 * pa[2]["rho2"]) > 1e-8 * pa[2]["rho2"]:
        fails.append("path_d_truth")
    return fails


def test_unmodified_oracle_passes_battery():
    with open(SRC) as f:
        text = f.read()
    assert _battery(_load_variant(text, "clean")) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, name
    fails = _battery(_load_variant(text.replace(old, new), name))
    assert fails, f"mutation {name} passed every pin"


@pytest.mark.parametrize("kind,p_max", [(WC.ROTATION, 0), (WC.ROTATION, 2), (WC.FINITE_ARM, 3)])
def test_oracle_gradient_against_central_differences(kind, p_max):
    """The chain-rule gradient against central differences of lnL itself, on
    draws whose arrival times stay inside one table interval over the steps
    (the cubic's slope is only continuous inside an interval)."""
    point, exact, info, draws, logw = WC.comp_small(kind, p_max, n_draws=48)
    pt = OC.CompPoint(point)
    lnl, g = OC.lnL_grad(pt, draws)
    assert np.allclose(lnl, OC.lnL(pt, draws), rtol=0, atol=1e-9 * np.max(np.abs(lnl)))
    steps = [1e-5, 1e-5, 1e-5, 1e-5, 1e-5, 1e-6, 1e-7]
    keep = np.ones(len(lnl), dtype=bool)
    for i in range(len(lnl)):
        for k in range(pt.K):
            tk = O.delay(pt.pos[k], draws["ra"][i], draws["dec"][i], pt.gmst, draws["t"][i])
            u = (tk - pt.t0[k]) / pt.dt
            fr = u - math.floor(u)
            if min(fr, 1 - fr) < 3e-3 or u < 2 or u > pt.n - 3:
                keep[i] = False
    assert keep.sum() >= 24
    scale = np.abs(g) + np.sqrt(np.mean(g ** 2, axis=0))
    for j, p in enumerate(W.PARAMS):
        up = {q: np.array(draws[q], dtype=float) for q in W.PARAMS}
        dn = {q: np.array(draws[q], dtype=float) for q in W.PARAMS}
        up[p] += steps[j]
        dn[p] -= steps[j]
        fd = (OC.lnL(pt, up) - OC.lnL(pt, dn)) / (2 * steps[j])
        err = (np.abs(fd - g[:, j]) / scale[:, j])[keep]
        assert err.max() <= 2e-6, (p, err.max())
