"""Pins of the Q/U/V oracle (eq. QUV as plain sums), against things other
than itself:

* the direct Fourier sums equal the workloads' table builder, which gets the
  same table by one zero-padded inverse FFT per (detector, mode) (eq.
  q-time-pregrid's pregrid), to rounding;
* U is Hermitian and positive semi-definite, V complex symmetric;
* with noise-free data the factored likelihood assembled from these products
  (oracle antenna factor, harmonics and delays) equals rho^2/2 at the
  injection, and the quadratic term alone equals rho^2/4 x 2 = <h|h>/2;
* planted mistakes (dropped conjugate, time sign, missing reflection in V)
  each fail one of these.
"""
import importlib.util
import math
import os
import sys
import tempfile

import numpy as np
import pytest

import oracle as O
import oracle.precompute as OP
import workload as W


def small_point():
    rng = np.random.default_rng(41)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:4], f_low=20.0, f_max=512.0, df=0.5, rate=4096.0,
        half_window=0.02, snr=30.0, truth=truth, gmst=0.4, d_ref=100.0, rng=rng, noise=False,
        q_dtype=np.complex128)
    return point, exact, info


FIX = small_point()


def physical_lnl(point, exact, info, qfun, uvfun):
    """lnL at the injection from products computed by qfun / uvfun."""
    tr = info["truth"]
    U, V = uvfun(exact["wgt"], exact["hlm"])
    x = point["d_ref"] / math.exp(tr["lnD"])
    Y = np.array([O.sylm(-2, l, m, tr["incl"], tr["phase"])
                  for l, m in zip(point["ell"], point["em"])])
    td = tq = 0.0
    for k in range(point["K"]):
        F = O.antenna(point["det_resp"][k], tr["ra"], tr["dec"], tr["psi"], point["gmst"])
        tk = O.delay(point["det_pos"][k], tr["ra"], tr["dec"], point["gmst"], tr["t"])
        Q = qfun(exact["freq"], exact["wgt"][k], exact["hlm"], exact["dk"][k], [tk])[0]
        td += x * np.real(np.conj(F) * np.vdot(Y, Q))
        tq += 0.25 * x * x * (abs(F) ** 2 * np.real(np.conj(Y) @ U[k] @ Y)
                              + np.real(F * F * (Y @ V[k] @ Y)))
    return td - tq, tq


def test_direct_sum_equals_fft_table():
    point, exact, info = FIX
    n = point["Q"].shape[1]
    Qd = OP.q_table_direct(exact["freq"], exact["wgt"], exact["hlm"], exact["dk"],
                           point["q_t0"], point["q_dt"], n)
    Qf = np.asarray(point["Q"])
    assert np.max(np.abs(Qd - Qf)) <= 1e-12 * np.max(np.abs(Qf))


def test_uv_symmetries_and_fixture():
    point, exact, info = FIX
    U, V = OP.uv_direct(exact["wgt"], exact["hlm"])
    s = np.max(np.abs(U))
    assert np.max(np.abs(U - np.conj(np.transpose(U, (0, 2, 1))))) <= 1e-14 * s
    assert np.max(np.abs(V - np.transpose(V, (0, 2, 1)))) <= 1e-14 * s
    for k in range(U.shape[0]):
        assert np.min(np.linalg.eigvalsh(U[k])) >= -1e-12 * s
    assert np.max(np.abs(U - point["U"])) <= 1e-13 * s
    assert np.max(np.abs(V - point["V"])) <= 1e-13 * s


def test_noise_free_injection_gives_half_rho2():
    point, exact, info = FIX
    lnl, tq = physical_lnl(point, exact, info, OP.q_direct, OP.uv_direct)
    rho2 = info["rho2"]
    assert abs(lnl - 0.5 * rho2) <= 1e-10 * rho2
    assert abs(tq - 0.5 * rho2) <= 1e-10 * rho2


SRC = os.path.join(os.path.dirname(OP.__file__), "precompute.py")
MUTATIONS = {
    "q_no_conj": ("* np.conj(np.asarray(hlm)) *", "* np.asarray(hlm) *"),
    "q_time_sign": ("np.exp(2j * np.pi * np.outer(t, freq))", "np.exp(-2j * np.pi * np.outer(t, freq))"),
    "v_no_reflection": ("hm = hlm[:, ::-1]", "hm = hlm"),
    "u_no_conj": ("np.sum(wgt[k] * np.conj(hlm[i]) * hlm[j])", "np.sum(wgt[k] * hlm[i] * hlm[j])"),
}


def _load(text, tag):
    d = tempfile.mkdtemp()
    path = os.path.join(d, f"precompute_{tag}.py")
    with open(path, "w") as f:
        f.write(text)
    spec = importlib.util.spec_from_file_location(f"oracle._precompute_{tag}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def _battery(mod):
    point, exact, info = FIX
    fails = []
    n = 16
    Qd = mod.q_table_direct(exact["freq"], exact["wgt"], exact["hlm"], exact["dk"],
                            point["q_t0"], point["q_dt"], n)
    if np.max(np.abs(Qd - np.asarray(point["Q"])[:, :n])) > 1e-12 * np.max(np.abs(point["Q"])):
        fails.append("fft")
    lnl, tq = physical_lnl(point, exact, info, mod.q_direct, mod.uv_direct)
    if abs(lnl - 0.5 * info["rho2"]) > 1e-10 * info["rho2"]:
        fails.append("physical")
    return fails


def test_unmodified_passes():
    with open(SRC) as f:
        assert _battery(_load(f.read(), "clean")) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1
    assert _battery(_load(text.replace(old, new), name)), name


def test_rotation_bank_round_trip_is_exact_for_a_compact_pulse():
    """For a Gaussian pulse well inside the grid's period the DFT round trip
    of the bank construction reproduces the analytic spectra of
    e^{i n Omega t} d^p h/dt^p: (2 pi i f')^p h(f'), f' = f - n Omega / 2 pi."""
    df, fmax, sig, om = 0.25, 64.0, 0.05, 3.0
    freq = W.freq_grid(fmax, df)
    def pulse(f, t0=0.2, phase=0.7):
        return np.exp(-0.5 * (2 * np.pi * f * sig) ** 2 - 2j * np.pi * f * t0 + 1j * phase)
    h = np.stack([pulse(freq), pulse(freq, -0.3, 1.9)])
    bank = OP.rotation_bank_fft(h, df, om, 2)
    rows = []
    for p in range(3):
        for n in range(-(2 + p), 3 + p):
            fs = freq - n * om / (2 * np.pi)
            rows.append(np.stack([(2j * np.pi * fs) ** p * pulse(fs),
                                  (2j * np.pi * fs) ** p * pulse(fs, -0.3, 1.9)]))
    ref = np.concatenate(rows)
    assert bank.shape == ref.shape
    assert np.max(np.abs(bank - ref)) <= 1e-12 * np.max(np.abs(ref))
    # no modulation: the identity (up to the derivative weights)
    b0 = OP.rotation_bank_fft(h, df, 0.0, 0)
    assert np.max(np.abs(b0[4:6] - h)) <= 1e-14


def test_arm_weights_series():
    """W_0 = sinc(x) cos x; the series in u sums back to the two-leg transfer
    function for |u| <= 1; the arm bank at p_max = 0 is the tapered,
    delayed mode."""
    x = np.linspace(-1.2, 1.2, 25)
    W = OP.arm_weights_series(x, 30)
    assert np.max(np.abs(W[0] - np.sinc(x / np.pi) * np.cos(x))) <= 1e-14
    for u in (-1.0, -0.4, 0.3, 0.9):
        def sinc(z):
            return np.where(np.abs(z) < 1e-12, 1.0 + 0j, np.sin(z + 0j) / np.where(z == 0, 1, z))
        full = 0.5 * (np.exp(1j * x * (1 - u)) * sinc(x * (1 + u))
                      + np.exp(-1j * x * (1 + u)) * sinc(x * (1 - u)))
        assert np.max(np.abs(np.tensordot(u ** np.arange(31), W, axes=1) - full)) <= 1e-13
    freq = np.arange(-8, 9) * 0.5
    h = np.exp(1j * freq)[None, :]
    b = OP.arm_bank(h, 0.5, 1e-4, 0)
    xx = np.pi * freq * 1e-4
    assert np.max(np.abs(b[0] - np.sinc(xx / np.pi) * np.cos(xx) * np.exp(-2j * np.pi * freq * 1e-4) * h[0])) <= 1e-15
