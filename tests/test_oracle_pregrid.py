"""Pins of the reflected-series pregrid oracle (eq. q-time-pregrid,
eq. ap:q-pregrid-rate, eq. ap:q-pregrid-accuracy), against things other than
itself:

* the fine table passes through the native samples (a band-limited
  interpolant must);
* it is exact, at every fine sample, for the series the reflection extends
  periodically without a kink: sums of cos(pi k (j + 1/2) / n), k < n, whose
  continuous form is known in closed form;
* on a band-limited wave packet evaluated exactly (a direct Fourier sum),
  the four-point cubic read from the fine table has an error that falls by
  about 16 per doubling of r (the fourth-order law of eq. ap:q-pregrid-accuracy);
* planted mistakes (no reflection, negative frequencies misplaced, wrong
  scale, reflection shifted by one sample) each fail one of these.
"""
import os

import numpy as np
import pytest

import oracle as O
import oracle.precompute as OP


def reflection_basis(n, r, rng, n_terms=None):
    """(native [1][n][2], exact fine values [1][r(n-1)+1][2]) of
    sum_k a_k cos(pi k (x + 1/2) / n), k < n, with complex a_k."""
    ks = np.arange(n if n_terms is None else n_terms)
    a = rng.standard_normal((len(ks), 2)) + 1j * rng.standard_normal((len(ks), 2))
    def at(x):
        return np.cos(np.pi * np.outer(x + 0.5, ks) / n) @ a
    native = at(np.arange(n, dtype=np.float64))[None]
    fine = at(np.arange(r * (n - 1) + 1) / r)[None]
    return native, fine, np.sum(np.abs(a))


def packet(times, fc=600.0, width=250.0, tc=0.0013, fmax=2040.0, df=1.0):
    """A band-limited wave packet Q(t) = sum_f c(f) e^{2 pi i f t} with a
    Gaussian spectral envelope (two modes with different centres), evaluated
    by the direct sum: [len(times)][2]."""
    f = np.arange(-fmax, fmax + df / 2, df)
    c1 = np.exp(-0.5 * ((f - fc) / width) ** 2) * np.exp(-2j * np.pi * f * tc)
    c2 = 0.5 * np.exp(-0.5 * ((f + 1.5 * fc) / width) ** 2) * np.exp(-2j * np.pi * f * (tc - 4e-4))
    E = np.exp(2j * np.pi * np.outer(times, f))
    return np.stack([E @ c1, E @ c2], axis=1)


def pregrid_battery(fn):
    """The pins as a battery: names of those that fail for pregrid function fn."""
    failed = []
    rng = np.random.default_rng(7)
    q = rng.standard_normal((2, 37, 3)) + 1j * rng.standard_normal((2, 37, 3))
    for r in (1, 4, 8):
        fine = fn(q, r)
        if fine.shape != (2, r * 36 + 1, 3) or not np.max(np.abs(fine[:, ::r, :] - q)) < 1e-13 * np.max(np.abs(q)):
            failed.append("native_samples")
            break
    for n, r in ((16, 8), (37, 4), (5, 16)):
        native, exact, scale = reflection_basis(n, r, rng)
        if not np.max(np.abs(fn(native, r) - exact)) < 1e-12 * scale:
            failed.append("reflection_basis")
            break
    return failed


def test_pregrid_passes_battery():
    assert pregrid_battery(OP.q_pregrid) == []


def test_pregrid_fine_rate_of_the_paper():
    """A 4096 Hz native table over +-20 ms refined by r = 8: 32 768 Hz fine
    samples (eq. ap:q-pregrid-rate), spanning the same window."""
    n = 165  # 4096 Hz over [-20 ms, +20 ms]
    h = 1.0 / 4096.0
    fine = OP.q_pregrid(np.zeros((1, n, 1), dtype=np.complex128), 8)
    assert fine.shape[1] == 8 * (n - 1) + 1
    assert abs(1.0 / (h / 8) - 32768.0) < 1e-9
    assert abs((fine.shape[1] - 1) * h / 8 - (n - 1) * h) < 1e-15


def test_cubic_error_falls_16x_per_doubling_of_r():
    """eq. ap:q-pregrid-accuracy: the four-point cubic on the fine table has an
    error ~ (2 pi f dt_Q)^4, so each doubling of r cuts it by ~16, until the
    reflection's own error (tiny for a packet that has decayed at the window
    edges) takes over."""
    rate, half = 4096.0, 0.02
    t0 = -half
    n = int(round(2 * half * rate)) + 1
    native = packet(t0 + np.arange(n) / rate)[None]           # [1][n][2]
    rng = np.random.default_rng(3)
    ts = rng.uniform(-0.008, 0.008, 400)
    exact = packet(ts)
    errs = {}
    for r in (4, 8, 16, 32):
        fine = OP.q_pregrid(native, r)[0]
        got = np.array([O.qinterp(fine, t0, 1.0 / (rate * r), t)[0] for t in ts])
        errs[r] = np.max(np.abs(got - exact)) / np.max(np.abs(exact))
    for r in (4, 8):
        assert 12.0 < errs[r] / errs[2 * r] < 20.0, errs
    # at r = 32 the cubic's share (~6e-8) meets the floor of the native
    # window's own error (~1e-7): the fall slows there, as the paper says
    assert errs[16] / errs[32] > 4.0 and errs[32] < 2e-7, errs


MUTATIONS = {
    "no_reflection": ("refl = np.concatenate([q, q[:, ::-1, :]], axis=1)",
                      "refl = np.concatenate([q, q], axis=1)"),
    "negative_frequencies_misplaced": ("Y[:, L - n + 1:, :] = X[:, n + 1:, :]",
                                       "Y[:, n + 1:2 * n, :] = X[:, n + 1:, :]"),
    "wrong_scale": ("y = np.fft.ifft(Y, axis=1) * (L / N)", "y = np.fft.ifft(Y, axis=1) * L"),
    "reflection_shifted": ("refl = np.concatenate([q, q[:, ::-1, :]], axis=1)",
                           "refl = np.concatenate([q, q[:, -2::-1, :], q[:, -1:, :]], axis=1)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(OP.__file__).read()
    assert src.count(old) == 1, name
    ns = {}
    exec(compile(src.replace(old, new), os.path.basename(OP.__file__), "exec"), ns)
    assert pregrid_battery(ns["q_pregrid"]), f"planted mistake {name} passed every pin"
