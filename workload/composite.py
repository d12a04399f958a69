"""Seeded inputs for the composite-index response of Sec. III (shared input only).

Like the rest of this package it produces inputs and evaluates no part of the
likelihood.  It builds

* detectors with their arm vectors and arm lengths (for the finite-arm case);
* analytic mode spectra h_lm(f) that can be evaluated at any frequency (the
  same spectral model as the static workloads), so that the elementary
  templates of eq. slowrot:master are exact: chi^(p,n)_lm(f) =
  (2 pi i f')^p h_lm(f'), f' = f - n Omega / 2 pi (a time derivative and a
  sidereal modulation of h_lm; Appendix B), and for finite arms
  chi^(p)_lm(f) = e^{-2 pi i f T} W_p(pi f T) h_lm(f) (eq. fsize:factorization);
* the tables Q, U, V of eq. slowrot:QUV over those banks, by the same discrete
  sums as the static tables;
* injections made without the composite expansion: for Earth rotation the
  detector sees F_k(t) h_Y(t - t_k) with F_k(t) the static antenna factor of
  the rotated Earth (its five sidereal harmonics taken by a DFT over the
  sidereal angle), placed first and then modulated, which is the ordering of
  eq. resp:strain:rot; for finite arms the full transfer function of eq.
  slowrot:armtransfer in the two-arm response of eq. fsize:FA.

Readings: the source direction in eq. fsize:bp and the arm transfer is the
unit vector towards the source; times are relative to the reference time
(t_ref = 0), and GMST(t) = gmst + Omega t.
"""
from __future__ import annotations

import math

import numpy as np

from . import (C_LIGHT, CE20_SITE, CE40_SITE, D_REF, ET_SITE, MODE_AMP, PARAMS, Prior,
               R_EARTH, _pol_tensors, _site_frame, _tensor, as_float, freq_grid,
               harmonic_for_injection, inner_weight, mixture_draws, proposal_sigma, q_table,
               seed_for, uv_matrices)

ROTATION = 1
FINITE_ARM = 2
OMEGA_EARTH = 7.2921159e-5  # rad/s


def detector_arms(lat, lon, azimuth, opening=math.pi / 2, arm_length=4.0e3):
    """Detector at (lat, lon) with its x-arm at `azimuth` (east towards north)
    and y-arm `opening` further round: position (light-seconds), response
    tensor (xx, xy, xz, yy, yz, zz), unit arm vectors and one-way light time."""
    up, east, north = _site_frame(lat, lon)
    xa = math.cos(azimuth) * east + math.sin(azimuth) * north
    ya = math.cos(azimuth + opening) * east + math.sin(azimuth + opening) * north
    D = 0.5 * (np.outer(xa, xa) - np.outer(ya, ya))
    return {"pos": up * R_EARTH / C_LIGHT,
            "resp": np.array([D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2]]),
            "arm_x": xa, "arm_y": ya, "T": arm_length / C_LIGHT}


def network_3g_arms(n_det: int):
    """ET triangle (10 km, 60-degree arms) + CE 40 km (+ CE 20 km) with arms."""
    lat, lon, az = ET_SITE
    dets = [detector_arms(lat, lon, az + i * 2 * math.pi / 3, math.pi / 3, 1.0e4)
            for i in range(3)]
    dets.append(detector_arms(*CE40_SITE, arm_length=4.0e4))
    dets.append(detector_arms(*CE20_SITE, arm_length=2.0e4))
    return dets[:n_det]


def random_detectors_arms(rng, n_det: int, arm_length: float):
    out = []
    for _ in range(n_det):
        lat = math.asin(rng.uniform(-1.0, 1.0))
        lon = rng.uniform(-math.pi, math.pi)
        az = rng.uniform(0.0, math.pi)
        out.append(detector_arms(lat, lon, az, arm_length=arm_length))
    return out


class ModeModel:
    """h_lm(f) = a_lm |f|^(-7/6) e^{i (c0 + c2 f^2)} on the band, m > 0 modes
    on f < 0, partners by h_{l,-m}(f) = (-1)^l conj h_lm(-f); callable at any
    frequencies.  `scale` multiplies every mode."""

    def __init__(self, rng, modes, f_low, f_max):
        self.modes = list(modes)
        self.f_low, self.f_max = f_low, f_max
        self.scale = 1.0
        self.par = {}
        for (l, m) in self.modes:
            if m > 0 or (l, -m) not in self.modes:
                amp = MODE_AMP.get(l, {}).get(abs(m), 0.1)
                self.par[(l, m)] = (amp, rng.uniform(0.0, 2 * math.pi),
                                    rng.uniform(-1.0, 1.0) * 2e-4)

    def _own(self, lm, f):
        amp, c0, c2 = self.par[lm]
        af = np.abs(f)
        side = (f < 0) if lm[1] > 0 else (f > 0)
        sel = (af >= self.f_low) & (af <= self.f_max) & side
        h = np.zeros(f.shape, dtype=np.complex128)
        h[sel] = amp * af[sel] ** (-7.0 / 6.0) * np.exp(1j * (c0 + c2 * af[sel] ** 2))
        return h

    def __call__(self, f):
        f = np.asarray(f, dtype=np.float64)
        out = []
        for (l, m) in self.modes:
            if (l, m) in self.par:
                out.append(self._own((l, m), f))
            else:
                out.append((-1) ** l * np.conj(self._own((l, -m), -f)))
        return self.scale * np.stack(out)


def rotation_bank(model, freq, omega, p_max):
    """chi^(p,n)_lm on the grid, composite order (p, n) then mode: [A][nf]."""
    rows = []
    for p in range(p_max + 1):
        for n in range(-(2 + p), 3 + p):
            fs = freq - n * omega / (2 * math.pi)
            rows.append((2j * math.pi * fs) ** p * model(fs))
    return np.concatenate(rows)


def _sinc(z):
    z = np.asarray(z, dtype=np.complex128)
    out = np.ones(z.shape, dtype=np.complex128)
    nz = np.abs(z) > 1e-8
    out[nz] = np.sin(z[nz]) / z[nz]
    small = ~nz
    out[small] = 1.0 - z[small] ** 2 / 6.0
    return out


def dhat(u, x):
    """Residual arm transfer D^(u, x) = e^{+2 pi i f T} D~ (eq. fsize:Dhat),
    u = arm . n, x = pi f T, from the two legs of eq. slowrot:armtransfer."""
    return 0.5 * (np.exp(1j * x * (1 - u)) * _sinc(x * (1 + u))
                  + np.exp(-1j * x * (1 + u)) * _sinc(x * (1 - u)))


def arm_weights(x, p_max, nodes=64):
    """W_p(x) = (1/p!) d^p D^/du^p at u = 0 (eq. fsize:Wp), p <= p_max, by the
    Cauchy integral over |u| = 1 (D^ is entire in u): [p_max + 1][len(x)]."""
    x = np.asarray(x, dtype=np.float64)
    phi = 2 * math.pi * np.arange(nodes) / nodes
    vals = np.stack([dhat(np.exp(1j * a), x) for a in phi])       # [nodes][nx]
    return np.stack([np.mean(vals * np.exp(-1j * p * phi)[:, None], axis=0)
                     for p in range(p_max + 1)])


def arm_bank(model, freq, T, p_max):
    """chi^(p)_lm = e^{-2 pi i f T} W_p(pi f T) h_lm(f): [A][nf], a = p major."""
    W = arm_weights(math.pi * freq * T, p_max)
    h = model(freq)
    shift = np.exp(-2j * math.pi * freq * T)
    return np.concatenate([W[p][None, :] * shift[None, :] * h for p in range(p_max + 1)])


def _hY(model, f, truth):
    Y = np.array([harmonic_for_injection(l, m, truth["incl"], truth["phase"])
                  for (l, m) in model.modes])
    return np.tensordot(Y, model(f), axes=1)


def _real_strain(hk):
    """FT of Re h(t) from the FT of the complex h(t) on a symmetric grid."""
    return 0.5 * (hk + np.conj(hk[::-1]))


def inject_rotation(dets, model, freq, truth, gmst, d_ref, omega):
    """d_k(f) for h_k(t) = Re[F_k(t) h_Y(t - t_k)] on the rotating Earth
    (eq. resp:strain:rot with the delay held at its reference-time value):
    the five sidereal harmonics F_k(t) = sum_n C_n e^{i n Omega t} are taken by
    a DFT of the static antenna factor over the sidereal angle, and each
    modulates the template already placed at t_k."""
    x = d_ref / math.exp(truth["lnD"])
    th = 2 * math.pi * np.arange(8) / 8
    out, arrival = [], []
    src, _, _ = _pol_tensors(truth["ra"], truth["dec"], truth["psi"], gmst)
    for det in dets:
        D = _tensor(det["resp"])
        F = []
        for a in th:
            _, e_plus, e_cross = _pol_tensors(truth["ra"], truth["dec"], truth["psi"], gmst + a)
            F.append(np.sum(D * e_plus) + 1j * np.sum(D * e_cross))
        F = np.array(F)
        tk = truth["t"] - float(det["pos"] @ src)
        arrival.append(tk)
        hk = np.zeros(freq.shape, dtype=np.complex128)
        for n in range(-2, 3):
            Cn = np.mean(F * np.exp(-1j * n * th))
            fs = freq - n * omega / (2 * math.pi)
            # FT of e^{i n Omega t} g(t - t_k) at f is FT[g](f') e^{-2 pi i f' t_k}
            hk += Cn * np.exp(-2j * math.pi * fs * tk) * _hY(model, fs, truth)
        out.append(_real_strain(x * hk))
    return np.stack(out), np.array(arrival)


def inject_arms(dets, model, freq, truth, gmst, d_ref):
    """d_k(f) with the full two-arm response of eq. fsize:FA, each arm through
    the transfer function of eq. slowrot:armtransfer (no expansion in u)."""
    x = d_ref / math.exp(truth["lnD"])
    src, e_plus, e_cross = _pol_tensors(truth["ra"], truth["dec"], truth["psi"], gmst)
    eps = e_plus + 1j * e_cross            # eps_+ - i eps_x in the sign of the static injection
    hY = _hY(model, freq, truth)
    out, arrival = [], []
    for det in dets:
        T = det["T"]
        xa, ya = det["arm_x"], det["arm_y"]
        trans = np.exp(-2j * math.pi * freq * T)
        Dx = trans * dhat(float(xa @ src), math.pi * freq * T)
        Dy = trans * dhat(float(ya @ src), math.pi * freq * T)
        Ff = 0.5 * (Dx * (xa @ eps @ xa) - Dy * (ya @ eps @ ya))
        tk = truth["t"] - float(det["pos"] @ src)
        arrival.append(tk)
        out.append(_real_strain(x * Ff * hY * np.exp(-2j * math.pi * freq * tk)))
    return np.stack(out), np.array(arrival)


def make_comp_point(*, kind, p_max, dets, modes, f_low, f_max, df, rate, half_window, snr,
                    truth, gmst, d_ref, rng, omega=OMEGA_EARTH, q_dtype=np.complex128):
    """One composite point: widened Q, U, V (composite index A = a M + i),
    geometry, the response description, and the injection's bookkeeping.  The
    table has an odd length centred on each detector's injected arrival time,
    so that the injection sits on a table sample."""
    freq = freq_grid(f_max, df)
    K = len(dets)
    model = ModeModel(rng, modes, f_low, f_max)
    wgt = inner_weight(freq, df, f_low, f_max, K)
    if kind == ROTATION:
        dk, arrival = inject_rotation(dets, model, freq, truth, gmst, d_ref, omega)
    else:
        dk, arrival = inject_arms(dets, model, freq, truth, gmst, d_ref)
    rho2 = float(np.sum(wgt * np.abs(dk) ** 2))
    scale = snr / math.sqrt(rho2)
    model.scale = scale
    dk = dk * scale
    dt = 1.0 / rate
    n = 2 * int(math.ceil(half_window * rate)) + 1
    t0 = arrival - 0.5 * (n - 1) * dt
    if kind == ROTATION:
        bank = rotation_bank(model, freq, omega, p_max)
        Q = q_table(wgt, bank, dk, freq, df, t0, dt, n)
        U, V = uv_matrices(wgt, bank)
    else:
        Qs, Us, Vs = [], [], []
        for k, det in enumerate(dets):
            bank = arm_bank(model, freq, det["T"], p_max)
            Qs.append(q_table(wgt[k:k + 1], bank, dk[k:k + 1], freq, df, t0[k:k + 1], dt, n)[0])
            u, v = uv_matrices(wgt[k:k + 1], bank)
            Us.append(u[0])
            Vs.append(v[0])
        Q, U, V = np.stack(Qs), np.stack(Us), np.stack(Vs)
    point = {
        "K": K, "M": len(modes), "kind": kind, "p_max": p_max,
        "ell": np.array([lm[0] for lm in modes], dtype=np.int32),
        "em": np.array([lm[1] for lm in modes], dtype=np.int32),
        "Q": Q.astype(q_dtype), "q_t0": t0, "q_dt": dt, "U": U, "V": V,
        "det_pos": np.stack([d["pos"] for d in dets]),
        "det_resp": np.stack([d["resp"] for d in dets]),
        "arm_x": np.stack([d["arm_x"] for d in dets]),
        "arm_y": np.stack([d["arm_y"] for d in dets]),
        "omega": float(omega), "gmst": float(gmst), "d_ref": float(d_ref),
    }
    info = {"snr": snr, "rho2": float(np.sum(wgt * np.abs(dk) ** 2)), "arrival": arrival,
            "truth": dict(truth), "modes": list(modes), "hk": dk}
    exact = {"freq": freq, "wgt": wgt, "dk": dk, "model": model}
    return point, exact, info


def _truth(rng):
    return {"ra": rng.uniform(0.3, 2 * math.pi - 0.3), "dec": rng.uniform(-1.0, 1.0),
            "psi": rng.uniform(0.2, math.pi - 0.2), "incl": rng.uniform(0.5, 1.3),
            "phase": rng.uniform(0.3, 2 * math.pi - 0.3), "lnD": math.log(D_REF), "t": 0.0}


MODES4 = [(2, 2), (2, -2), (3, 3), (3, -3)]


def comp_small(kind: int, p_max: int, n_draws: int = 2048, omega: float = 2.0,
               snr: float = 20.0):
    """Small composite point that the oracle evaluates in seconds: two seeded
    detectors, modes (2,+-2), (3,+-3) on 20-1024 Hz (rotation) or 20-2048 Hz
    (40 km arms), df 0.25 Hz, table at 8192 Hz over +-25 ms, zero noise; draws
    from the defensive mixture about the injection, float64.  Rotation uses a
    stress sidereal rate (omega rad/s) so that the modulation over the signal
    is large."""
    config = 10 + kind
    rng = np.random.default_rng(seed_for(config, 0))
    gmst = rng.uniform(0, 2 * math.pi)
    truth = _truth(rng)
    if kind == ROTATION:
        dets = random_detectors_arms(rng, 2, 4.0e3)
        f_max = 1024.0
    else:
        dets = random_detectors_arms(rng, 2, 4.0e4)
        f_max = 2048.0
    point, exact, info = make_comp_point(
        kind=kind, p_max=p_max, dets=dets, modes=MODES4, f_low=20.0, f_max=f_max, df=0.25,
        rate=8192.0, half_window=0.025, snr=snr, truth=truth, gmst=gmst, d_ref=D_REF, rng=rng,
        omega=omega)
    prior = Prior(0.5 * D_REF, 2.0 * D_REF, 0.01)
    sig = proposal_sigma(info, exact)
    draws, logw = mixture_draws(np.random.default_rng(seed_for(config, 1)), prior, truth, sig,
                                n_draws)
    info["sigma"] = sig
    return point, exact, info, as_float(draws, np.float64), logw


def comp_3g(kind: int, p_max: int, n_draws: int = 1 << 22, omega: float = OMEGA_EARTH):
    """3G-network composite workload: ET triangle + CE 40 km (K = 4), the ten
    modes on 5-2048 Hz, SNR 600, zero noise, complex128 tables at 32768 Hz over
    +-20 ms, float32 draws from the defensive mixture."""
    config = 20 + kind
    rng = np.random.default_rng(seed_for(config, 0))
    gmst = rng.uniform(0, 2 * math.pi)
    truth = _truth(rng)
    from . import MODES10
    point, exact, info = make_comp_point(
        kind=kind, p_max=p_max, dets=network_3g_arms(4), modes=MODES10, f_low=5.0, f_max=2048.0,
        df=0.25, rate=32768.0, half_window=0.02, snr=600.0, truth=truth, gmst=gmst,
        d_ref=D_REF, rng=rng, omega=omega)
    prior = Prior(0.5 * D_REF, 2.0 * D_REF, 0.01)
    sig = proposal_sigma(info, exact)
    draws, logw = mixture_draws(np.random.default_rng(seed_for(config, 1)), prior, truth, sig,
                                n_draws)
    return point, exact, info, as_float(draws, np.float32), logw.astype(np.float32)


__all__ = ["ROTATION", "FINITE_ARM", "OMEGA_EARTH", "comp_small", "comp_3g", "make_comp_point",
           "arm_weights", "dhat", "rotation_bank", "arm_bank", "ModeModel", "PARAMS"]
