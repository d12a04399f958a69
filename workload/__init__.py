"""Seeded synthetic workloads for the extrinsic likelihood (shared input only).

This module is the only code that the CUDA path and the oracle both use.  It
produces inputs; it does not evaluate the likelihood, the harmonics used by
the likelihood, or any lnZ reduction.  What it does:

* builds detector networks: seeded L-shaped detectors on a spherical Earth,
  an ET-like co-located 60-degree triangle and CE-like L detectors;
* builds synthetic mode spectra h_lm(f) (amplitude a_lm |f|^(-7/6), seeded
  quadratic phase; m > 0 modes on f < 0 and h_{l,-m}(f) = (-1)^l conj h_lm(-f));
* simulates the strain each detector records for an injected source, as the
  projection of the strain tensor h_+ e^+ + h_x e^x onto the detector tensor,
  time-shifted to the detector (the data model of eqs. strain and strain_mode
  and of h_k = Re[F_k h(t - t_k)]), plus optional coloured Gaussian noise;
* precomputes Q_{k,lm}(t) on a uniform fine table by an exact inverse FFT of
  the frequency-domain sum of eq. QUV, and U_k, V_k by the same discrete sums;
* draws extrinsic samples from the prior or from a defensive mixture
  0.1 prior + 0.9 Gaussian about the injection, with ln p - ln q.

The workloads stand in for the paper's 3G injections (no waveform model,
noise curve or strain data is available); the recipe is stated in the design
notes and in the config builders below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

C_LIGHT = 299_792_458.0          # m/s
R_EARTH = 6.371e6                # m
PARAMS = ("ra", "dec", "psi", "incl", "phase", "lnD", "t")

MODES10 = [(2, 2), (2, -2), (2, 1), (2, -1), (3, 3), (3, -3), (3, 2), (3, -2), (4, 4), (4, -4)]
MODE_AMP = {2: {2: 1.0, 1: 0.3}, 3: {3: 0.3, 2: 0.1}, 4: {4: 0.1}}


def seed_for(config: int, stream: int) -> int:
    """Seeds of the stated recipe: 37393 + 100 config + stream."""
    return 37393 + 100 * config + stream


# ------------------------------------------------------------------ detectors

def _site_frame(lat: float, lon: float):
    up = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.array([-math.sin(lat) * math.cos(lon), -math.sin(lat) * math.sin(lon),
                      math.cos(lat)])
    return up, east, north


def detector(lat: float, lon: float, azimuth: float, opening: float = math.pi / 2):
    """(position in light-seconds, response tensor xx,xy,xz,yy,yz,zz) of a
    detector at (lat, lon) whose x-arm points at `azimuth` (from east towards
    north) and whose y-arm is `opening` further round; D = (xx^T - yy^T)/2."""
    up, east, north = _site_frame(lat, lon)
    xa = math.cos(azimuth) * east + math.sin(azimuth) * north
    ya = math.cos(azimuth + opening) * east + math.sin(azimuth + opening) * north
    D = 0.5 * (np.outer(xa, xa) - np.outer(ya, ya))
    pos = up * R_EARTH / C_LIGHT
    return pos, np.array([D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2]])


def et_triangle(lat: float, lon: float, azimuth: float):
    """Three co-located detectors with 60-degree arms, rotated by 120 degrees."""
    return [detector(lat, lon, azimuth + i * 2 * math.pi / 3, math.pi / 3) for i in range(3)]


ET_SITE = (math.radians(40.5), math.radians(9.4), math.radians(20.0))
CE40_SITE = (math.radians(46.5), math.radians(-119.4), math.radians(36.0))
CE20_SITE = (math.radians(30.6), math.radians(-90.8), math.radians(-18.0))


def network_3g(n_det: int):
    """ET triangle + CE 40 km (+ CE 20 km): the 3G networks of the configs."""
    dets = et_triangle(*ET_SITE) + [detector(*CE40_SITE), detector(*CE20_SITE)]
    return dets[:n_det]


def random_l_detectors(rng: np.random.Generator, n_det: int):
    out = []
    for _ in range(n_det):
        lat = math.asin(rng.uniform(-1.0, 1.0))
        lon = rng.uniform(-math.pi, math.pi)
        az = rng.uniform(0.0, math.pi)
        out.append(detector(lat, lon, az))
    return out


# ---------------------------------------------------------------- spectra

def psd(f: np.ndarray) -> np.ndarray:
    """S(f) = (f/100)^-4 + 1 + (f/100)^2, evaluated at |f|."""
    a = np.abs(f) / 100.0
    with np.errstate(divide="ignore"):
        return a ** -4 + 1.0 + a ** 2


def freq_grid(f_max: float, df: float) -> np.ndarray:
    n = int(math.ceil(f_max / df))
    return np.arange(-n, n + 1) * df


def mode_spectra(rng: np.random.Generator, modes, freq, f_low, f_max):
    """h_lm(f) on the two-sided grid.  m > 0 modes occupy f < 0; a negative-m
    mode is the reflection of its positive partner when that partner is in the
    list, and is drawn on its own (on f > 0) otherwise."""
    band = (np.abs(freq) >= f_low) & (np.abs(freq) <= f_max)
    out = {}
    for (l, m) in modes:
        if m > 0 or (l, -m) not in modes:
            amp = MODE_AMP.get(l, {}).get(abs(m), 0.1)
            c0 = rng.uniform(0.0, 2 * math.pi)
            c2 = rng.uniform(-1.0, 1.0) * 2e-4
            af = np.abs(freq)
            h = np.zeros(freq.shape, dtype=np.complex128)
            side = (freq < 0) if m > 0 else (freq > 0)
            sel = band & side
            with np.errstate(divide="ignore"):
                h[sel] = amp * af[sel] ** (-7.0 / 6.0) * np.exp(1j * (c0 + c2 * af[sel] ** 2))
            out[(l, m)] = h
    for (l, m) in modes:
        if (l, m) not in out:
            partner = out[(l, -m)]
            out[(l, m)] = (-1) ** l * np.conj(partner[::-1])
    return np.stack([out[lm] for lm in modes])


# ------------------------------------------------------- independent injection

def wigner_d(l: int, mp: int, m: int, beta: float) -> float:
    """Wigner small-d d^l_{m' m}(beta), explicit factorial sum (injection only)."""
    tot = 0.0
    for s in range(0, 2 * l + 1):
        a, b, c, d = l + m - s, s, mp - m + s, l - mp - s
        if min(a, b, c, d) < 0:
            continue
        num = math.sqrt(math.factorial(l + mp) * math.factorial(l - mp) *
                        math.factorial(l + m) * math.factorial(l - m))
        den = math.factorial(a) * math.factorial(b) * math.factorial(c) * math.factorial(d)
        tot += ((-1) ** (mp - m + s)) * num / den * \
            math.cos(beta / 2) ** (2 * l + m - mp - 2 * s) * math.sin(beta / 2) ** (mp - m + 2 * s)
    return tot


def harmonic_for_injection(l: int, m: int, incl: float, phase: float) -> complex:
    """-2Y_lm = sqrt((2l+1)/4pi) d^l_{m,2}(incl) e^{i m phase} (injection only)."""
    return math.sqrt((2 * l + 1) / (4 * math.pi)) * wigner_d(l, m, 2, incl) * \
        complex(math.cos(m * phase), math.sin(m * phase))


def _pol_tensors(ra, dec, psi, gmst):
    lam = ra - gmst
    src = np.array([math.cos(dec) * math.cos(lam), math.cos(dec) * math.sin(lam), math.sin(dec)])
    east = np.array([-math.sin(lam), math.cos(lam), 0.0])
    north = np.array([-math.sin(dec) * math.cos(lam), -math.sin(dec) * math.sin(lam),
                      math.cos(dec)])
    p = math.cos(psi) * east + math.sin(psi) * north
    q = -math.sin(psi) * east + math.cos(psi) * north
    e_plus = np.outer(p, p) - np.outer(q, q)
    # cross tensor with the sign that makes h_k = Re[(F_+ - i F_x)(h_+ - i h_x)]
    e_cross = -(np.outer(p, q) + np.outer(q, p))
    return src, e_plus, e_cross


def _tensor(resp6):
    xx, xy, xz, yy, yz, zz = resp6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def inject(dets, modes, hlm, freq, truth, gmst, d_ref):
    """Frequency-domain strain of each detector for the injected source."""
    x = d_ref / math.exp(truth["lnD"])
    hY = np.zeros(freq.shape, dtype=np.complex128)
    for i, (l, m) in enumerate(modes):
        hY += harmonic_for_injection(l, m, truth["incl"], truth["phase"]) * hlm[i]
    hY *= x
    hY_ref = np.conj(hY[::-1])                      # FT of conj(h_Y) at f
    h_plus = 0.5 * (hY + hY_ref)                    # h_+ = Re h_Y
    h_cross = 0.5j * (hY - hY_ref)                  # h_x = -Im h_Y
    src, e_plus, e_cross = _pol_tensors(truth["ra"], truth["dec"], truth["psi"], gmst)
    out = []
    arrival = []
    for pos, resp in dets:
        D = _tensor(resp)
        fp = float(np.sum(D * e_plus))
        fc = float(np.sum(D * e_cross))
        tk = truth["t"] - float(pos @ src)
        arrival.append(tk)
        out.append((fp * h_plus + fc * h_cross) * np.exp(-2j * math.pi * freq * tk))
    return np.stack(out), np.array(arrival)


def colored_noise(rng, freq, df, n_det):
    """Gaussian noise with E[<n|a>^2] = <a|a>: n(f) = sqrt(S/4df)(g1 + i g2)
    for f > 0 and n(-f) = conj n(f)."""
    noise = np.zeros((n_det, freq.shape[0]), dtype=np.complex128)
    pos = freq > 0
    sig = np.sqrt(psd(freq[pos]) / (4.0 * df))
    for k in range(n_det):
        g = rng.standard_normal(pos.sum()) + 1j * rng.standard_normal(pos.sum())
        noise[k, pos] = sig * g
        noise[k] = noise[k] + np.conj(noise[k][::-1]) * (freq < 0)[:]
    return noise


# -------------------------------------------------------------- Q, U, V

def inner_weight(freq, df, f_low, f_max, n_det):
    band = (np.abs(freq) >= f_low) & (np.abs(freq) <= f_max)
    w = np.where(band, 2.0 * df / np.where(band, psd(freq), 1.0), 0.0)
    return np.tile(w, (n_det, 1))


def q_table(wgt, hlm, dk, freq, df, t0, dt, n):
    """Q_{k,lm}(t0_k + j dt), j < n, by inverse FFT of the discrete sum of
    eq. QUV (exact: the grid spacing df and dt fit an integer FFT length)."""
    nfft = int(round(1.0 / (df * dt)))
    assert abs(nfft * df * dt - 1.0) < 1e-9, "1/(df dt) must be an integer"
    assert nfft >= n and nfft > freq.shape[0]
    idx = np.round(freq / df).astype(np.int64) % nfft
    K, M = dk.shape[0], hlm.shape[0]
    Q = np.empty((K, n, M), dtype=np.complex128)
    for k in range(K):
        shift = np.exp(2j * math.pi * freq * t0[k])
        for i in range(M):
            X = np.zeros(nfft, dtype=np.complex128)
            np.add.at(X, idx, wgt[k] * np.conj(hlm[i]) * dk[k] * shift)
            Q[k, :, i] = nfft * np.fft.ifft(X)[:n]
    return Q


def uv_matrices(wgt, hlm):
    """U_{k,ij} = sum_n W conj h_i h_j;  V_{k,ij} = sum_n W h_i(-f) h_j(f)."""
    U = np.einsum("kn,in,jn->kij", wgt, np.conj(hlm), hlm)
    V = np.einsum("kn,in,jn->kij", wgt, hlm[:, ::-1], hlm)
    return U, V


# ------------------------------------------------------------------ draws

@dataclass
class Prior:
    d_min: float
    d_max: float
    t_half: float

    def sample(self, rng, n):
        u = rng.uniform(size=(7, n))
        d3 = self.d_min ** 3 + u[5] * (self.d_max ** 3 - self.d_min ** 3)
        return {
            "ra": 2 * math.pi * u[0],
            "dec": np.arcsin(2 * u[1] - 1),
            "psi": math.pi * u[2],
            "incl": np.arccos(2 * u[3] - 1),
            "phase": 2 * math.pi * u[4],
            "lnD": np.log(d3) / 3.0,
            "t": (2 * u[6] - 1) * self.t_half,
        }

    def logpdf(self, th):
        """ln p with respect to (ra, dec, psi, incl, phase, lnD, t)."""
        D = np.exp(th["lnD"])
        inside = ((D >= self.d_min) & (D <= self.d_max) & (np.abs(th["t"]) <= self.t_half)
                  & (np.abs(th["dec"]) <= math.pi / 2) & (th["incl"] >= 0) & (th["incl"] <= math.pi))
        with np.errstate(divide="ignore", invalid="ignore"):
            lp = (-math.log(2 * math.pi) + np.log(np.cos(th["dec"]) / 2) - math.log(math.pi)
                  + np.log(np.sin(th["incl"]) / 2) - math.log(2 * math.pi)
                  + math.log(3.0) + 3 * th["lnD"] - math.log(self.d_max ** 3 - self.d_min ** 3)
                  - math.log(2 * self.t_half))
        return np.where(inside, lp, -np.inf)


_PERIOD = {"ra": 2 * math.pi, "psi": math.pi, "phase": 2 * math.pi}


def mixture_draws(rng, prior: Prior, truth: dict, sigma: dict, n: int, frac_prior=0.1):
    """Defensive mixture q = frac_prior p + (1 - frac_prior) N(truth, diag sigma^2),
    angles wrapped into their prior ranges; returns (draws, ln p - ln q)."""
    pri = prior.sample(rng, n)
    use_g = rng.uniform(size=n) >= frac_prior
    th = {}
    for p in PARAMS:
        g = truth[p] + sigma[p] * rng.standard_normal(n)
        if p in _PERIOD:
            g = np.mod(g, _PERIOD[p])
        th[p] = np.where(use_g, g, pri[p])
    lp = prior.logpdf(th)
    lg = np.zeros(n)
    for p in PARAMS:
        d = th[p] - truth[p]
        if p in _PERIOD:
            P = _PERIOD[p]
            d = np.mod(d + P / 2, P) - P / 2
        lg += -0.5 * (d / sigma[p]) ** 2 - math.log(sigma[p] * math.sqrt(2 * math.pi))
    lq = np.logaddexp(math.log(frac_prior) + lp, math.log1p(-frac_prior) + lg)
    return th, lp - lq


def noise_moments(freq, wgt_row, hk_row):
    """<f^n>, n = 0..2 over f > 0 with weights |h|^2/S (eq. ap:fmoments)."""
    pos = freq > 0
    p = wgt_row[pos] * np.abs(hk_row[pos]) ** 2
    tot = p.sum()
    return [float((p * freq[pos] ** n).sum() / tot) for n in range(3)]


# ---------------------------------------------------------------- points

def make_point(*, dets, modes, f_low, f_max, df, rate, half_window, snr, truth, gmst,
               d_ref, rng, noise=False, q_dtype=np.complex64, center=None):
    """One intrinsic point: Q, U, V, geometry, plus the frequency-domain arrays
    for exact-Q evaluation and the injection's bookkeeping."""
    freq = freq_grid(f_max, df)
    K, M = len(dets), len(modes)
    hlm = mode_spectra(rng, modes, freq, f_low, f_max)
    wgt = inner_weight(freq, df, f_low, f_max, K)
    hk, arrival = inject(dets, modes, hlm, freq, truth, gmst, d_ref)
    rho2 = float(np.sum(wgt * np.abs(hk) ** 2))
    scale = snr / math.sqrt(rho2) if snr else 1.0
    hlm = hlm * scale
    hk = hk * scale
    dk = hk + (colored_noise(rng, freq, df, K) if noise else 0.0)
    dt = 1.0 / rate
    n = int(math.ceil(2 * half_window * rate))
    centre = arrival if center is None else np.asarray(center, dtype=float)
    t0 = centre - 0.5 * (n - 1) * dt
    Q = q_table(wgt, hlm, dk, freq, df, t0, dt, n)
    U, V = uv_matrices(wgt, hlm)
    pos = np.stack([d[0] for d in dets])
    resp = np.stack([d[1] for d in dets])
    point = {
        "K": K, "M": M,
        "ell": np.array([lm[0] for lm in modes], dtype=np.int32),
        "em": np.array([lm[1] for lm in modes], dtype=np.int32),
        "Q": Q.astype(q_dtype), "q_t0": t0, "q_dt": dt,
        "U": U, "V": V, "det_pos": pos, "det_resp": resp,
        "gmst": float(gmst), "d_ref": float(d_ref),
    }
    exact = {"freq": freq, "wgt": wgt, "hlm": hlm, "dk": dk}
    info = {"snr": snr, "rho2": snr ** 2 if snr else rho2, "arrival": arrival, "hk": hk,
            "truth": dict(truth), "modes": list(modes)}
    return point, exact, info


def default_truth(rng, d_ref: float):
    return {
        "ra": rng.uniform(0.3, 2 * math.pi - 0.3),
        "dec": rng.uniform(-1.0, 1.0),
        "psi": rng.uniform(0.2, math.pi - 0.2),
        "incl": rng.uniform(0.5, 1.3),
        "phase": rng.uniform(0.3, 2 * math.pi - 0.3),
        "lnD": math.log(d_ref),
        "t": 0.0,
    }


def proposal_sigma(info, exact):
    """Diagonal widths of the Gaussian component: twice the Fisher-scale widths
    of each parameter, from sigma_t = 1/(2 pi rho sigma_f) (eq. ap:sigmat) and
    1/rho for the amplitude and angles."""
    rho = math.sqrt(info["rho2"])
    k0 = 0
    m = noise_moments(exact["freq"], exact["wgt"][k0], info["hk"][k0])
    sig_f = math.sqrt(max(m[2] - m[1] ** 2, 1e-12))
    sig_t = 1.0 / (2 * math.pi * rho * sig_f)
    sky = sig_t / 0.01
    return {"ra": 2 * sky, "dec": 2 * sky, "psi": 2.0 / rho, "incl": 6.0 / rho,
            "phase": 2.0 / rho, "lnD": 6.0 / rho, "t": 2 * sig_t}


def as_float(draws: dict, dtype) -> dict:
    return {p: np.ascontiguousarray(np.asarray(draws[p]), dtype=dtype) for p in PARAMS}


# --------------------------------------------------------------- configs

D_REF = 100.0


def config0(n_draws: int = 10_000):
    """2 seeded L detectors, (2,+-2), 20-1024 Hz, df 0.25 Hz, SNR 20 + noise,
    Q complex128 at 4096 Hz over +-0.1 s, 1e4 prior draws in float64."""
    rng = np.random.default_rng(seed_for(0, 0))
    dets = random_l_detectors(rng, 2)
    gmst = rng.uniform(0, 2 * math.pi)
    truth = default_truth(rng, D_REF)
    point, exact, info = make_point(
        dets=dets, modes=[(2, 2), (2, -2)], f_low=20.0, f_max=1024.0, df=0.25, rate=4096.0,
        half_window=0.1, snr=20.0, truth=truth, gmst=gmst, d_ref=D_REF, rng=rng,
        noise=True, q_dtype=np.complex128)
    prior = Prior(0.5 * D_REF, 2.0 * D_REF, 0.01)
    draws = prior.sample(np.random.default_rng(seed_for(0, 1)), n_draws)
    logw = np.zeros(n_draws)
    return point, exact, info, as_float(draws, np.float64), logw


def config_3g(config: int, n_det: int, snr: float, half_window: float, n_draws: int,
              draw_stream: int = 1):
    """The 3G network configs (1: K=4 SNR 600 +-20 ms; 2: SNR 1000; 4: K=5
    SNR 1000 +-50 ms): 10 modes on 5-2048 Hz, zero noise, complex64 Q at
    32768 Hz, float32 draws from the defensive mixture."""
    rng = np.random.default_rng(seed_for(config, 0))
    gmst = rng.uniform(0, 2 * math.pi)
    truth = default_truth(rng, D_REF)
    point, exact, info = make_point(
        dets=network_3g(n_det), modes=MODES10, f_low=5.0, f_max=2048.0, df=0.25,
        rate=32768.0, half_window=half_window, snr=snr, truth=truth, gmst=gmst, d_ref=D_REF,
        rng=rng, noise=False, q_dtype=np.complex64)
    prior = Prior(0.5 * D_REF, 2.0 * D_REF, 0.01)
    sig = proposal_sigma(info, exact)
    draws, logw = mixture_draws(np.random.default_rng(seed_for(config, draw_stream)), prior,
                                truth, sig, n_draws)
    info["prior"] = prior
    info["sigma"] = sig
    return point, exact, info, as_float(draws, np.float32), logw.astype(np.float32)


def config1(n_draws: int = 1 << 22):
    return config_3g(1, 4, 600.0, 0.02, n_draws)


def config2(n_draws: int = 1 << 20):
    return config_3g(2, 4, 1000.0, 0.02, n_draws)


def config4(n_draws: int = 1 << 22, chunk: int = 0):
    """One 2^22 chunk (index `chunk`) of the 2^26-draw full-event config."""
    return config_3g(4, 5, 1000.0, 0.05, n_draws, draw_stream=1 + chunk)


def config3_point(index: int):
    """Point `index` of the 512-point batching config: K in [2,5] seeded L
    detectors, M in {2,4,...,10} of the ten modes, n = 2^U[13,16] samples at
    32768 Hz, SNR log-uniform in [20, 1000], N_p = 10^U[4,6] mixture draws."""
    rng = np.random.default_rng(seed_for(3, 1000 + index))
    K = int(rng.integers(2, 6))
    M = 2 * int(rng.integers(1, 6))
    n = int(2 ** rng.uniform(13, 16))
    snr = float(math.exp(rng.uniform(math.log(20.0), math.log(1000.0))))
    n_draws = int(10 ** rng.uniform(4, 6))
    gmst = rng.uniform(0, 2 * math.pi)
    truth = default_truth(rng, D_REF)
    point, exact, info = make_point(
        dets=random_l_detectors(rng, K), modes=MODES10[:M], f_low=5.0, f_max=2048.0, df=0.25,
        rate=32768.0, half_window=0.5 * n / 32768.0, snr=snr, truth=truth, gmst=gmst,
        d_ref=D_REF, rng=rng, noise=False, q_dtype=np.complex64)
    prior = Prior(0.5 * D_REF, 2.0 * D_REF, 0.01)
    sig = proposal_sigma(info, exact)
    draws, logw = mixture_draws(rng, prior, truth, sig, n_draws)
    return point, exact, info, as_float(draws, np.float32), logw.astype(np.float32)
