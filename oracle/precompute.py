"""Plain FP64 CPU oracle of the per-point products of eq. QUV.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

On a two-sided uniform frequency grid f_q = (q - (nf - 1)/2) df with inner
product weights w_k(f) = 2 df / S_k(|f|) inside the band (eq. QUV, as a
Riemann sum), the products are the plain sums

    Q_{k,lm}(t)     = sum_q w_k(f_q) e^{2 pi i f_q t} conj(h_lm(f_q)) d_k(f_q)
    U_{k,lm,l'm'}   = sum_q w_k(f_q) conj(h_lm(f_q)) h_l'm'(f_q)
    V_{k,lm,l'm'}   = sum_q w_k(f_q) h_lm(-f_q) h_l'm'(f_q)

evaluated here term by term (the exponential per (t, f) pair, no FFT).  The
tests pin them against the FFT-based table builder of the workloads (a
different algorithm), the symmetries U = U^+ and V = V^T, and the physical
normalisation: with noise-free data the factored likelihood built from these
products equals rho^2/2 at the injection.
"""
from __future__ import annotations

import math

import numpy as np


def q_direct(freq, wgt_k, hlm, dk_k, times, chunk: int = 64):
    """Q_{k,lm}(t) for every t in `times`: [len(times)][M] complex128."""
    freq = np.asarray(freq, dtype=np.float64)
    X = np.asarray(wgt_k)[None, :] * np.conj(np.asarray(hlm)) * np.asarray(dk_k)[None, :]
    times = np.asarray(times, dtype=np.float64)
    out = np.empty((times.shape[0], X.shape[0]), dtype=np.complex128)
    for a in range(0, times.shape[0], chunk):
        t = times[a:a + chunk]
        E = np.exp(2j * np.pi * np.outer(t, freq))          # [chunk][nf]
        out[a:a + chunk] = E @ X.T
    return out


def q_table_direct(freq, wgt, hlm, dk, t0, dt, n):
    """Q_{k,lm}(t0_k + j dt), j < n: [K][n][M]."""
    K = np.asarray(dk).shape[0]
    return np.stack([q_direct(freq, wgt[k], hlm, dk[k], t0[k] + dt * np.arange(n))
                     for k in range(K)])


def q_pregrid(q_native, r: int):
    """The fine table of eq. q-time-pregrid from a native-rate table, in the
    four steps the paper states: reflect each (detector, mode) series
    q_0 .. q_{n-1} into q_0 .. q_{n-1}, q_{n-1} .. q_0 (its periodic extension
    is then continuous), take its DFT, zero-pad the coefficients from length
    2n to 2rn (the Z_r of eq. q-time-pregrid: positive frequencies at the
    start, negative at the end, zeros between), and invert with the 1/(2n) of
    the shorter series; sample m is the trigonometric interpolant at
    t0 + m h / r.  The reflected series has no Nyquist component (its
    (-1)^j sum cancels between the halves), so no bin needs splitting.
    q_native [K][n][M] -> [K][r (n - 1) + 1][M] complex128 (the native window)."""
    q = np.asarray(q_native, dtype=np.complex128)
    K, n, M = q.shape
    refl = np.concatenate([q, q[:, ::-1, :]], axis=1)        # [K][2n][M]
    X = np.fft.fft(refl, axis=1)                              # sum_j x_j e^{-2 pi i k j / 2n}
    N, L = 2 * n, 2 * n * r
    Y = np.zeros((K, L, M), dtype=np.complex128)
    Y[:, :n, :] = X[:, :n, :]                                 # frequencies 0 .. n-1
    Y[:, L - n + 1:, :] = X[:, n + 1:, :]                     # -(n-1) .. -1
    y = np.fft.ifft(Y, axis=1) * (L / N)                      # (1/N) sum_k Y_k e^{+2 pi i k m / L}
    return y[:, :r * (n - 1) + 1, :]


def uv_direct(wgt, hlm):
    """(U, V): [K][M][M] each; h(-f_q) is the grid's mirror entry nf - 1 - q."""
    wgt = np.asarray(wgt)
    hlm = np.asarray(hlm)
    K, M = wgt.shape[0], hlm.shape[0]
    U = np.empty((K, M, M), dtype=np.complex128)
    V = np.empty((K, M, M), dtype=np.complex128)
    hm = hlm[:, ::-1]
    for k in range(K):
        for i in range(M):
            for j in range(M):
                U[k, i, j] = np.sum(wgt[k] * np.conj(hlm[i]) * hlm[j])
                V[k, i, j] = np.sum(wgt[k] * hm[i] * hlm[j])
    return U, V


def rotation_bank_fft(hlm, df, omega, p_max):
    """The widened bank of Earth-rotation templates chi^(p,n)_lm =
    M_n h_lm^(p) (eq. slowrot:master) built as Appendix B does: the p-th time
    derivative as the weight (2 pi i f)^p, then the sidereal modulation
    e^{i n Omega t} applied as a linear phase in the time domain through one
    DFT round trip on the grid's period 1/df, times centred on the reference
    time.  Composite order (p, n) then mode: [n_index * M][nf]."""
    hlm = np.asarray(hlm, dtype=np.complex128)
    M, nf = hlm.shape
    nh = (nf - 1) // 2
    q = np.arange(nf) - nh                       # f_q / df
    f = q * df
    # unshifted order: index (q mod nf)
    perm = np.mod(q, nf)
    j = np.arange(nf)
    t = np.where(j <= nh, j, j - nf) / (nf * df)  # centred times of the period
    rows = []
    for p in range(p_max + 1):
        X = hlm * (2j * np.pi * f) ** p
        Xs = np.zeros_like(X)
        Xs[:, perm] = X
        x = np.fft.ifft(Xs, axis=1) * nf          # sum_q X_q e^{+2 pi i q j / nf}
        for n in range(-(2 + p), 3 + p):
            y = x * np.exp(1j * n * omega * t)[None, :]
            Ys = np.fft.fft(y, axis=1) / nf
            rows.append(Ys[:, perm])
    return np.concatenate(rows)


def _sinc_derivs(y, kmax):
    """d^k sinc / dy^k at y for k <= kmax, from sinc(y) = int_0^1 cos(y s) ds:
    the k-th derivative is int_0^1 s^k cos(y s + k pi/2) ds (Gauss-Legendre)."""
    s, w = np.polynomial.legendre.leggauss(64)
    s = 0.5 * (s + 1.0)
    w = 0.5 * w
    y = np.asarray(y, dtype=np.float64)
    return np.stack([np.sum(w * s ** k * np.cos(np.multiply.outer(y, s) + k * np.pi / 2), axis=-1)
                     for k in range(kmax + 1)])


def arm_weights_series(x, p_max):
    """W_p(x), p <= p_max, of eq. fsize:Wp: the Taylor coefficients in u of
    D^(u, x) = 1/2 [e^{i x (1-u)} sinc(x(1+u)) + e^{-i x (1+u)} sinc(x(1-u))]
    (eq. slowrot:armtransfer without its common delay) as the Cauchy products
    of the series of e^{-i x u} and of sinc(x (1 +- u))."""
    x = np.asarray(x, dtype=np.float64)
    sd = _sinc_derivs(x, p_max)                      # [p_max + 1][...]
    fact = np.array([math.factorial(k) for k in range(p_max + 1)], dtype=np.float64)
    e = np.stack([(-1j * x) ** k / fact[k] for k in range(p_max + 1)])
    sp = np.stack([sd[k] * x ** k / fact[k] for k in range(p_max + 1)])
    sm = np.stack([sd[k] * (-x) ** k / fact[k] for k in range(p_max + 1)])
    out = []
    for p in range(p_max + 1):
        a = sum(e[p - j] * sp[j] for j in range(p + 1))
        b = sum(e[p - j] * sm[j] for j in range(p + 1))
        out.append(0.5 * (np.exp(1j * x) * a + np.exp(-1j * x) * b))
    return np.stack(out)


def arm_bank(hlm, df, T, p_max):
    """The finite-arm bank chi^(p)_lm(f) = e^{-2 pi i f T} W_p(pi f T) h_lm(f)
    (eq. fsize:factorization) on the two-sided grid: [(p_max + 1) M][nf]."""
    hlm = np.asarray(hlm, dtype=np.complex128)
    M, nf = hlm.shape
    f = (np.arange(nf) - (nf - 1) // 2) * df
    W = arm_weights_series(np.pi * f * T, p_max)
    shift = np.exp(-2j * np.pi * f * T)
    return np.concatenate([W[p][None, :] * shift[None, :] * hlm for p in range(p_max + 1)])
