"""Plain FP64 CPU oracle of the composite-index likelihood (Sec. III).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

With a time- or frequency-dependent response the template of detector k is a
short sum over a composite index a of sky-independent elementary templates
chi^(a)_lm times analytic coefficients (eq. slowrot:master, eq.
fsize:factorization), and the likelihood keeps the static form with the mode
index widened to A = (a, lm) (eq. slowrot:lnL:Decomposed):

    lnL = x Re sum_k sum_A conj(c_kA) Q_{k,A}(t_k)
        - x^2/4 sum_k [c_k^+ U_k c_k + Re(c_k^T V_k c_k)],   c_kA = C~^k_a Y_lm.

Two responses are covered.

* Earth rotation (Sec. III.A; Path A is p_max = 0, Path B p_max >= 1).  The
  antenna factor over one sidereal turn, F_k(gmst + theta), is exactly a
  trigonometric polynomial of degree 2 in theta (eq. slowrot:Fharm); its five
  coefficients are taken here by an 8-point DFT of the static antenna factor
  evaluated at shifted sidereal angles, which is exact for that degree.  The
  arrival-time drift -dt_k(theta) = -(t_k(theta) - t_k(0)) has degree 1 and is
  taken the same way.  The coefficient of chi^(p, n) is the n-th harmonic of
  F_k (-dt_k)^p / p! (eq. slowrot:delay, eq. slowrot:master), computed as a
  discrete convolution of the harmonic lists, and the arrival-time post-phase
  e^{i n Omega t_k} (eq. slowrot:postphase) multiplies it.  Times are relative
  to the reference time, so t_ref = 0 and theta = Omega t.
  Composite order: a = (p, n), p = 0..p_max, n = -(2 + p)..(2 + p).

* Finite arms (Sec. III.B, Path D).  b^k_p = 1/2 [(x.s)^p eps:xx - (y.s)^p eps:yy]
  (eq. fsize:bp) with eps = eps_+ - i eps_x the complex polarisation tensor,
  x, y the unit arm vectors of detector k and s the unit vector towards the
  source; the frequency weights W_p live in the precomputed tables.
  Composite order: a = p = 0..p_max.

Composite index A = a * M + i (a-major), i the mode.  The paper prints no
value of this likelihood for a reproducible input; the tests pin it by the
limits the paper names (Omega -> 0 and p_max = 0
recover the static likelihood), by the coefficient identities above at
off-grid sidereal angles, by the Cauchy-Schwarz bound lnL <= <d|d>/2 with
equality at the injected parameters, and by convergence in p_max.
"""
from __future__ import annotations

import math

import numpy as np

from . import antenna, delay, lib, sky_basis, sylm, _ptr

ROTATION = 1
FINITE_ARM = 2
_NDFT = 8


def n_index(kind: int, p_max: int) -> int:
    """Number of composite response indices a."""
    if kind == ROTATION:
        return (p_max + 1) * (p_max + 5)
    if kind == FINITE_ARM:
        return p_max + 1
    raise ValueError(kind)


def rotation_harmonics(resp, pos, ra, dec, psi, gmst, tc):
    """(C0[5] for n = -2..2, E[3] for m = -1..1, t_k): harmonics in theta of
    F_k(gmst + theta) and of -(t_k(gmst + theta) - t_k(gmst)), by DFT."""
    th = 2.0 * math.pi * np.arange(_NDFT) / _NDFT
    F = np.array([antenna(resp, ra, dec, psi, gmst + a) for a in th])
    tk0 = delay(pos, ra, dec, gmst, tc)
    mdt = np.array([-(delay(pos, ra, dec, gmst + a, tc) - tk0) for a in th])
    C0 = np.array([np.mean(F * np.exp(-1j * n * th)) for n in range(-2, 3)])
    E = np.array([np.mean(mdt * np.exp(-1j * m * th)) for m in range(-1, 2)])
    return C0, E, tk0


def rotation_coeffs(resp, pos, omega, p_max, ra, dec, psi, gmst, tc):
    """C~^k_a for a = (p, n) in composite order (eq. slowrot:master with the
    post-phase of eq. slowrot:postphase)."""
    C0, E, tk = rotation_harmonics(resp, pos, ra, dec, psi, gmst, tc)
    out = []
    P = np.array([1.0 + 0j])            # harmonics of (-dt)^p, centred
    for p in range(p_max + 1):
        Cp = np.convolve(C0, P) / math.factorial(p)      # n = -(2+p)..(2+p)
        n = np.arange(-(2 + p), 3 + p)
        out.append(Cp * np.exp(1j * n * omega * tk))
        P = np.convolve(P, E)
    return np.concatenate(out)


def arm_coeffs(arm_x, arm_y, p_max, ra, dec, psi, gmst):
    """b^k_p, p = 0..p_max (eq. fsize:bp)."""
    s, e1, e2 = sky_basis(ra, dec, gmst)
    p = math.cos(psi) * e1 + math.sin(psi) * e2
    q = -math.sin(psi) * e1 + math.cos(psi) * e2
    eps = (np.outer(p, p) - np.outer(q, q)) - 1j * (np.outer(p, q) + np.outer(q, p))
    x = np.asarray(arm_x, dtype=np.float64)
    y = np.asarray(arm_y, dtype=np.float64)
    ex, ey = x @ eps @ x, y @ eps @ y
    ux, uy = float(x @ s), float(y @ s)
    return np.array([0.5 * (ux ** j * ex - uy ** j * ey) for j in range(p_max + 1)])


class CompPoint:
    """FP64 copies of one composite point's inputs."""

    def __init__(self, point: dict):
        self.K, self.M = int(point["K"]), int(point["M"])
        self.kind, self.p_max = int(point["kind"]), int(point["p_max"])
        self.na = n_index(self.kind, self.p_max)
        self.A = self.na * self.M
        Q = np.asarray(point["Q"])
        assert Q.shape[0] == self.K and Q.shape[2] == self.A, Q.shape
        self.n = Q.shape[1]
        self.Qv = [np.ascontiguousarray(Q[k].astype(np.complex128)).view(np.float64)
                   for k in range(self.K)]
        self.U = np.asarray(point["U"], dtype=np.complex128)
        self.V = np.asarray(point["V"], dtype=np.complex128)
        assert self.U.shape == (self.K, self.A, self.A) and self.V.shape == self.U.shape
        self.t0 = np.asarray(point["q_t0"], dtype=np.float64)
        self.dt = float(point["q_dt"])
        self.pos = np.asarray(point["det_pos"], dtype=np.float64)
        self.resp = np.asarray(point["det_resp"], dtype=np.float64)
        self.gmst, self.d_ref = float(point["gmst"]), float(point["d_ref"])
        self.omega = float(point.get("omega", 0.0))
        self.arm_x = np.asarray(point.get("arm_x", np.zeros((self.K, 3))), dtype=np.float64)
        self.arm_y = np.asarray(point.get("arm_y", np.zeros((self.K, 3))), dtype=np.float64)
        self.ell = [int(v) for v in point["ell"]]
        self.em = [int(v) for v in point["em"]]

    def coeffs(self, k, ra, dec, psi, tc):
        if self.kind == ROTATION:
            return rotation_coeffs(self.resp[k], self.pos[k], self.omega, self.p_max, ra, dec,
                                   psi, self.gmst, tc)
        return arm_coeffs(self.arm_x[k], self.arm_y[k], self.p_max, ra, dec, psi, self.gmst)

    def qinterp(self, k, t):
        """Q_{k,A}(t) by the four-point Lagrange cubic (taps outside read 0)."""
        out = np.empty(2 * self.A)
        dout = np.empty(2 * self.A)
        oob = lib().ora_qinterp(_ptr(self.Qv[k]), self.n, self.A, float(self.t0[k]), self.dt,
                                float(t), _ptr(out), _ptr(dout))
        return out.view(np.complex128), int(oob)


def lnL(pt: CompPoint, draws, terms: bool = False):
    """lnL per draw of eq. slowrot:lnL:Decomposed (composite index widened
    mode sum), evaluated term by term in FP64.  With terms=True also returns
    the data sum, the quadratic sum (both at x = 1) and the out-of-table taps."""
    th = {p: np.asarray(draws[p], dtype=np.float64) for p in
          ("ra", "dec", "psi", "incl", "phase", "lnD", "t")}
    N = th["ra"].shape[0]
    out, tds, tqs = np.empty(N), np.empty(N), np.empty(N)
    oob = 0
    for i in range(N):
        ra, dec, psi = th["ra"][i], th["dec"][i], th["psi"][i]
        tc = th["t"][i]
        Y = np.array([sylm(-2, l, m, th["incl"][i], th["phase"][i])
                      for l, m in zip(pt.ell, pt.em)])
        x = pt.d_ref * math.exp(-th["lnD"][i])
        td = tq = 0.0
        for k in range(pt.K):
            c = np.kron(pt.coeffs(k, ra, dec, psi, tc), Y)
            tk = delay(pt.pos[k], ra, dec, pt.gmst, tc)
            q, o = pt.qinterp(k, tk)
            oob += o
            td += float(np.real(np.vdot(c, q)))
            tq += float(np.real(np.conj(c) @ pt.U[k] @ c) + np.real(c @ pt.V[k] @ c))
        tds[i], tqs[i] = td, tq
        out[i] = x * td - 0.25 * x * x * tq
    if terms:
        return out, tds, tqs, oob
    return out


def _coeff_derivs(pt: CompPoint, k, ra, dec, psi, tc, h=1e-4):
    """d C~^k / d(ra, dec, psi, t_c) by fourth-order central differences of
    the coefficient functions (smooth trigonometric polynomials of the angles
    and of the arrival time; no table is involved)."""
    base = np.array([ra, dec, psi, tc], dtype=np.float64)
    steps = np.array([h, h, h, h * 1e-2])
    out = []
    for j in range(4):
        def f(v):
            a = base.copy()
            a[j] += v
            return pt.coeffs(k, a[0], a[1], a[2], a[3])
        s = steps[j]
        out.append((-f(2 * s) + 8 * f(s) - 8 * f(-s) + f(-2 * s)) / (12 * s))
    return out


def lnL_grad(pt: CompPoint, draws):
    """(lnL, grad[N, 7]) of the composite likelihood by the chain rule:
    d T_d = Re sum conj(dc) Q + Re sum conj(c) Q' dt_k and
    d T_q = 2 Re(dc^+ U c) + 2 Re(dc^T V c) (U Hermitian, V symmetric), with
    the template derivative dc = dC~ (x) Y + C~ (x) dY: dY/d phase = i m Y,
    dY/d incl analytic, Q' the slope of the same cubic, dt_k from the delay,
    and dC~ by central differences of the coefficient functions.  Parameter
    order (ra, dec, psi, incl, phase, lnD, t)."""
    th = {p: np.asarray(draws[p], dtype=np.float64) for p in
          ("ra", "dec", "psi", "incl", "phase", "lnD", "t")}
    N = th["ra"].shape[0]
    out = np.empty(N)
    g = np.zeros((N, 7))
    for i in range(N):
        ra, dec, psi, tc = th["ra"][i], th["dec"][i], th["psi"][i], th["t"][i]
        incl, phase = th["incl"][i], th["phase"][i]
        Y = np.array([sylm(-2, l, m, incl, phase) for l, m in zip(pt.ell, pt.em)])
        dYi = np.array([sylm(-2, l, m, incl, phase, dtheta=True) for l, m in zip(pt.ell, pt.em)])
        dYp = 1j * np.array(pt.em) * Y
        x = pt.d_ref * math.exp(-th["lnD"][i])
        td = tq = 0.0
        dtd = np.zeros(7)
        dtq = np.zeros(7)
        for k in range(pt.K):
            C = pt.coeffs(k, ra, dec, psi, tc)
            dC = _coeff_derivs(pt, k, ra, dec, psi, tc)
            c = np.kron(C, Y)
            tk = delay(pt.pos[k], ra, dec, pt.gmst, tc)
            hh = 1e-6
            dtk = [(delay(pt.pos[k], ra + hh, dec, pt.gmst, tc)
                    - delay(pt.pos[k], ra - hh, dec, pt.gmst, tc)) / (2 * hh),
                   (delay(pt.pos[k], ra, dec + hh, pt.gmst, tc)
                    - delay(pt.pos[k], ra, dec - hh, pt.gmst, tc)) / (2 * hh)]
            out_q = np.empty(2 * pt.A)
            dout_q = np.empty(2 * pt.A)
            lib().ora_qinterp(_ptr(pt.Qv[k]), pt.n, pt.A, float(pt.t0[k]), pt.dt, float(tk),
                              _ptr(out_q), _ptr(dout_q))
            q, dq = out_q.view(np.complex128), dout_q.view(np.complex128)
            Uc, Vc = pt.U[k] @ c, pt.V[k] @ c
            td += float(np.real(np.vdot(c, q)))
            tq += float(np.real(np.conj(c) @ Uc) + np.real(c @ Vc))
            dcs = {0: np.kron(dC[0], Y), 1: np.kron(dC[1], Y), 2: np.kron(dC[2], Y),
                   3: np.kron(C, dYi), 4: np.kron(C, dYp), 6: np.kron(dC[3], Y)}
            dts = {0: dtk[0], 1: dtk[1], 6: 1.0}
            for j, dc in dcs.items():
                v = float(np.real(np.vdot(dc, q)))
                if j in dts:
                    v += dts[j] * float(np.real(np.vdot(c, dq)))
                dtd[j] += v
                dtq[j] += 2.0 * float(np.real(np.conj(dc) @ Uc)) + 2.0 * float(np.real(dc @ Vc))
        out[i] = x * td - 0.25 * x * x * tq
        g[i] = x * dtd - 0.25 * x * x * dtq
        g[i, 5] = -x * td + 0.5 * x * x * tq
    return out, g
