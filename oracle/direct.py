"""Plain FP64 CPU oracle of the in-likelihood direct marginalisation over
(phi_ref, psi) and distance (Sec. II.D, eq. direct_marginalization; App. F).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

For one draw of the sampled coordinates (ra, dec, incl, t_c) it computes

    L_dir = int dphi dpsi dx  p(phi) p(psi) p_x(x) exp[lnL(phi, psi, x)],

and optionally integrates t_c as well (fixed-spacing rule, eq. ap:tfixed,
the band-limited full-window rule, eq. ap:tband, or the peak-local rule,
eq. ap:tlocal, on the band-limited rule's fine nodes).

following the paper's steps:

1. ERAI reconstruction (eq. ap:angleharm, eq. ap:nyquist): at fixed time the
   data term K(phi, psi) and the model norm R(phi, psi) of lnL(x) = K x - R x^2/2
   (eq. ap:dexp; K and R at x = 1) are finite trigonometric polynomials, with
   harmonics e^{2 i p psi}, |p| <= 2, and e^{i q phi}, |q| <= 2 m_max.  They are
   sampled with the static oracle on a product grid of N_psi = 5 polarisations
   and N_phi = 4 m_max + 1 phases and their coefficients recovered by a 2D DFT.
2. The exponential is integrated on an arithmetic (periodic trapezoid) grid of
   n_phi x n_psi points in [0, 2 pi) x [0, pi), sized by the caller from the
   amplitude, with the uniform priors p(phi) = 1/(2 pi), p(psi) = 1/pi.
3. At each grid point the distance is integrated by adaptive Gauss-Hermite in
   x = d_ref / D (eq. ap:dgh) centred at x* = K/R with width sigma_x = R^(-1/2)
   (eq. ap:dpeak), with the prior uniform in volume, p(D) = 3 D^2 /
   (D_max^3 - D_min^3) on [D_min, D_max], i.e. p_x(x) = 3 d_ref^3 x^-4 /
   (D_max^3 - D_min^3) on [d_ref/D_max, d_ref/D_min]:
   int p_x e^{K x - R x^2/2} dx ~ e^{K^2/(2R)} sqrt(2) sigma_x sum_i w_i
   p_x(x* + sqrt(2) sigma_x xi_i) with the Gauss-Hermite rule (xi_i, w_i) of
   weight e^{-xi^2}.

Readings: the phase grid of the reconstruction covers |q| <= 2 m_max with
4 m_max + 1 samples (the model norm carries m_i + m_j; the printed
2 m_max + 1 assumes even-only harmonics); the draw's own phase, psi and lnD
are not used; where the Gaussian in x lies outside the prior the rule is
applied as printed (no fallback).
"""
from __future__ import annotations

import math

import numpy as np
import numpy.polynomial.hermite as _herm

from . import OraclePoint, lnL as _static_lnL

PARAMS = ("ra", "dec", "psi", "incl", "phase", "lnD", "t")


def _terms_on_grid(pt: OraclePoint, d_ref, ra, dec, incl, tc, phis, psis):
    """K and R at x = 1 on the product grid [len(psis)][len(phis)]."""
    P, F = np.meshgrid(psis, phis, indexing="ij")
    n = P.size
    th = {"ra": np.full(n, ra), "dec": np.full(n, dec), "psi": P.ravel(),
          "incl": np.full(n, incl), "phase": F.ravel(), "lnD": np.full(n, math.log(d_ref)),
          "t": np.full(n, tc)}
    _, Td, Tq, _ = _static_lnL(pt, th, terms=True, threads=1)
    return Td.reshape(P.shape), (2.0 * Tq).reshape(P.shape)


def reconstruct(pt: OraclePoint, point: dict, ra, dec, incl, tc):
    """ERAI step 1: the harmonic coefficients of K and R, as 2D DFTs over the
    Nyquist grid: returns (cK, cR, m_max) with c[p, q] the coefficient of
    e^{i (2 p psi + q phi)} stored at [p mod 5][q mod (4 m_max + 1)]."""
    m_max = int(np.max(np.abs(point["em"])))
    n_psi, n_phi = 5, 4 * m_max + 1
    psis = np.pi * np.arange(n_psi) / n_psi
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    K, R = _terms_on_grid(pt, point["d_ref"], ra, dec, incl, tc, phis, psis)
    return np.fft.fft2(K) / K.size, np.fft.fft2(R) / R.size, m_max


def evaluate(c, psi, phi):
    """The trigonometric polynomial with DFT coefficients c at (psi, phi)."""
    n_psi, n_phi = c.shape
    p = np.fft.fftfreq(n_psi, 1.0 / n_psi)
    q = np.fft.fftfreq(n_phi, 1.0 / n_phi)
    E = np.exp(1j * (2 * np.multiply.outer(np.asarray(psi), p)))          # [..., n_psi]
    G = np.exp(1j * np.multiply.outer(np.asarray(phi), q))                # [..., n_phi]
    return np.real(np.einsum("...p,pq,...q->...", E, c, G))


def distance_gh(K, R, d_ref, d_min, d_max, n_gh):
    """ln of the adaptive Gauss-Hermite distance integral (eq. ap:dgh)."""
    xi, w = _herm.hermgauss(n_gh)
    K = np.asarray(K, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    xs, sig = K / R, 1.0 / np.sqrt(R)
    lo, hi = d_ref / d_max, d_ref / d_min
    norm = 3.0 * d_ref ** 3 / (d_max ** 3 - d_min ** 3)
    x = xs[..., None] + math.sqrt(2.0) * sig[..., None] * xi
    px = np.where((x >= lo) & (x <= hi), norm * np.abs(x) ** -4.0, 0.0)
    s = np.sum(w * px, axis=-1)
    with np.errstate(divide="ignore"):
        return K * K / (2.0 * R) + np.log(math.sqrt(2.0) * sig * s)


def mirrored_kernel(z, n):
    """The reconstruction kernel of the mirrored series: the trigonometric
    interpolant, of period 2n samples and harmonics |k| <= n - 1,
    D(z) = (1/2n) sum_{|k|<n} e^{i pi k z / n} = sin((2n-1) pi z/(2n)) /
    (2n sin(pi z/(2n))), z in units of the coarse spacing."""
    z = np.asarray(z, dtype=np.float64)
    den = 2 * n * np.sin(np.pi * z / (2 * n))
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.sin((2 * n - 1) * np.pi * z / (2 * n)) / den
    return np.where(np.abs(den) < 1e-300, (2 * n - 1) / (2 * n), v)


def mirrored_upsample(coarse, t_up: int):
    """The mirrored band-limited reconstruction (the "terminal band-limited,
    mirrored" option beside eq. ap:tband): the n window samples at the
    midpoints (j + 1/2) h are extended by their reflection about the window's
    ends (sample j mirrored to -(j + 1/2) h; the extension of period 2n h is
    continuous, as the pregrid's reflected series), and the trigonometric
    interpolant of that series is taken at the t_up fine midpoints of each
    interval: sum_j value_j [D(t_f - t_j) + D(t_f + t_j)] in units of h.  The
    reflected series has no Nyquist component, so the kernel omits it.
    `coarse` is [n, ...]; returns [n t_up, ...]."""
    coarse = np.asarray(coarse)
    n = coarse.shape[0]
    tf = (0.5 + np.arange(n * t_up)) / t_up
    tj = np.arange(n) + 0.5
    S = mirrored_kernel(np.subtract.outer(tf, tj), n) + mirrored_kernel(np.add.outer(tf, tj), n)
    return np.tensordot(S, coarse, axes=1)


def sinc_upsample(coarse, t_up: int):
    """The band-limited reconstruction of eq. ap:tband: samples taken at
    spacing h on the midpoints (j + 1/2) h, j < n, are carried to the t_up
    fine midpoints of each interval, (f + 1/2) h / t_up, f < n t_up, by
    sum_j value_j sinc((t_f - t_j) / h), sinc(x) = sin(pi x)/(pi x) (eq.
    ap:sinc), the sum running over the n samples of the window.  `coarse` is
    [n, ...]; returns [n t_up, ...]."""
    coarse = np.asarray(coarse)
    n = coarse.shape[0]
    tf = (np.arange(n * t_up) + 0.5) / t_up          # fine times in units of h
    tj = np.arange(n) + 0.5
    S = np.sinc(np.subtract.outer(tf, tj))            # numpy's sinc is sin(pi x)/(pi x)
    return np.tensordot(S, coarse, axes=1)


class ProjectionBound:
    """The envelope of the peak-local rule: an upper bound of ln of the
    angular-and-distance integrand at one time node.  Per detector k the
    template is a x F_k Y with a amplitude vector a in C^M; writing y =
    (Re a, Im a), the data term is y.q_k with q_k = (Re Q_k(t_k), Im Q_k(t_k))
    and the quadratic term is (1/2) y^T G_k y with G_k the Hessian of
    (1/4)(a^dag U_k a + Re a^T V_k a).  Every (phi, psi, x) template is one
    such y per detector, so by Cauchy-Schwarz over the detectors
    K^2/(2R) <= (1/2) sum_k q_k^T G_k^+ q_k, and since the distance prior
    integrates to one, int p_x e^{K x - R x^2/2} dx <= e^{K^2/(2R)}: the bound
    U(t) = (1/2) sum_k q_k^T G_k^+ q_k at the detectors' arrival times.  It is
    attained at a noise-free injection (the data lie in the template span)."""

    def __init__(self, point: dict):
        self.point = point
        K, M = int(point["K"]), int(point["M"])
        self.Ginv = []
        for k in range(K):
            U = np.asarray(point["U"][k], dtype=np.complex128)
            V = np.asarray(point["V"][k], dtype=np.complex128)

            def quad(y):
                a = y[:M] + 1j * y[M:]
                return 0.25 * float(np.real(np.conj(a) @ U @ a + a @ V @ a))

            E = np.eye(2 * M)
            G = np.empty((2 * M, 2 * M))
            for i in range(2 * M):
                G[i, i] = 2.0 * quad(E[i])
                for j in range(i):
                    G[i, j] = G[j, i] = quad(E[i] + E[j]) - quad(E[i]) - quad(E[j])
            self.Ginv.append(np.linalg.pinv(G, rcond=1e-12))

    def __call__(self, ra, dec, tc):
        P = self.point
        total = 0.0
        for k in range(int(P["K"])):
            from . import delay as _delay, qinterp as _qinterp
            tk = _delay(P["det_pos"][k], ra, dec, P["gmst"], tc)
            qv, _, _ = _qinterp(np.asarray(P["Q"][k]), float(P["q_t0"][k]), float(P["q_dt"]), tk)
            q = np.concatenate([qv.real, qv.imag])
            total += 0.5 * float(q @ self.Ginv[k] @ q)
        return total


def peak_local_nodes(U, h, c, depth):
    """The nodes eq. ap:tlocal keeps: every local maximum f of the envelope
    U (U_f >= U_{f-1} and U_f > U_{f+1}; beyond the ends the neighbour is
    mirrored) that lies within `depth` nat of the largest (a lower one
    contributes less than e^-depth of the peak even whole, and its nodes are
    covered by the remainder bound), its width sigma_t from the three-point
    curvature, sigma_t^2 = h^2 / (2 U_f - U_{f-1} - U_{f+1}) (U ~ U_f -
    (t - t_f)^2 / (2 sigma_t^2) near the maximum), and the nodes within
    c sigma_t of any such maximum (overlapping neighbourhoods merge).
    Returns (mask, maxima, widths), or None where a maximum is flat (no
    justified width)."""
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    if n == 1:
        return np.ones(1, bool), [0], [np.inf]
    ext = np.concatenate([[U[1]], U, [U[n - 2]]])
    tf = np.arange(n) * h
    keep = np.zeros(n, bool)
    peaks, widths = [], []
    top = np.max(U)
    for f in range(n):
        l, m, r = ext[f], ext[f + 1], ext[f + 2]
        if m >= l and m > r and m >= top - depth:
            curv = 2.0 * m - l - r
            if not curv > 0.0:
                return None
            sig = h / math.sqrt(curv)
            keep |= np.abs(tf - tf[f]) <= c * sig
            peaks.append(f)
            widths.append(sig)
    return keep, peaks, widths


def lnL_direct(point: dict, draws, n_phi: int, n_psi: int, n_gh: int, d_min: float,
               d_max: float, n_t: int = 0, t_lo: float = 0.0, t_hi: float = 0.0,
               t_up: int = 1, t_local: bool = False, t_c: float = 16.0, t_tol: float = 1e-10,
               diag: list | None = None, t_mirror: bool = False):
    """ln L_dir per draw.  With n_t = 0 the draw's t is used; otherwise t is
    integrated too, by the fixed-spacing rule of eq. ap:tfixed on n_t
    midpoints t_j = t_lo + (j + 1/2) h, h = (t_hi - t_lo)/n_t, with the
    uniform prior on [t_lo, t_hi] (weight 1/n_t per node); the harmonic model
    is reconstructed at every time node before any integration, as the
    fixed-time qualification of App. F.1 requires.

    With t_up > 1 the band-limited full-window rule of eq. ap:tband: the data
    term's harmonic coefficients (linear in Q, hence band limited) are
    reconstructed at the n_t coarse midpoints, carried to t_up fine midpoints
    per interval by ``sinc_upsample``, and the angular and distance integrals
    run at each of the n_t t_up fine nodes (weight 1/(n_t t_up)).  The model
    norm does not depend on t at a fixed sky position; it is taken from the
    first coarse node.

    With t_mirror the fine coefficients come from the mirrored series
    (``mirrored_upsample``) instead of the truncated sinc sum.

    With t_local (needs t_up > 1) the peak-local rule of eq. ap:tlocal on the
    same fine nodes: the envelope bound U_f of every fine node
    (``ProjectionBound``), the nodes within t_c sigma_t of its maxima
    (``peak_local_nodes``) integrated as above, and the others bounded:
    together they add at most ln R = LSE_skipped(U_f) - ln(n_t t_up).  If
    that bound exceeds t_tol of the kept value, or no justified width or
    bound exists, every fine node is integrated (the band-limited rule).
    `diag`, if a list, receives per draw a dict: kept (node mask or None),
    maxima (node indices), widths (their sigma_t), gap (ln R - kept value),
    fallback (bool)."""
    pt = OraclePoint(point)
    th = {p: np.asarray(draws[p], dtype=np.float64) for p in PARAMS}
    N = th["ra"].shape[0]
    psis = np.pi * np.arange(n_psi) / n_psi
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    PS, PH = np.meshgrid(psis, phis, indexing="ij")
    lnw = -math.log(n_phi * n_psi)   # trapezoid weights times the uniform priors
    out = np.empty(N)
    bound_fn = None
    for i in range(N):
        if n_t > 0:
            h = (t_hi - t_lo) / n_t
            times = t_lo + (np.arange(n_t) + 0.5) * h
            lnwt = -math.log(n_t)
        else:
            times, lnwt = [th["t"][i]], 0.0
        coefs = [reconstruct(pt, point, th["ra"][i], th["dec"][i], th["incl"][i], t)[:2]
                 for t in times]
        if n_t > 0 and t_up > 1:
            cR = coefs[0][1]
            up = mirrored_upsample if t_mirror else sinc_upsample
            coefs = [(cK, cR) for cK in up(np.stack([c[0] for c in coefs]), t_up)]
            lnwt = -math.log(n_t * t_up)

        def node_values(cK, cR):
            K = evaluate(cK, PS, PH)
            R = evaluate(cR, PS, PH)
            return (distance_gh(K, R, point["d_ref"], d_min, d_max, n_gh) + lnw + lnwt).ravel()

        def lse(v):
            m = np.max(v) if v.size else -np.inf
            return m + math.log(np.sum(np.exp(v - m))) if m > -np.inf else -np.inf

        keep, maxima, widths = None, [], []
        if t_local and n_t > 0 and t_up > 1:
            if bound_fn is None:
                bound_fn = ProjectionBound(point)
            hf = (t_hi - t_lo) / (n_t * t_up)
            U = [bound_fn(th["ra"][i], th["dec"][i], t_lo + (f + 0.5) * hf)
                 for f in range(n_t * t_up)]
            # maxima lower than the largest by more than ln(1/t_tol) + ln(n_f)
            # cannot matter at the tolerance
            sel = peak_local_nodes(U, hf, t_c, -math.log(t_tol) + math.log(n_t * t_up))
            if sel is not None:
                keep, maxima, widths = sel
        if keep is None or keep.all():
            out[i] = lse(np.concatenate([node_values(cK, cR) for cK, cR in coefs]))
            if diag is not None:
                diag.append({"kept": keep, "maxima": maxima, "widths": widths, "gap": -np.inf,
                             "fallback": keep is None})
            continue
        kept = lse(np.concatenate([node_values(*coefs[f]) for f in np.flatnonzero(keep)]))
        bound = lse(np.asarray([U[f] for f in np.flatnonzero(~keep)])) + lnwt
        if bound - kept > math.log(t_tol):  # the remainder may matter: the full rule
            rest = lse(np.concatenate([node_values(*coefs[f]) for f in np.flatnonzero(~keep)]))
            m = max(kept, rest)
            out[i] = m + math.log(math.exp(kept - m) + math.exp(rest - m))
            if diag is not None:
                diag.append({"kept": keep, "maxima": maxima, "widths": widths, "gap": bound - kept,
                             "fallback": True})
        else:
            out[i] = kept
            if diag is not None:
                diag.append({"kept": keep, "maxima": maxima, "widths": widths, "gap": bound - kept,
                             "fallback": False})
    return out
