"""The oracle's pins are strong enough to catch plausible mistakes.

Each case copies the oracle source, plants one typical error (a dropped
conjugate, a flipped sign, a transposed matrix, a wrong factor, a wrong
Jacobian), compiles the copy on the CPU and checks that at least one pin of
the battery below fails for it, while the unmodified oracle passes them all.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.integrate

import oracle as O
import workload as W

SRC = os.path.join(os.path.dirname(O.__file__), "rift_oracle.c")

MUTATIONS = {
    "v_term_sign": ("tq += F2 * creal(A) + creal(F * F * B);",
                    "tq += F2 * creal(A) - creal(F * F * B);"),
    "data_term_no_conj": ("G += conj(Y[i]) * Qh[i];", "G += Y[i] * Qh[i];"),
    "u_transposed": ("cplx u = Uk[(i * M + j) * 2] + I * Uk[(i * M + j) * 2 + 1];",
                     "cplx u = Uk[(j * M + i) * 2] + I * Uk[(j * M + i) * 2 + 1];"),
    "delay_sign": ("double tk = tc - (xk[0] * s[0] + xk[1] * s[1] + xk[2] * s[2]);",
                   "double tk = tc + (xk[0] * s[0] + xk[1] * s[1] + xk[2] * s[2]);"),
    "cross_sign": ("  return fp - I * fx;\n}\n\n/* Derivative",
                   "  return fp + I * fx;\n}\n\n/* Derivative"),
    "quad_factor": ("*Tq = 0.25 * x * x * tq;", "*Tq = 0.5 * x * x * tq;"),
    "lagrange_weight": ("w[1] = (a * c * d) / 2.0;", "w[1] = (a * c * d) / 3.0;"),
    "condon_shortley": ("double norm = ((m & 1) ? -1.0 : 1.0) *", "double norm = 1.0 *"),
    "lnz_no_mean": ("out[0] = m + log(s) - log((double)N);", "out[0] = m + log(s);"),
    "grad_lnD": ("g[ORA_LND] = -td + 2.0 * tq;", "g[ORA_LND] = -td + tq;"),
    "grad_psi": ("cplx dF_psi = 2.0 * I * F;", "cplx dF_psi = 2.0 * F;"),
    "dist_jacobian": ("lnw_nodes[j] = log(wtrap) + lnZp + 2.0 * lnd + lnd;",
                      "lnw_nodes[j] = log(wtrap) + lnZp + 2.0 * lnd;"),
    "time_slope_scale": ("dout[2 * i] += dw[tap] * row[2 * i] / dt;",
                         "dout[2 * i] += dw[tap] * row[2 * i];"),
    # distance-marginalised gradient E[x] dK - E[x^2] dR/2 (dR/2 = dT_q at x = 1)
    "dist_grad_half_dropped": ("g[p] = ex * dtd[p] - ex2 * dtq[p];",
                               "g[p] = ex * dtd[p] - 2.0 * ex2 * dtq[p];"),
    "dist_grad_mean_squared": ("g[p] = ex * dtd[p] - ex2 * dtq[p];",
                               "g[p] = ex * dtd[p] - ex * ex * dtq[p];"),
}


def _fixture():
    rng = np.random.default_rng(31)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:6], f_low=20.0, f_max=256.0, df=0.5, rate=8192.0,
        half_window=0.05, snr=25.0, truth=truth, gmst=0.7, d_ref=100.0, rng=rng, noise=True,
        q_dtype=np.complex128)
    return dets, point, exact, info


FIX = _fixture()


def battery():
    """Run the quick pins; return the names of those that fail."""
    dets, point, exact, info = FIX
    pt = O.OraclePoint(point, exact)
    failed = []
    truth = info["truth"]
    rng = np.random.default_rng(32)
    pri = W.Prior(50.0, 200.0, 0.01).sample(rng, 6)
    draws = {p: np.asarray(pri[p], dtype=np.float64) for p in W.PARAMS}
    # 1. lnL against direct inner products with the independent injection
    lnl = O.lnL(pt, draws, exact_q=True)
    for i in range(6):
        th = {p: float(draws[p][i]) for p in W.PARAMS}
        hk, _ = W.inject(dets, W.MODES10[:6], exact["hlm"], exact["freq"], th, point["gmst"],
                         point["d_ref"])
        dh = float(np.sum(exact["wgt"] * np.real(np.conj(hk) * exact["dk"])))
        hh = float(np.sum(exact["wgt"] * np.abs(hk) ** 2))
        if not abs(lnl[i] - (dh - 0.5 * hh)) < 1e-9 * max(1.0, abs(dh) + hh):
            failed.append("direct")
            break
    # 2. table + cubic close to exact Q near the truth
    near = {p: np.full(4, truth[p]) + 1e-4 * np.arange(4) for p in W.PARAMS}
    if not np.max(np.abs(O.lnL(pt, near) - O.lnL(pt, near, exact_q=True))) < 1e-2:
        failed.append("table")
    # 3. gradient against central differences (exact Q)
    th = np.stack([draws[p] for p in W.PARAMS], axis=1)[:3]
    _, g = O.lnL_grad(pt, th, exact_q=True)
    for j in range(7):
        step = 1e-6 * (1e-3 if j == 6 else 1.0)
        tp, tm = th.copy(), th.copy()
        tp[:, j] += step
        tm[:, j] -= step
        fd = (O.lnL(pt, tp, exact_q=True) - O.lnL(pt, tm, exact_q=True)) / (2 * step)
        if not np.all(np.abs(g[:, j] - fd) < 1e-5 * np.maximum(1, np.abs(g[:, j]))):
            failed.append("fd")
            break
    # 4. table-gradient time slope against central differences of the table lnL
    tp, tm = th.copy(), th.copy()
    tp[:, 6] += 1e-9
    tm[:, 6] -= 1e-9
    fd = (O.lnL(pt, tp) - O.lnL(pt, tm)) / 2e-9
    gt = O.lnL_grad(pt, th)[1][:, 6]
    if not np.median(np.abs(gt - fd) / np.maximum(1, np.abs(gt))) < 1e-3:
        failed.append("fd_table")
    # 5. lnZ closed form
    lz = O.lnZ(np.array([0.0, 0.0, 0.0, math.log(2.0)]))
    if not (abs(lz[0] - math.log(1.25)) < 1e-14 and abs(lz[2] - 2.5) < 1e-14):
        failed.append("lnz")
    # 6. distance marginal against adaptive quadrature
    x, lnw = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, 200.0)
    d1 = {p: np.array([truth[p]]) for p in W.PARAMS}
    marg = O.lnL_distmarg(pt, d1, x, lnw)[0]
    _, td, tq, _ = O.lnL(pt, {**d1, "lnD": np.array([math.log(100.0)])}, terms=True)
    K, R = td[0], 2 * tq[0]
    f = lambda D: 3 * D ** 2 / (200.0 ** 3 - 50.0 ** 3) * math.exp(
        K * 100.0 / D - 0.5 * R * (100.0 / D) ** 2 - K * K / (2 * R))
    val, _ = scipy.integrate.quad(f, 50.0, 200.0, epsrel=1e-12, limit=400, points=[100.0 * R / K])
    if not abs(marg - (math.log(val) + K * K / (2 * R))) < 1e-5:
        failed.append("dist")
    # 7. distance-marginalised gradient against central differences of the
    # distance-marginalised lnL (eq. ap:dexp summed on the node table)
    rng8 = np.random.default_rng(33)
    dn = {p: truth[p] + s * rng8.standard_normal(8) for p, s in
          (("ra", 0.02), ("dec", 0.02), ("psi", 0.1), ("incl", 0.1), ("phase", 0.1),
           ("lnD", 0.3), ("t", 3e-4))}
    thn = np.stack([dn[p] for p in W.PARAMS], axis=1)
    _, gd = O.lnL_distmarg(pt, thn, x, lnw, grad=True)
    for j in (0, 1, 2, 3, 4, 6):
        step = 1e-6 * (1e-3 if j == 6 else 1.0)
        tp, tm = thn.copy(), thn.copy()
        tp[:, j] += step
        tm[:, j] -= step
        fd = (O.lnL_distmarg(pt, tp, x, lnw) - O.lnL_distmarg(pt, tm, x, lnw)) / (2 * step)
        if not np.median(np.abs(gd[:, j] - fd) / np.maximum(1, np.abs(gd[:, j]))) < 1e-5:
            failed.append("dist_grad")
            break
    # 8. harmonic closed form
    if not abs(O.sylm(-2, 2, 1, 1.0, 0.0) - math.sqrt(5 / (16 * math.pi)) * math.sin(1.0) *
               (1 + math.cos(1.0))) < 1e-14:
        failed.append("sylm")
    return failed


def test_unmodified_oracle_passes_battery():
    assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mdir = tmp_path / "mut"
    mdir.mkdir()
    (mdir / "rift_oracle.c").write_text(src.replace(old, new))
    (mdir / "rift_oracle.h").write_text(open(SRC.replace(".c", ".h")).read())
    so = str(mdir / "libmut.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-o", so, str(mdir / "rift_oracle.c"), "-lm", "-lpthread"])
    with O.use_library(so):
        failed = battery()
    assert failed, f"planted mistake {name} passed every pin"
