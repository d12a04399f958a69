"""GPU parity of d lnL / d(ra, dec, psi, incl, phase, lnD, t) (Sec. II.B).

FP64 path: the analytic gradient matches the oracle's analytic gradient to
1e-8 of each component's scale.  FP32-mixed path: matches it to 1e-4 of the
component's scale on draws within 50 nat of the best draw (the adjoint works
in FP32 on the residual e - w, with the large time slope in double-float, so
its error grows with |e - w| far from the peak: 1e-2 there), and matches
central finite differences of the
FP64 oracle lnL (step 1e-6) on 1024 draws of the SNR-1000 workload; the 7x7
Fisher matrix at the injected truth from finite differences of the GPU
gradient matches the oracle's.
"""
import numpy as np
import pytest

import oracle as O
import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


@pytest.fixture(scope="module")
def cfg2():
    return W.config2(n_draws=1 << 14)


def scale(g):
    """Per-component scale: |g| plus the component's RMS over the draws."""
    return np.abs(g) + np.sqrt(np.mean(g ** 2, axis=0))[None, :]


def gpu_grad(R, pt, draws, prec):
    lnl, g = R.rift_ile_lnL_grad(pt, draws, prec)
    return lnl.cpu().numpy(), g.cpu().numpy().T


@pytest.mark.parametrize("which", ["cfg0", "cfg2"])
def test_fp64_gradient_matches_oracle(R, which, cfg2):
    point, exact, info, draws, logw = W.config0() if which == "cfg0" else cfg2
    pt = R.Point(point)
    lnl, g = gpu_grad(R, pt, draws, R.FP64)
    rl, rg = O.lnL_grad(O.OraclePoint(point), draws)
    assert np.all(np.abs(lnl - rl) <= 1e-9 * np.maximum(1, np.abs(rl)))
    err = np.abs(g - rg) / scale(rg)
    assert err.max() < 1e-8, err.max(axis=0)


def test_mixed_gradient_matches_oracle(R, cfg2):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    lnl, g = gpu_grad(R, pt, draws, R.FP32_MIXED)
    rl, rg = O.lnL_grad(O.OraclePoint(point), draws)
    near = rl >= rl.max() - 50
    assert np.max(np.abs(lnl - rl)[near]) <= 1e-3
    err = np.abs(g - rg) / scale(rg)
    assert err[near].max() < 1e-4, err[near].max(axis=0)
    assert err.max() < 1e-2, err.max(axis=0)


def test_mixed_gradient_matches_central_differences(R, cfg2):
    """Central differences of the FP64 oracle lnL, step 1e-6 (t: 1e-9 s), on
    1024 draws near the peak; draws whose tap window moves across a table knot
    within the step are skipped (the cubic's slope is only C0 there)."""
    point, exact, info, draws, logw = cfg2
    opt = O.OraclePoint(point)
    rl = O.lnL(opt, draws)
    idx = np.argsort(-rl)[:1024]
    sub = {p: np.asarray(draws[p], dtype=np.float64)[idx] for p in W.PARAMS}
    pt = R.Point(point)
    _, g = gpu_grad(R, pt, sub, R.FP32_MIXED)
    th = np.stack([sub[p] for p in W.PARAMS], axis=1)
    for j in range(7):
        h = 1e-9 if j == 6 else 1e-6
        tp, tm = th.copy(), th.copy()
        tp[:, j] += h
        tm[:, j] -= h
        fd = (O.lnL(opt, tp) - O.lnL(opt, tm)) / (2 * h)
        s = np.abs(fd) + np.sqrt(np.mean(fd ** 2))
        rel = np.abs(g[:, j] - fd) / s
        # FD truncation/rounding with step h at lnL ~ 5e5 is ~1e-5 of the scale
        assert np.median(rel) < 1e-4, (j, np.median(rel))
        assert np.mean(rel < 1e-3) > 0.95, (j, np.mean(rel < 1e-3))


def test_fisher_at_truth_matches_oracle(R, cfg2):
    """7x7 Fisher matrix = -Hessian of lnL at the injected truth, by central
    differences of the analytic gradients (GPU FP32-mixed vs oracle) on a
    stencil of float32-representable points (the draws' storage type)."""
    point, exact, info, draws, logw = cfg2
    truth = info["truth"]
    th0 = np.array([truth[p] for p in W.PARAMS], dtype=np.float32).astype(np.float64)
    ulps = np.array([64, 64, 256, 256, 256, 256, 0])
    rows, steps = [], []
    for j in range(7):
        if j == 6:
            hp, hm = th0[j] + 1e-9, th0[j] - 1e-9
        else:
            x = np.float32(th0[j])
            hp = float(x + ulps[j] * np.spacing(x))
            hm = float(x - ulps[j] * np.spacing(x))
        for v in (hp, hm):
            t = th0.copy()
            t[j] = v
            rows.append(t)
        steps.append(hp - hm)
    pts = np.array(rows)
    d = {p: pts[:, k].copy() for k, p in enumerate(W.PARAMS)}
    pt = R.Point(point)
    _, g = gpu_grad(R, pt, d, R.FP32_MIXED)
    _, rg = O.lnL_grad(O.OraclePoint(point), pts)
    H = np.zeros((7, 7))
    Hr = np.zeros((7, 7))
    for j in range(7):
        H[j] = (g[2 * j] - g[2 * j + 1]) / steps[j]
        Hr[j] = (rg[2 * j] - rg[2 * j + 1]) / steps[j]
    F = -0.5 * (H + H.T)
    Fr = -0.5 * (Hr + Hr.T)
    dg = np.sqrt(np.abs(np.diag(Fr)))
    rel = np.abs(F - Fr) / np.outer(dg, dg)
    assert rel.max() < 2e-3, rel.max()
