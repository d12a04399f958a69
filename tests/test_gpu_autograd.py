"""The differentiable lnL (torch.autograd wrapper of the adjoint kernels,
Sec. II.B): backward gives grad_output * d lnL / d theta, identical to the
C-ABI gradient call, with or without recomputation, in both precisions, and
with the distance marginalised; it matches the oracle's analytic gradient and
passes torch.autograd.gradcheck on float64 draws in the FP64 path.
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
    return W.config2(n_draws=1 << 12)


def leaves(draws, dtype=torch.float32):
    return [torch.tensor(np.asarray(draws[p]), dtype=dtype, device="cuda", requires_grad=True)
            for p in W.PARAMS]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("recompute", [False, True])
def test_backward_equals_abi_gradient(R, cfg2, prec, recompute):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    th = leaves(draws)
    lnl = R.lnL(pt, *th, precision=prec, recompute=recompute)
    wts = torch.linspace(-1.0, 2.0, lnl.numel(), dtype=torch.float64, device="cuda")
    (lnl * wts).sum().backward()
    ref_l, ref_g = R.rift_ile_lnL_grad(pt, draws, prec)
    # recompute=True runs the forward-only kernel; otherwise the fused one
    fwd = R.rift_ile_lnL(pt, draws, prec) if recompute else ref_l
    assert torch.equal(lnl.detach(), fwd)
    for j in range(7):
        assert th[j].grad.dtype == torch.float32
        assert torch.equal(th[j].grad, (ref_g[j] * wts).to(torch.float32)), W.PARAMS[j]


def test_forward_only_without_grad(R, cfg2):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    th = [x.detach() for x in leaves(draws)]
    lnl = R.lnL(pt, *th)
    assert not lnl.requires_grad
    assert torch.equal(lnl, R.rift_ile_lnL(pt, draws, R.FP32_MIXED))


def test_partial_requires_grad(R, cfg2):
    """Only the tensors that require a gradient receive one."""
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    th = leaves(draws)
    for j in (0, 2, 4):
        th[j].requires_grad_(False)
    R.lnL(pt, *th).sum().backward()
    _, g = R.rift_ile_lnL_grad(pt, draws, R.FP32_MIXED)
    for j in range(7):
        if j in (0, 2, 4):
            assert th[j].grad is None
        else:
            assert torch.equal(th[j].grad, g[j].to(torch.float32))


def test_matches_oracle_gradient_fp64(R, cfg2):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    th = leaves(draws, torch.float64)
    R.lnL(pt, *th, precision=R.FP64).sum().backward()
    _, rg = O.lnL_grad(O.OraclePoint(point), draws)
    for j in range(7):
        g = th[j].grad.cpu().numpy()
        s = np.abs(rg[:, j]) + np.sqrt(np.mean(rg[:, j] ** 2))
        assert np.max(np.abs(g - rg[:, j]) / s) < 1e-8, W.PARAMS[j]


def test_gradcheck_fp64(R):
    """torch.autograd.gradcheck (central differences of the wrapper itself)
    on 6 prior draws of the small two-detector workload, FP64 path.  Time
    enters as t = 1e-4 tau so that one step size suits all seven inputs."""
    point, exact, info, draws, logw = W.config0(n_draws=6)
    pt = R.Point(point)
    d = dict(draws)
    d["t"] = np.asarray(d["t"]) * 1e4
    th = tuple(leaves(d, torch.float64))

    def f(ra, dec, psi, incl, phase, lnD, tau):
        return R.lnL(pt, ra, dec, psi, incl, phase, lnD, tau * 1e-4, precision=R.FP64)

    # FP64 rounding of lnL ~1e-11 over a step of 1e-6: ~1e-5 noise
    assert torch.autograd.gradcheck(f, th, eps=1e-6, atol=1e-4, rtol=1e-4, nondet_tol=0.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_backward_distance_marginalised(R, cfg2, prec):
    point, exact, info, draws, logw = cfg2
    pt = R.Point(point)
    nodes = R.rift_ile_dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)
    th = leaves(draws)
    lnl = R.lnL(pt, *th, precision=prec, dist=nodes)
    lnl.sum().backward()
    ref_l, ref_g = R.rift_ile_lnL_dist(pt, draws, nodes, prec, grad=True)
    assert torch.equal(lnl.detach(), ref_l)
    assert torch.count_nonzero(th[5].grad) == 0
    for j in range(7):
        assert torch.equal(th[j].grad, ref_g[j].to(torch.float32))
