"""GPU parity of the batched lnZ over many intrinsic points (config-3 shapes:
2-5 detectors, 2-10 modes, 8k-65k-sample tables, uneven draw counts).

FP32-mixed batch: each point's lnZ matches the FP64 oracle within 1e-4 (six
points, and 64 points in one launch against the oracle as well) and
the single-point rift_ile_lnZ within 1e-6; FP64 batch matches the oracle
within 1e-9 max(1, |lnZ|).  The launch replays identically from a captured
CUDA graph and is deterministic.
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
def batch_inputs():
    pts = [W.config3_point(i) for i in (0, 1, 2, 3, 5, 8)]
    return pts


@pytest.fixture(scope="module")
def oracle_lnz(batch_inputs):
    out = []
    for point, exact, info, draws, logw in batch_inputs:
        lnl = O.lnL(O.OraclePoint(point), draws)
        out.append(O.lnZ(lnl, np.asarray(logw, dtype=np.float64)))
    return out


def test_batch_mixed_matches_oracle_and_single(R, batch_inputs, oracle_lnz):
    points = [R.Point(p[0]) for p in batch_inputs]
    draws = [R.Draws(p[3], p[4]) for p in batch_inputs]
    b = R.Batch(points, draws, R.FP32_MIXED)
    out = b.launch().cpu().numpy()
    for i, (ref, pt, d) in enumerate(zip(oracle_lnz, points, draws)):
        assert abs(out[i, 0] - ref[0]) <= 1e-4, (i, out[i], ref)
        assert abs(out[i, 2] - ref[2]) <= 1e-3 * ref[2]
        single = R.rift_ile_lnZ(pt, d, R.FP32_MIXED)
        assert abs(out[i, 0] - single[0]) <= 1e-6 * max(1, abs(single[0]))


def test_batch_fp64_matches_oracle(R, batch_inputs, oracle_lnz):
    points = [R.Point(p[0]) for p in batch_inputs]
    draws = [R.Draws(p[3], p[4]) for p in batch_inputs]
    out = R.Batch(points, draws, R.FP64).launch().cpu().numpy()
    for i, ref in enumerate(oracle_lnz):
        assert abs(out[i, 0] - ref[0]) <= 1e-9 * max(1, abs(ref[0])), (i, out[i], ref)
        assert abs(out[i, 2] - ref[2]) <= 1e-6 * ref[2]


def test_batch_graph_replay_and_determinism(R, batch_inputs):
    points = [R.Point(p[0]) for p in batch_inputs[:4]]
    draws = [R.Draws(p[3], p[4]) for p in batch_inputs[:4]]
    b = R.Batch(points, draws, R.FP32_MIXED)
    eager = b.launch()
    again = b.launch()
    assert torch.equal(eager, again)
    out = torch.empty_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.launch(out, stream=s)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.launch(out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_batch_with_empty_point(R, batch_inputs):
    p0 = batch_inputs[0]
    empty = {p: np.zeros(0, dtype=np.float32) for p in W.PARAMS}
    points = [R.Point(p0[0]), R.Point(p0[0])]
    draws = [R.Draws(empty, np.zeros(0, dtype=np.float32)), R.Draws(p0[3], p0[4])]
    out = R.Batch(points, draws, R.FP32_MIXED).launch().cpu().numpy()
    assert out[0, 0] == -np.inf and out[0, 2] == 0
    single = R.rift_ile_lnZ(points[1], draws[1], R.FP32_MIXED)
    assert abs(out[1, 0] - single[0]) <= 1e-6 * max(1, abs(single[0]))


def test_batch_autotune_keeps_results(R, batch_inputs):
    """The autotuner picks a tile size and grid by timing; the tuned launch
    gives the same lnZ to rounding, stays deterministic and replays from a
    graph captured after tuning."""
    points = [R.Point(p[0]) for p in batch_inputs]
    draws = [R.Draws(p[3], p[4]) for p in batch_inputs]
    b = R.Batch(points, draws, R.FP32_MIXED)
    before = b.launch().cpu().numpy()
    tile, blocks, ms = b.tune(reps=2)
    assert tile in (512, 1024, 2048, 4096, 8192, 16384) and blocks >= 1 and ms > 0
    after = b.launch()
    a = after.cpu().numpy()
    assert np.all(np.abs(a[:, 0] - before[:, 0]) <= 1e-9 * np.maximum(1, np.abs(before[:, 0])))
    assert np.allclose(a[:, 1:], before[:, 1:], rtol=1e-6)
    assert torch.equal(b.launch(), after)
    out = torch.empty_like(after)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.launch(out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.launch(out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, after)


def test_fp64_batch_tune_is_a_no_op(R, batch_inputs):
    points = [R.Point(p[0]) for p in batch_inputs[:2]]
    draws = [R.Draws(p[3], p[4]) for p in batch_inputs[:2]]
    b = R.Batch(points, draws, R.FP64)
    tile, blocks, ms = b.tune(reps=1)
    assert ms == -1.0


def test_batch_64_points_against_oracle(R):
    """64 config-3 points (2-5 detectors, 2-10 modes, uneven draw counts) in
    one batched launch, both precisions, every point's lnZ against the
    oracle: FP32-mixed within 1e-4, FP64 within 1e-9 max(1, |lnZ|)."""
    inputs = [W.config3_point(i) for i in range(64)]
    points = [R.Point(p[0]) for p in inputs]
    draws = [R.Draws(p[3], p[4]) for p in inputs]
    o32 = R.Batch(points, draws, R.FP32_MIXED).launch().cpu().numpy()
    o64 = R.Batch(points, draws, R.FP64).launch().cpu().numpy()
    for i, (point, exact, info, d, logw) in enumerate(inputs):
        ref = O.lnZ(O.lnL(O.OraclePoint(point), d), np.asarray(logw, dtype=np.float64))
        assert abs(o32[i, 0] - ref[0]) <= 1e-4, (i, o32[i], ref)
        assert abs(o64[i, 0] - ref[0]) <= 1e-9 * max(1, abs(ref[0])), (i, o64[i], ref)
