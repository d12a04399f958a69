"""Multi-rank lnZ on CPU ranks (gloo, world size 2 and 3): each rank owns a
contiguous shard of the draws, reduces it to an LSE state, and the ranks
exchange only those states (lnZ_merge_ranks, which calls the library's
rift_ile_lnZ_merge).  The merged lnZ, sigma and n_eff equal the oracle's over
all draws; shards cover the draws exactly once."""
import math
import os
import socket

import numpy as np
import pytest

import oracle as O
import workload as W

torch = pytest.importorskip("torch")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def state_of(x):
    """LSE state of the log-weights x (test-side, from oracle lnL values)."""
    if x.size == 0:
        return (-math.inf, 0.0, 0.0, 0.0)
    m = float(np.max(x))
    return (m, float(np.sum(np.exp(x - m))), float(np.sum(np.exp(2 * (x - m)))), float(x.size))


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import paper_2609_37393_b300 as R
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        point, exact, info, draws, logw = W.config0(n_draws=3000)
        a, b = R.shard_bounds(3000, rank, world)
        sub = {p: np.asarray(draws[p])[a:b] for p in W.PARAMS}
        lnl = O.lnL(O.OraclePoint(point), sub)
        res, merged = R.lnZ_merge_ranks(state_of(lnl + np.asarray(logw)[a:b]))
        q.put((rank, a, b, res, merged))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_lnz_matches_oracle(world):
    import multiprocessing as mp
    try:
        import paper_2609_37393_b300  # noqa: F401  (the library must be built)
    except ImportError as e:
        pytest.skip(str(e))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    bounds = [(a, b) for _, a, b, _, _ in out]
    assert bounds[0][0] == 0 and bounds[-1][1] == 3000
    assert all(bounds[i][1] == bounds[i + 1][0] for i in range(world - 1))
    point, exact, info, draws, logw = W.config0(n_draws=3000)
    ref = O.lnZ(O.lnL(O.OraclePoint(point), draws), np.asarray(logw, dtype=np.float64))
    for _, _, _, res, merged in out:
        assert res == out[0][3]  # every rank gets the same merge
        assert abs(res[0] - ref[0]) <= 1e-12 * max(1.0, abs(ref[0]))
        assert abs(res[1] - ref[1]) <= 1e-9 * ref[1]
        assert abs(res[2] - ref[2]) <= 1e-9 * ref[2]
        assert merged[3] == 3000


def test_shard_bounds_cover_exactly():
    try:
        import paper_2609_37393_b300 as R
    except ImportError as e:
        pytest.skip(str(e))
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = R.shard_bounds(n, r, world)
                seen.extend(range(a, b))
                assert b - a in (n // world, n // world + 1)
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        R.shard_bounds(10, 2, 2)
