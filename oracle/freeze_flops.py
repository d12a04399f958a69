"""Writes oracle/flops.json: the algorithmic operation counts per draw.

The counts come from the counted plain FP64 evaluation (opcount.cpp, checked
against the oracle by tests/test_oracle_opcount.py) run on seeded draws of
each workload; they depend only on the network and the mode set (and, for the
distance marginal, the node count), not on the data, apart from the online
log-sum-exp's rare rescaling.  The benchmark reads this file as its roofline
numerator: flops per draw x draws per second.

    python oracle/freeze_flops.py            # rewrite oracle/flops.json
    python oracle/freeze_flops.py --check    # exit 1 if the file is stale
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "flops.json")
N_SAMPLE = 2048


def _per_draw(r: dict) -> dict:
    n = r["n"]
    return {"flops": r["flops"] / n, "add": r["add"] / n, "mul": r["mul"] / n,
            "div": r["div"] / n, "special": r["special"] / n}


def counts_for(point: dict, draws: dict, logw, nodes=None) -> dict:
    import oracle as O
    pt = O.OraclePoint(point)
    sub = {p: np.asarray(draws[p][:N_SAMPLE], dtype=np.float64) for p in O.PARAMS}
    lw = np.asarray(logw[:N_SAMPLE], dtype=np.float64)
    out = {
        "K": int(point["K"]), "M": int(point["M"]),
        "modes": [[int(l), int(m)] for l, m in zip(point["ell"], point["em"])],
        "draws_counted": N_SAMPLE,
        "lnZ_forward": _per_draw(O.op_counts(pt, sub, "lnZ", logw=lw)),
        "fwd_bwd": _per_draw(O.op_counts(pt, sub, "grad")),
    }
    if nodes is not None:
        x, w = nodes
        out["dist_nodes"] = int(len(x))
        out["dist_forward"] = _per_draw(O.op_counts(pt, sub, "dist", x_nodes=x, lnw_nodes=w))
        out["dist_fwd_bwd"] = _per_draw(O.op_counts(pt, sub, "dist_grad", x_nodes=x,
                                                    lnw_nodes=w))
    return out


def compute() -> dict:
    import oracle as O
    import workload as W
    res = {
        "rule": ("per-draw operations of a plain FP64 evaluation (oracle/opcount.cpp): add, "
                 "subtract, multiply and divide one flop each (a multiply-add two); sin, cos, "
                 "exp, log counted as special-function calls, not flops; per-point constants "
                 "not counted"),
        "workloads": {},
    }
    p1, _, _, d1, w1 = W.config1(n_draws=N_SAMPLE)
    res["workloads"]["3g_ile_k4_m10"] = counts_for(p1, d1, w1)
    p0, _, _, d0, w0 = W.config0(n_draws=N_SAMPLE)
    res["workloads"]["small_k2_m2"] = counts_for(p0, d0, np.zeros(N_SAMPLE))
    p4, _, _, d4, w4 = W.config4(n_draws=N_SAMPLE)
    nodes = O.dist_nodes(50.0, 200.0, 100.0, 1e-4, 1000.0)
    res["workloads"]["3g_event_k5_m10"] = counts_for(p4, d4, w4, nodes)
    return res


def main():
    res = compute()
    text = json.dumps(res, indent=1, sort_keys=True) + "\n"
    if "--check" in sys.argv:
        ok = os.path.exists(OUT) and open(OUT).read() == text
        print("flops.json up to date" if ok else "flops.json stale")
        sys.exit(0 if ok else 1)
    with open(OUT, "w") as f:
        f.write(text)
    print(OUT)


if __name__ == "__main__":
    main()
