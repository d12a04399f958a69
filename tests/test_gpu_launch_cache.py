"""The launch shape of each FP32-mixed kernel is its own: the occupancy cache
is keyed by the kernel, so the grid of the fused lnZ (and hence its per-block
partials and the bitwise result) does not depend on which other kernel a
process launched first.  Two fresh processes, one running lnZ alone and one
running the gradient kernel first, must print the same LSE state bit for bit.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_2609_37393_b300 as R
import workload as W
point, exact, info, draws, logw = W.config0(n_draws=1 << 16)
pt = R.Point(point)
d = R.Draws(draws, logw)
if {grad_first}:
    R.rift_ile_set_small_batch(0)
    R.rift_ile_lnL_grad(pt, d, R.FP32_MIXED)
    torch.cuda.synchronize()
st = R.rift_ile_lnZ_state(pt, d, R.FP32_MIXED)
print(json.dumps([float(v).hex() for v in st]))
"""


def run(grad_first):
    code = SCRIPT.format(root=ROOT, grad_first=grad_first)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_lnz_grid_independent_of_launch_history():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert run(False) == run(True)
