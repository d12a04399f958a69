"""Benchmark of the extrinsic-likelihood hot path on B300.

Workload (one step): the FP32-mixed fused lnL -> lnZ pass (rift_ile_lnZ_state)
over one batch of 2^22 float32 extrinsic draws of the 3G precision
workload: an ET-like triangle plus a CE-like 40 km L (K = 4), ten modes
(2,+-1),(2,+-2),(3,+-2),(3,+-3),(4,+-4), zero-noise injection at network SNR
600, Q complex64 on a 32768 Hz table over +-20 ms (1311 samples), draws from
the defensive mixture 0.1 prior + 0.9 Gaussian about the injection.  The
draws (134 MB) exceed the 126 MB L2, so every step streams them from HBM.

The JSON line reports draws/s of that step (value), the same through the
public API with host buffers (e2e), the FP64 and lnL-output and
forward+backward variants, the error of the FP32-mixed path against the FP64
path, the ALU roofline of the kernel, sampled clocks and the FP64 CPU oracle
as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DRAWS = 1 << 22
WORKLOAD = "3G ILE: ET triangle + CE40 (K=4), 10 modes, SNR 600, 2^22 float32 draws"


def algorithmic_ops(K: int, M: int, R: int, ncls: int) -> dict:
    """Declared FP32-pipe operation count of one draw of the FP32-mixed lnL
    (the arithmetic the method needs at the stated precision, double-float
    steps charged at their FP32 operation counts: two-sum 6, two-product 2,
    pair product 7, pair sum 20, anchored sine/cosine 90, anchored exp 50).
    Overheads (addressing, loads, branches, the draw loop) are not counted."""
    df_mul, df_add, sincos, expo = 7, 20, 90, 50
    sky = 2 * sincos + 4 * df_mul + 20            # lam, dec, s and e2 products
    angles = 2 * sincos                           # 2 psi, iota/2
    per_mode_y = sincos + 10 * df_mul + 2 * df_add  # e^{i m phi}, Wigner-d polynomial, Y
    matvec = R * M * 22 + 6 * M + 12 * R          # split product a1, a2
    antenna = 15 * df_mul + 10 * df_add + 4 * df_mul + 2 * df_add
    w = 19 * R + 2 * df_mul
    time_ = 4 * df_mul + 4 * df_add + 8
    poly = 6 * (6 + df_add)
    residual = 4 * R * 4 + R + 2 * R + 45
    per_det = antenna + w + time_ + poly + residual
    total = expo + sky + angles + ncls * (M * per_mode_y + matvec) + K * per_det + 40
    return {"ops_per_draw": int(total), "per_detector": int(per_det),
            "per_class": int(M * per_mode_y + matvec)}


def plain_formula_flops(K: int, M: int) -> int:
    """FLOPs of a plain single-precision evaluation of eq. def:lnL:Decomposed
    per draw (the survey's count F(K, M))."""
    return 40 + 66 * K + 20 * M + K * (12 + 16 * M) + K * (8 * M + 6) + (K + 1) * 6 * M * (M + 1) + 10 * K + 4


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(point, draws, logw, budget_s: float = 12.0):
    """The FP64 oracle on a bounded sample of the workload's draws, all host
    cores; scaled to draws/s."""
    import oracle as O
    opt = O.OraclePoint(point)
    threads = O.default_threads()
    n = 2048
    while True:
        idx = slice(0, n)
        sub = {p: np.asarray(draws[p][idx]) for p in draws}
        t0 = time.perf_counter()
        lnl = O.lnL(opt, sub, threads=threads)
        O.lnZ(lnl, np.asarray(logw[idx], dtype=np.float64))
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n >= len(draws["t"]):
            break
        n = min(len(draws["t"]), int(n * max(2.0, min(8.0, budget_s / 4 / max(dt, 1e-3)))))
    return {"value": n / dt, "unit": "draws/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n} draws of the 2^22-draw batch, lnL + lnZ in FP64 C, {threads} threads"}


def run_reference(args, world, rank):
    """--impl reference: the FP64 CPU oracle on the same workload and metric."""
    if rank != 0:
        return
    import oracle as O
    import workload as W
    point, exact, info, draws, logw = W.config1(n_draws=N_DRAWS)
    opt = O.OraclePoint(point)
    threads = O.default_threads()
    n = 1 << 15
    sub = {p: np.asarray(draws[p][:n]) for p in draws}
    lw = np.asarray(logw[:n], dtype=np.float64)
    for _ in range(args.warmup):
        O.lnZ(O.lnL(opt, sub, threads=threads), lw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.lnZ(O.lnL(opt, sub, threads=threads), lw)
    dt = (time.perf_counter() - t0) / args.steps
    v = n / dt
    line = {
        "impl": "reference", "metric": "lnL draws/s (fwd) FP32-mixed vs FP64 at |dlnL|<=1e-3",
        "value": v, "unit": "draws/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_draws": n, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": "draws/s", "cores": threads, "kind": "oracle",
                         "sample": f"{n} draws per step, lnL + lnZ, FP64 C oracle"},
        "e2e": {"value": v, "unit": "draws/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_2609_37393_b300 as R
    import workload as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- inputs: each rank its own batch of the same workload (weak scaling)
    point, exact, info, draws, logw = W.config_3g(1, 4, 600.0, 0.02, N_DRAWS, draw_stream=1 + rank)
    pt = R.Point(point)
    d_dev = R.Draws(draws, logw)
    K, M = point["K"], point["M"]
    stream = torch.cuda.current_stream()

    # ALU peak of this GPU (roofline denominator), measured before the timing
    fp32_ops, probe_mhz = R.rift_ile_probe_alu(0, 0.2)

    def step():
        return R.rift_ile_lnZ_state(pt, d_dev, R.FP32_MIXED)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            state = step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_t = torch.tensor([ms], device="cuda")
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    value = world * N_DRAWS / (ms * 1e-3)
    lnz = R.lnZ_from_state(state)

    # ---- variants (outside the timed region; same GPU)
    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out64 = torch.empty(N_DRAWS, dtype=torch.float64, device="cuda")
    out32 = torch.empty(N_DRAWS, dtype=torch.float64, device="cuda")
    ms_fp64 = timed(lambda: R.rift_ile_lnZ_state(pt, d_dev, R.FP64), 2)
    ms_lnl = timed(lambda: R.rift_ile_lnL(pt, d_dev, R.FP32_MIXED, out32), 5)
    variants = {
        "fp32_mixed_lnZ_draws_per_s": N_DRAWS / (ms * 1e-3),
        "fp32_mixed_lnL_out_draws_per_s": N_DRAWS / (ms_lnl * 1e-3),
        "fp64_lnZ_draws_per_s": N_DRAWS / (ms_fp64 * 1e-3),
        "speedup_mixed_vs_fp64": ms_fp64 / ms,
    }
    try:
        g = torch.empty((7, N_DRAWS), dtype=torch.float64, device="cuda")
        ms_grad = timed(lambda: R.rift_ile_lnL_grad(pt, d_dev, R.FP32_MIXED, out32, g), 3)
        variants["fp32_mixed_fwd_bwd_draws_per_s"] = N_DRAWS / (ms_grad * 1e-3)
        ms_grad64 = timed(lambda: R.rift_ile_lnL_grad(pt, d_dev, R.FP64, out64, g), 1)
        variants["fp64_fwd_bwd_draws_per_s"] = N_DRAWS / (ms_grad64 * 1e-3)
        del g
    except R.RiftError as e:
        variants["fwd_bwd"] = f"unavailable: {e}"

    # precision of the measured path against the FP64 GPU path, same draws
    R.rift_ile_lnL(pt, d_dev, R.FP64, out64)
    R.rift_ile_lnL(pt, d_dev, R.FP32_MIXED, out32)
    ref = out64.cpu().numpy()
    got = out32.cpu().numpy()
    near = ref >= ref.max() - 50.0
    z64 = R.rift_ile_lnZ(pt, d_dev, R.FP64)
    precision = {
        "max_abs_dlnL_within_50nat_vs_fp64": float(np.max(np.abs(got - ref)[near])),
        "draws_within_50nat": int(near.sum()),
        "abs_dlnZ_vs_fp64": abs(lnz[0] - z64[0]),
        "lnZ": lnz[0], "sigma_lnZ": lnz[1], "n_eff": lnz[2],
    }
    del out64, out32

    # ---- end to end through the public API with host buffers
    pinned = {p: torch.from_numpy(np.ascontiguousarray(draws[p])).pin_memory() for p in W.PARAMS}
    pinned_w = torch.from_numpy(np.ascontiguousarray(logw)).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in pinned.values()) + pinned_w.numel() * 4

    def e2e_step():
        dd = R.Draws({p: pinned[p].to("cuda", non_blocking=True) for p in W.PARAMS},
                     pinned_w.to("cuda", non_blocking=True))
        return R.rift_ile_lnZ_state(pt, dd, R.FP32_MIXED)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(3, args.steps // 4)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) / max(3, args.steps // 4) * 1e3

    # ---- roofline of the dominant kernel (the fused lnL -> LSE kernel)
    pinfo = pt.info()
    ops = algorithmic_ops(K, M, pinfo["R"], pinfo["ncls"])
    achieved = ops["ops_per_draw"] * N_DRAWS / (ms * 1e-3)
    roofline = {
        "bound": "alu", "achieved": achieved / 1e12, "peak": fp32_ops / 1e12,
        "unit": "Tops/s (FP32-pipe ops, one FMA = one op)", "frac": achieved / fp32_ops,
        "traffic": None,
        "ops_per_draw": ops["ops_per_draw"],
        "peak_source": f"measured FP32 FMA issue rate at {probe_mhz:.0f} MHz (rift_ile_probe_alu)",
        "plain_formula_flops_per_draw": plain_formula_flops(K, M),
    }

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(point, draws, logw)

    if rank == 0:
        line = {
            "metric": "lnL draws/s (fwd) FP32-mixed vs FP64 at |dlnL|<=1e-3",
            "value": value, "unit": "draws/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+df (FP32 template, double-float sums)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "draws_per_step": N_DRAWS, "K": K, "M": M,
                       "R": pinfo["R"], "detector_classes": pinfo["ncls"],
                       "snr": 600, "q_len": point["Q"].shape[1],
                       "l2": "inputs (134 MB of draws) larger than the 126 MB L2"},
            "e2e": {"value": world * N_DRAWS / (e2e_ms * 1e-3), "unit": "draws/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 32 + 8},
            "gpu_launches": 2 * args.steps,
            "variants": variants,
            "precision": precision,
            "roofline": roofline,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
