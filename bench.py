"""Benchmark of the FBIM hot path on one GB300 (replicas on N GPUs).

Workload: 1024 starfish bodies r(s) = 0.5 (1 + 0.3 cos 5s), 128 nodes each
(131072 nodes), area fraction 0.25 (box side 57.98), seeded non-overlapping
placement, Ewald tolerance 1e-8, r_c = L/115.  A step is one application of
the single-layer operator v = M mu (real-space pairs + Alpert band + Gaussian
spread, FFT, Fourier scale, inverse FFT, interpolation) to a resident force
vector; inputs and outputs stay in HBM, and L2 is flushed between timed steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokeslet matvecs/s (nodes) & mobility solves/s at 1e-6 residual: chosen vs plain FP64"
UNIT = "node-matvecs/s"
WORKLOAD = "starfish1024_np128_phi0.25"
N_BOX = 115


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def pair_count(X, L, r_c):
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(X, L), boxsize=L)
    return len(t.query_pairs(r_c))


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_matvec_rate(w, xi, n_rows=48, n_src=4096, seed=0):
    """Extrapolated oracle throughput (node-matvecs/s) from a bounded sample.

    The oracle's matrix-free matvec costs a source transform over all N sources
    (wave space) plus, per target row, a periodic real-space sum over all
    sources and a mode sum.  The sample times the transform on n_src sources
    and n_rows full rows, and scales each part to N.
    """
    from oracle import singlelayer
    X = singlelayer.node_positions(w.Q, w.ref_nodes)
    Xf = X.reshape(-1, 2)
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal((w.n, 2))
    rows = [int(r) for r in rng.choice(w.n, n_rows, replace=False)]
    t0 = time.perf_counter()
    singlelayer.apply_real_rows(X, mu, rows, w.L, xi)
    t_real = time.perf_counter() - t0
    mu_s = np.zeros_like(mu)
    src = rng.choice(w.n, n_src, replace=False)
    mu_s[src] = mu[src]
    t0 = time.perf_counter()
    singlelayer.apply_wave_rows(Xf, mu_s, rows, w.L, xi, cut=30.0)
    t_wave = time.perf_counter() - t0
    t_full = t_real * (w.n / n_rows) + t_wave * (w.n / n_src)
    sample = (f"{n_rows} target rows of the real-space sum over all {w.n} sources, and the wave-space "
              f"lattice sum with {n_src} of {w.n} sources and the same rows; each part scaled to one "
              f"full matvec ({t_full:.1f} s)")
    return w.n / t_full, t_full, sample


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import fbim_synth
    w = fbim_synth.workload(WORKLOAD)
    xi = math.sqrt(math.log(100.0 / w.tol)) / (w.L / N_BOX)
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, t_full, sample = oracle_matvec_rate(w, xi, n_rows=16, n_src=1024, seed=i)
        if i >= args.warmup:
            vals.append(t_full)
    t = float(np.mean(vals))
    value = w.n / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_nodes": w.n, "tol": w.tol, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_steps(torch, op, mu, v, steps, flush, stream):
    """Per-step CUDA-event times (ms) with an L2 flush before each step."""
    times = []
    for _ in range(steps):
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        op.apply_stokeslet(mu, out=v)
        e.record(stream)
        e.synchronize()
        times.append(s.elapsed_time(e))
    return times


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import fbim_synth
    import paper_1709_01480_gb300 as fb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    peaks, peak_kind = load_peaks()

    w = fbim_synth.workload(WORKLOAD)
    xi = math.sqrt(math.log(100.0 / w.tol)) / (w.L / N_BOX)
    ops = {p: fb.FBIM(w.ref_nodes, w.Q, w.L, tol=w.tol, r_c=w.L / N_BOX, xi=xi, precision=p)
           for p in ("fp32", "fp64")}
    info = ops["fp32"].info
    g = torch.Generator(device="cuda").manual_seed(1234 + rank)
    mu = torch.randn((w.n, 2), dtype=torch.float64, device="cuda", generator=g)
    v = torch.empty_like(mu)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for p in ("fp32", "fp64"):
        for _ in range(args.warmup):
            ops[p].apply_stokeslet(mu, out=v)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: chosen form (FP32 operator) --------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    t32 = time_steps(torch, ops["fp32"], mu, v, args.steps, flush, stream)
    barrier()
    clk = clocks.stop()
    ms32 = float(np.sum(t32)) / args.steps
    if world > 1:
        tt = torch.tensor([ms32], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms32 = float(tt.item())
    value = world * w.n / (ms32 * 1e-3)

    # ---- plain FP64 operator --------------------------------------------------
    barrier()
    t64 = time_steps(torch, ops["fp64"], mu, v, args.steps, flush, stream)
    ms64 = float(np.sum(t64)) / args.steps

    # ---- per-stage times (dominant kernel) -----------------------------------
    stage = {}
    for p in ("fp32", "fp64"):
        op = ops[p]
        op.set_timing(True)
        for _ in range(args.steps):
            flush.zero_()
            op.apply_stokeslet(mu, out=v)
        stage[p] = {k: ms / max(c, 1) for k, (ms, c) in op.stage_times().items()}
        op.set_timing(False)

    M, N = info["grid"], w.n
    n_pairs = pair_count(singlelayer_positions(w), w.L, info["r_c"])
    n_entries = info["pair_entries"]
    # minimum DRAM bytes per launch of each stage, FP32 operator (grids: 2 components x 4 B;
    # half spectrum: 2 x M (M/2 + 1) complex x 8 B; node vectors: 8 B per node and order)
    spec_b = 16 * M * (M // 2 + 1)
    algo_bytes = {
        "gather": N * (4 + 4 + 16 + 8 + 8),            # perm, tperm, mu (FP64), two FP32 copies
        "spread": 24 * N + 8 * M * M,                   # tbase, tfrac, mu_t; grid written once
        "fft_fwd": 8 * M * M + spec_b,
        "scale": 2 * spec_b,
        "fft_inv": spec_b + 8 * M * M,
        "pairs": 16 * n_entries + 8 * N + 8 * N,        # pair list streamed once, mu_s, v_s
        "interp": 8 * M * M + 24 * N + 8 * N,
        "finish": N * (4 + 4 + 8 + 8 + 16 + 16) + 16 * N,   # slots, v_s, v_t, mu band reads, v
    }
    st32 = stage["fp32"]
    hbm_stages = {k: v_ for k, v_ in st32.items() if k in algo_bytes}
    dom = max(hbm_stages, key=lambda k: hbm_stages[k])
    dom_ms = hbm_stages[dom]
    achieved = algo_bytes[dom] / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_kind": peak_kind, "algorithmic_bytes": algo_bytes[dom], "launch_ms": dom_ms}

    # ---- end to end through the public API with host buffers ----------------
    mu_h = torch.empty((w.n, 2), dtype=torch.float64, pin_memory=True)
    mu_h.copy_(mu.cpu())
    v_h = torch.empty((w.n, 2), dtype=torch.float64, pin_memory=True)
    mu_d = torch.empty_like(mu)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        mu_d.copy_(mu_h, non_blocking=True)
        ops["fp32"].apply_stokeslet(mu_d, out=v)
        v_h.copy_(v, non_blocking=True)
        e.record(stream)
        e.synchronize()
        e2e_ms.append(s.elapsed_time(e))
    e2e = {"value": world * w.n / (float(np.mean(e2e_ms)) * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": mu_h.numel() * 8, "d2h_bytes_per_step": v_h.numel() * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, t_full, sample = oracle_matvec_rate(w, xi)
        cpu = {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample}

    launches_per_step = 6  # gather, spread, scale, pairs, interp, finish (+ 2 cuFFT calls, library)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_nodes": N, "n_bodies": w.n_b, "box": w.L, "tol": w.tol,
                       "xi": info["xi"], "r_c": info["r_c"], "grid": M, "support": info["support"],
                       "n_pairs_within_rc": n_pairs, "pair_entries": n_entries, "tile": info["tile"],
                       "wave_variant": info["wave_variant"], "variant_ms": info["variant_ms"],
                       "l2": "flushed (256 MB write) before every timed step",
                       "operator": "FP32 Ewald operator, FP64 Alpert band"},
            "plain_fp64": {"value": world * w.n / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64},
            "stage_ms": {"fp32": st32, "fp64": stage["fp64"]},
            "roofline": roofline,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for op in ops.values():
        op.close()
    if world > 1:
        dist.destroy_process_group()


def singlelayer_positions(w):
    c, s = np.cos(w.Q[:, 2]), np.sin(w.Q[:, 2])
    gx, gy = w.ref_nodes[:, 0], w.ref_nodes[:, 1]
    x = w.Q[:, None, 0] + c[:, None] * gx[None, :] - s[:, None] * gy[None, :]
    y = w.Q[:, None, 1] + s[:, None] * gx[None, :] + c[:, None] * gy[None, :]
    return np.stack([x.ravel(), y.ravel()], axis=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
