"""Throughput of GridShift mode seeking on one GB300 (and N independent replicas).

Workload (default): a synthetic 1920x1080 image of 40 Voronoi regions, noise
sigma 10, features (R, G, B, 0.1 x, 0.1 y) in float64 (d = 5), cell side h = 12,
at most 50 updates, the plain FP64 path.  One step = one complete GridShift run
(binning, all updates until convergence, labels and modes) over the image.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: a plain single-threaded FP64 program written from the paper).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixels/s end-to-end (1080p/4K, d=3/5), FP32 vs FP64, at stated label agreement"
UNIT = "Mpixels/s"

# Bytes each unit of work must move (algorithmic, not measured):
#   binning kernel: per point, read d coordinates and write its cell slot (4 B).
def bin_bytes_per_point(d: int, elem: int) -> int:
    return d * elem + 4


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def load_workload(name: str) -> dict:
    from paper_2206_02200_gb300 import synth
    return synth.WORKLOADS[name]()


def workload_config(w: dict, name: str) -> dict:
    n, d = w["points"].shape
    return {"workload": w["name"], "n": int(n), "d": int(d), "h": w["h"],
            "max_iter": w["max_iter"], "precision": "fp64",
            "input_dtype": str(w["points"].dtype),
            "l2": "flushed between timed steps (256 MiB device write)",
            "generator": "Voronoi image, seeded (paper_2206_02200_gb300.synth)"}


def cpu_baseline(w: dict, budget_s: float = 12.0, max_runs: int = 8) -> dict:
    """Times the CPU oracle (single-threaded, as it stands) on the same workload."""
    from oracle import oracle
    oracle.build()
    X, h, it = w["points"], w["h"], w["max_iter"]
    n = X.shape[0]
    runs, total = 0, 0.0
    while runs < max_runs and (runs == 0 or total < budget_s):
        t0 = time.perf_counter()
        oracle.fit(X, h, it)
        total += time.perf_counter() - t0
        runs += 1
    return {"value": n * runs / total / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{runs} full runs of the workload ({n} points each), {total:.1f} s"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    w = load_workload(args.workload)
    from oracle import oracle
    oracle.build()
    X, h, it = w["points"], w["h"], w["max_iter"]
    n = X.shape[0]
    for _ in range(args.warmup):
        oracle.fit(X, h, it)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit(X, h, it)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * args.steps / total / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full runs of the workload ({n} points each)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2206_02200_gb300 import gridshift

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    gridshift.load()
    w = load_workload(args.workload)
    X = w["points"]
    n, d = X.shape
    elem = X.dtype.itemsize
    g = gridshift.GridShift(d, w["h"], w["max_iter"])
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    modes = torch.empty((max(n // 16, 4096), d), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        st, k, info = g.fit_into(pts, labels, modes)
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(g._ctx))
        return k, info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        step()

    # -- device-resident inputs: K timed steps, L2 flushed between them
    g.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase_ms = {p: 0.0 for p in gridshift.PHASES}
    phase_cnt = {p: 0 for p in gridshift.PHASES}
    launches = 0
    cell_iters = 0
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    clocks = ClockSampler(vis[local_rank] if local_rank < len(vis) else local_rank)
    barrier()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        k, info = step()
        ev[i][1].record(stream)
        launches += info.launches
        cell_iters += info.cell_iters
        for p, (ms, c) in g.phase_times().items():
            phase_ms[p] += ms
            phase_cnt[p] += c
    barrier()
    clk = clocks.stop()
    g.set_timing(False)
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = n * args.steps * world / (total_ms / 1e3) / 1e6

    # -- end to end through the public API: host inputs, host outputs
    h_pts = torch.from_numpy(X).pin_memory()
    h_labels = torch.empty(n, dtype=torch.int32).pin_memory()
    h_modes = torch.empty(modes.shape, dtype=torch.float64).pin_memory()
    d_pts = torch.empty_like(pts)
    e2e_steps = args.steps
    barrier()
    t0 = time.perf_counter()
    kk = 0
    for _ in range(e2e_steps):
        d_pts.copy_(h_pts, non_blocking=True)
        st, kk, info = g.fit_into(d_pts, labels, modes)
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(g._ctx))
        h_labels.copy_(labels, non_blocking=True)
        h_modes[:kk].copy_(modes[:kk], non_blocking=True)
        stream.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = n * e2e_steps * world / float(t.item()) / 1e6

    # -- roofline of the dominant kernel (binning: one launch per step)
    pk = peaks()
    bin_ms = phase_ms["bin"] / max(phase_cnt["bin"], 1)
    bin_bytes = n * bin_bytes_per_point(d, elem)
    achieved = bin_bytes / (bin_ms / 1e3) / 1e9
    roof = {"kernel": "k_bin (binning, step i)", "bound": "hbm", "achieved": achieved,
            "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
            "peak_source": f"{pk['source']} (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": bin_bytes, "avg_launch_ms": bin_ms,
            "traffic": None}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(args.warmup, 3),
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(w, args.workload),
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": int(X.nbytes),
                        "d2h_bytes_per_step": int(n * 4 + kk * d * 8)},
                "gpu_launches": int(launches),
                "roofline": roof,
                "phases_ms_per_step": {p: phase_ms[p] / args.steps for p in phase_ms},
                "active_cell_iterations_per_s": cell_iters * world / (total_ms / 1e3),
                "clocks": clk}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="image_1080p_d5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
