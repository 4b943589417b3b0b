"""Throughput of GridShift mode seeking on one GB300 (and N independent replicas).

Workload (default): a synthetic 1920x1080 image of 40 Voronoi regions, noise
sigma 10, features (R, G, B, 0.1 x, 0.1 y) in float64 (d = 5), cell side h = 12,
at most 50 updates, the plain FP64 path.  One step = one complete GridShift run
(binning, all updates until convergence, labels and modes) over the image.
``--precision fp32`` runs the float32 mixed-precision path and reports its
label agreement and mode error against the FP64 path; ``--workload
batch_64_d3`` runs 64 uneven images in one batched call (and times 64
sequential plain calls beside it); ``--update sequential`` runs the
sequential update of Eq. 5 (float64, one point set) instead of the parallel
one of Eq. 6.

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

# Bytes each unit of work must move (algorithmic, not measured).
#
# The loop kernel (k_loop: the cell levels, steps ii-v), counted in 32-byte
# sectors as the scope states (the roofline's `achieved`): per active cell
# and update step (the stop test's step included, which probes too), one
# 32-byte key sector for each of the 3^d neighbour probes (Eq. 1), two
# payload sectors (the cell's own row and one neighbour row), the new
# centroid and key written (d x elem + 8 B), and the merge (a radix sort of 4
# passes over 12-byte (key, id) pairs, 48 B, plus a segmented reduction
# reading and writing the payload, 2 x (4 + d x elem) B).  Its DRAM count
# (what must leave the chip when the level tables stay in L2): per active
# cell and update step, its row read once and the next level's row and key
# written once (rows: count + d sums, 16 (d + 1) B in FP64, 4 (d + 1) B in
# FP32; keys 8 B).
#
# The per-point launches, DRAM bytes per point:
#   k_bin (binning, first pass): its d coordinates read, its cell slot
#     written (4 B);
#   k_prep_scatter: the slot read, the counting-sort position written (8 B);
#   k_prep_sums: the position and the slot read again, the d coordinates
#     re-read (8 + d x elem B);
#   k_labels_out: the slot read, the label written (8 B).
def bin_bytes_per_point(d: int, elem: int) -> int:
    return d * elem + 4


def per_point_bytes(kernel: str, d: int, elem: int) -> int:
    return {"bin": d * elem + 4, "k_scatter": 8, "k_sums": 8 + d * elem, "labels_out": 8}[kernel]


def loop_bytes(cell_steps: int, d: int, fp32: bool) -> int:
    """The DRAM count of k_loop per launch."""
    row = (4 if fp32 else 16) * (d + 1)
    return cell_steps * (2 * row + 8)


def scope_bytes_per_cell_step(d: int, fp32: bool) -> int:
    """The scope count per active cell and update step."""
    e = 4 if fp32 else 8
    return 3 ** d * 32 + 2 * 32 + (d * e + 8) + 48 + 2 * (4 + d * e)


def loop_scope_bytes(probe_cell_steps: int, d: int, fp32: bool) -> int:
    """The scope count of k_loop per launch (probe_cell_steps = active cells
    summed over every update step that probed, the stop test's included)."""
    return probe_cell_steps * scope_bytes_per_cell_step(d, fp32)


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from the committed ncu captures under profiles/, keyed by (workload,
# precision, kernel), each with the hash of the kernel sources it was taken
# on (the files that define k_range, k_bin and k_loop, not the host
# code): a figure is reported only while those sources still hash the same.
TRAFFIC = {
    ("image_1080p_d5", "fp64", "k_loop"): (147.09e6, "2e374b84c1aa7d39"),
    ("image_1080p_d5", "fp64", "k_bin"): (85.97e6, "2e374b84c1aa7d39"),
    # the 4M-point mixture with the per-point passes as launches of their own
    # (--tune split_min=0); taken on the sources before the image-feature
    # kernel's last change (the kernels below are the same code, but a figure
    # is reported only under the hash it was taken on)
    ("gmm_4M_d6", "fp64", "k_loop"): (1466.28e6, "1b49d2decd1369a4"),
    ("gmm_4M_d6", "fp64", "k_bin"): (105.81e6, "1b49d2decd1369a4"),
    ("gmm_4M_d6", "fp64", "k_prep_scatter"): (20.13e6, "1b49d2decd1369a4"),
    ("gmm_4M_d6", "fp64", "k_prep_sums"): (378.93e6, "1b49d2decd1369a4"),
    ("gmm_4M_d6", "fp32", "k_loop"): (880.22e6, "1b49d2decd1369a4"),
    # the 10M-point mixture: the 4M-point captures scaled by the units one
    # launch processes (points for the per-point kernels, x 2.5; active
    # cell-updates for k_loop, 285,298 against 205,764, x 1.3865)
    ("gmm_10M_d6", "fp64", "k_loop"): (2033.0e6, "1b49d2decd1369a4"),
    ("gmm_10M_d6", "fp64", "k_bin"): (264.5e6, "1b49d2decd1369a4"),
    ("gmm_10M_d6", "fp64", "k_prep_scatter"): (50.3e6, "1b49d2decd1369a4"),
    ("gmm_10M_d6", "fp64", "k_prep_sums"): (947.3e6, "1b49d2decd1369a4"),
    ("gmm_10M_d6", "fp32", "k_loop"): (1220.4e6, "1b49d2decd1369a4"),
}


KERNEL_SOURCES = ("gs_common.cuh", "gs_device.cuh", "gs_kernels.cu", "gs_kernels.h",
                  "gs_loop.cuh", "gs_loop_base.cuh", "gs_loop_fp64.cuh", "gs_loop_fp32.cuh",
                  "gs_loop_tail.cuh", "gs_loop_kernel.cuh", "gs_loop32.cu", "gs_loop64.cu",
                  "gs_plan.h", "gs_planner.cuh")


def sources_hash() -> str:
    import hashlib
    m = hashlib.sha256()
    for name in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_2206_02200_gb300", "csrc", name)
        m.update(name.encode())
        with open(p, "rb") as f:
            m.update(f.read())
    return m.hexdigest()[:16]


def traffic(workload: str, precision: str, kernel: str, update: str = "parallel"):
    """DRAM bytes per launch from the committed capture, or None when none was
    taken for this case or the kernel sources changed since."""
    if update != "parallel":
        return None
    t = TRAFFIC.get((workload, precision, kernel))
    return t[0] if t and t[1] == sources_hash() else None


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


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the job's ranks (a job's time is its slowest
    rank's); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput in millions of units per second: every rank
    processes units_per_rank per step, and the job takes `seconds`."""
    return units_per_rank * steps * world / seconds / 1e6


def load_workload(name: str) -> dict:
    from paper_2206_02200_gb300 import synth
    return synth.WORKLOADS[name]()


def workload_config(w: dict, name: str, precision: str = "fp64", update: str = "parallel") -> dict:
    if "parts" in w:
        n, d = sum(len(p) for p in w["parts"]), w["parts"][0].shape[1]
        dt = w["parts"][0].dtype
    else:
        (n, d), dt = w["points"].shape, w["points"].dtype
    gen = ("GMM points, seeded" if name.startswith("gmm") else "Voronoi image, seeded")
    cfg = {"workload": w["name"], "n": int(n), "d": int(d), "h": w["h"],
           "max_iter": w["max_iter"], "precision": precision, "update": update,
           "input_dtype": str(dt),
           "l2": "flushed between timed steps (256 MiB device write)",
           "generator": gen + " (paper_2206_02200_gb300.synth)"}
    if "parts" in w:
        cfg["instances"] = len(w["parts"])
    if "hs" in w:
        cfg["hs"] = list(w["hs"])
        cfg["instances"] = len(w["hs"])
    return cfg


def _oracle_sample(w: dict):
    """The CPU oracle's share of the workload: the whole point set (for the
    shuffled Gaussian-mixture workloads its first million points, a uniform
    subsample: the single-threaded oracle needs minutes for ten million
    six-dimensional points), or for a batched workload its first instances up
    to about 1.5 M points."""
    if "parts" not in w:
        X = w["points"]
        if w["name"].startswith("gmm") and len(X) > 1_000_000:
            return [X[:1_000_000]]
        return [X]
    out, tot = [], 0
    for p in w["parts"]:
        out.append(p)
        tot += len(p)
        if tot >= 1_500_000:
            break
    return out


def _sample_what(w: dict, sample) -> str:
    if "parts" in w:
        return f"the first {len(sample)} instances"
    if len(sample[0]) < len(w["points"]):
        return f"the first {len(sample[0])} points of the shuffled workload"
    return "the workload"


def host_cores() -> int:
    """Cores this process may run on (the host's, unless restricted)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


def _oracle_worker(paths, hs, it, update, cmd_q, done_q):
    """One oracle process: loads its copy of the sample, then runs the oracle
    once over it (for every bandwidth in hs) per command until told to stop."""
    import numpy as np
    from oracle import oracle
    sample = [np.load(p) for p in paths]
    oracle.lib()
    done_q.put(("ready", 0.0))
    while True:
        c = cmd_q.get()
        if c is None:
            return
        t0 = time.perf_counter()
        for X in sample:
            for h in hs:
                oracle.fit(X, h, it, update=update)
        done_q.put(("done", time.perf_counter() - t0))


class OracleWorkers:
    """P spawn-method processes, each running the oracle (as it stands,
    single-threaded) on its own copy of the sample: one step = every process
    runs the sample once, timed by wall clock from the command to the last
    completion.  The oracle is not parallelised; the host's cores run P
    independent copies of it (spawn, so no process inherits a CUDA context)."""

    def __init__(self, sample, hs, it, update="parallel", procs=None):
        import multiprocessing
        import tempfile

        import numpy as np
        from oracle import oracle
        oracle.build()
        self.procs = procs or host_cores()
        self.tmp = tempfile.mkdtemp(prefix="gs_oracle_sample_")
        paths = []
        for i, X in enumerate(sample):
            pth = os.path.join(self.tmp, f"part{i}.npy")
            np.save(pth, np.ascontiguousarray(X))
            paths.append(pth)
        ctx = multiprocessing.get_context("spawn")
        self.cmd = [ctx.Queue() for _ in range(self.procs)]
        self.done = ctx.Queue()
        self.ps = [ctx.Process(target=_oracle_worker, args=(paths, hs, it, update, q, self.done),
                               daemon=True) for q in self.cmd]
        for pr in self.ps:
            pr.start()
        for _ in self.ps:
            self.done.get(timeout=600)

    def step(self) -> float:
        t0 = time.perf_counter()
        for q in self.cmd:
            q.put(1)
        for _ in self.ps:
            self.done.get(timeout=3600)
        return time.perf_counter() - t0

    def close(self):
        import shutil
        for q in self.cmd:
            q.put(None)
        for pr in self.ps:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()
        shutil.rmtree(self.tmp, ignore_errors=True)


def cpu_baseline(w: dict, budget_s: float = 12.0, max_runs: int = 8,
                 update: str = "parallel", results: list | None = None) -> dict:
    """Times the CPU oracle (as it stands) on the same workload: single-threaded
    (a bounded number of full runs of the sample), and on all the host's cores
    as independent copies (two steps of OracleWorkers).  The all-core figure is
    the line's value; the single-core one is nested.  With `results`, the
    first run's oracle result is appended to it when that run covered the
    whole workload (one point set, one bandwidth)."""
    from oracle import oracle
    oracle.build()
    sample = _oracle_sample(w)
    hs, it = w.get("hs", [w["h"]]), w["max_iter"]
    n = sum(len(X) for X in sample) * len(hs)
    whole = "parts" not in w and len(hs) == 1 and len(sample[0]) == len(w["points"])
    runs, total = 0, 0.0
    while runs < max_runs and (runs == 0 or total < budget_s):
        t0 = time.perf_counter()
        for X in sample:
            for h in hs:
                r = oracle.fit(X, h, it, update=update)
        total += time.perf_counter() - t0
        if runs == 0 and whole and results is not None:
            results.append(r)
        runs += 1
    what = _sample_what(w, sample)
    single = {"value": n * runs / total / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{runs} full runs of {what} ({n} points each), {total:.1f} s"}
    ow = OracleWorkers(sample, hs, it, update)
    try:
        ts = [ow.step() for _ in range(2)]
    finally:
        ow.close()
    P = ow.procs
    return {"value": n * P * len(ts) / sum(ts) / 1e6, "unit": UNIT, "cores": P, "kind": "oracle",
            "nproc": host_cores(),
            "sample": (f"{len(ts)} steps of {P} independent single-threaded oracle processes, "
                       f"each running {what} ({n} points) once per step, {sum(ts):.1f} s"),
            "single_core": single}


def oracle_agreement(lab, md, k: int, iterations: int, ref: dict, h: float) -> dict:
    """The FP64 path's result (labels, the k modes, iterations) against the
    oracle's on the same workload: the partition and its numbering, the
    cluster count, the iteration count and the modes bit for bit, with the
    largest mode difference in units of h."""
    import numpy as np
    lab_ref, md_ref, k_ref = ref["labels"], ref["modes"][:int(ref["k"])], int(ref["k"])
    same_shape = lab.shape == lab_ref.shape
    out = {"against": "the oracle (FP64), the same workload, its first cpu_baseline run",
           "labels": float(np.mean(lab == lab_ref)) if same_shape and lab.size else
           (1.0 if same_shape else 0.0),
           "labels_identical": bool(same_shape and np.array_equal(lab, lab_ref)),
           "k": int(k), "k_ref": k_ref,
           "iterations": int(iterations), "iterations_ref": int(ref["iterations"])}
    if k == k_ref and md.shape == md_ref.shape:
        out["modes_bit_identical"] = bool(np.array_equal(md.view(np.int64), md_ref.view(np.int64)))
        out["max_mode_error_h"] = float(np.max(np.abs(md - md_ref))) / h if k_ref else 0.0
    else:
        out["modes_bit_identical"] = False
        out["max_mode_error_h"] = None
    return out


def run_reference(args, rank: int, world: int):
    """The reference arm: the oracle as it stands, as P independent
    single-threaded processes over the host's cores; one step = each process
    runs the sample once."""
    if rank != 0:
        return 0
    w = load_workload(args.workload)
    sample = _oracle_sample(w)
    hs, it = w.get("hs", [w["h"]]), w["max_iter"]
    n = sum(len(X) for X in sample) * len(hs)
    ow = OracleWorkers(sample, hs, it, args.update)
    try:
        for _ in range(args.warmup):
            ow.step()
        times = [ow.step() for _ in range(args.steps)]
    finally:
        ow.close()
    P = ow.procs
    total = sum(times)
    value = n * P * args.steps / total / 1e6
    what = _sample_what(w, sample)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps,
            "median_ms_per_step": 1e3 * statistics.median(times) if times else None,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k: v for k, v in workload_config(w, args.workload, update=args.update).items()
                       if k != "l2"},  # host cores: no device cache to flush
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                             "nproc": host_cores(),
                             "sample": (f"{args.steps} steps of {P} independent single-threaded "
                                        f"oracle processes, each running {what} ({n} points) "
                                        f"once per step")},
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
    batched = "parts" in w
    if batched:
        X = np.ascontiguousarray(np.concatenate(w["parts"], 0))
        offsets = np.concatenate([[0], np.cumsum([len(p) for p in w["parts"]])]).tolist()
    else:
        X = w["points"]
    n, d = X.shape
    elem = X.dtype.itemsize
    fp32 = args.precision == "fp32"
    prec = gridshift.GS_FP32_MIXED if fp32 else gridshift.GS_FP64
    form = (gridshift.GS_UPDATE_SEQUENTIAL if args.update == "sequential"
            else gridshift.GS_UPDATE_PARALLEL)
    g = gridshift.GridShift(d, w["h"], w["max_iter"], precision=prec, update=form,
                            tuning="auto" if args.tuning == "auto" else None)
    g._apply_auto_tuning(n, batched)
    if args.tune:
        t = g.tuning()
        for kv in args.tune:
            k, v = kv.split("=", 1)
            t[k] = int(v, 0)
        if gridshift.gs_set_tuning(g._ctx, t) != gridshift.GS_OK:
            raise SystemExit(f"bad --tune {args.tune}")
        g.tuning_source += " + " + ",".join(args.tune)
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    modes = torch.empty((max(n // 16, 4096), d), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call(p, lab, md, gg=g):
        if batched:
            st, mo, infos = gridshift.gs_fit_batched(gg._ctx, p.data_ptr(), gridshift.GS_IN_F64
                                                     if p.dtype == torch.float64 else
                                                     gridshift.GS_IN_F32, offsets,
                                                     lab.data_ptr(), md.data_ptr(), md.shape[0])
            if st != gridshift.GS_OK:
                raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(gg._ctx))
            return mo[-1], [x.as_dict() for x in infos]
        # the C entry point itself (the context's stream and launch choices
        # are set once, outside the timed calls)
        st, k, info = gridshift.gs_fit(gg._ctx, p.data_ptr(), dt_in, n, lab.data_ptr(),
                                       md.data_ptr(), md.shape[0])
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(gg._ctx))
        return k, [info.as_dict()]

    gridshift.gs_set_stream(g._ctx, stream.cuda_stream)
    dt_in = gridshift.GS_IN_F64 if X.dtype == np.float64 else gridshift.GS_IN_F32

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        call(pts, labels, modes)

    # -- device-resident inputs: K timed steps, L2 flushed between them
    g.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase_ms = {p: 0.0 for p in gridshift.PHASES}
    phase_cnt = {p: 0 for p in gridshift.PHASES}
    launches = 0
    cell_iters = 0
    m0_total = 0
    k_total = 0
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    clocks = ClockSampler(vis[local_rank] if local_rank < len(vis) else local_rank)
    barrier()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        k, infos = call(pts, labels, modes)
        ev[i][1].record(stream)
        launches += infos[0]["launches"]
        cell_iters += sum(x["cell_iters"] for x in infos)
        m0_total += sum(x["m0"] for x in infos)
        k_total += sum(x["k"] for x in infos)
        if not batched:
            for p, (ms, c) in g.phase_times().items():
                phase_ms[p] += ms
                phase_cnt[p] += c
    barrier()
    clk = clocks.stop()
    g.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # the last timed step's result (outside the timed region), for the
    # comparison with the oracle
    last = None
    if not batched and not fp32:
        last = (labels.cpu().numpy().copy(), modes[:k].cpu().numpy().copy(), int(k),
                int(infos[0]["iterations"]))
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    median_ms = max_over_ranks(statistics.median(step_ms), world, dev)
    value = job_rate(n, args.steps, world, total_ms / 1e3)

    # -- agreement of the float32 path with the FP64 path (which the tests
    #    hold bit-identical to the oracle)
    agreement = None
    if fp32:
        lab32 = labels.cpu().numpy().copy()
        md32 = modes[:k].cpu().numpy().copy()
        g64 = gridshift.GridShift(d, w["h"], w["max_iter"])
        gridshift.gs_set_stream(g64._ctx, stream.cuda_stream)
        lab64 = torch.empty_like(labels)
        md64 = torch.empty_like(modes)
        k64, infos64 = call(pts, lab64, md64, g64)
        torch.cuda.synchronize(dev)
        l64, m64 = lab64.cpu().numpy(), md64[:k64].cpu().numpy()
        from paper_2206_02200_gb300 import agreement as agm
        if batched:
            agree_n, err, k32, k64, worst = 0.0, 0.0, 0, 0, 1.0
            mo32 = np.concatenate([[0], np.cumsum([x["k"] for x in infos])])
            mo64 = np.concatenate([[0], np.cumsum([x["k"] for x in infos64])])
            for b in range(len(offsets) - 1):
                s0, s1 = offsets[b], offsets[b + 1]
                ab = agm.agreement(lab32[s0:s1], l64[s0:s1], md32[mo32[b]:mo32[b + 1]],
                                   m64[mo64[b]:mo64[b + 1]], w["h"])
                agree_n += ab["labels"] * (s1 - s0)
                worst = min(worst, ab["labels"])
                err = max(err, ab["max_mode_error_h"])
                k32 += ab["k"]
                k64 += ab["k_ref"]
            ag = {"labels": agree_n / n, "worst_instance_labels": worst,
                  "max_mode_error_h": err, "k": k32, "k_ref": k64}
        else:
            ag = agm.agreement(lab32, l64, md32, m64, w["h"])
            ag.pop("matched", None)
        agreement = dict(ag, metric="clusters matched one to one, greedily by overlap",
                         face_rechecks_per_step=sum(x["face_rechecks"] for x in infos),
                         against="FP64 GPU path (bit-identical to the FP64 oracle in the tests)")
        g64.close()

    # -- sequential plain calls beside the batched one
    sequential = None
    if batched:
        gp = gridshift.GridShift(d, w["h"], w["max_iter"])
        gridshift.gs_set_stream(gp._ctx, stream.cuda_stream)
        parts_dev = [pts[offsets[b]:offsets[b + 1]] for b in range(len(offsets) - 1)]
        def plain(P):
            return gridshift.gs_fit(gp._ctx, P.data_ptr(), dt_in, P.shape[0], labels.data_ptr(),
                                    modes.data_ptr(), modes.shape[0])

        for P in parts_dev[:3]:
            plain(P)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for P in parts_dev:
            st, _, _ = plain(P)
            if st != gridshift.GS_OK:
                raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(gp._ctx))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms = e0.elapsed_time(e1)
        sequential = {"what": f"{len(parts_dev)} sequential gs_fit calls, plain FP64 path",
                      "ms": seq_ms, "value": n / (seq_ms / 1e3) / 1e6, "unit": UNIT}
        gp.close()

    # -- end to end through the public API: every step uploads its input
    #    from pinned host memory and reads its labels and modes back.  The
    #    upload of step i + 1 and the read-back of step i run on a copy
    #    stream while step i's fit runs (double-buffered device inputs and
    #    outputs), as a stream of images would be served.  Image workloads
    #    upload the uint8 image and call the image entry point (the features
    #    are built on the device); the float64 feature upload through gs_fit
    #    is reported beside it.
    def run_e2e(h_in, call_in):
        h_labels = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
        h_modes = [torch.empty(modes.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        d_in = [torch.empty(h_in.shape, dtype=h_in.dtype, device=dev) for _ in range(2)]
        d_lab = [labels, torch.empty_like(labels)]
        d_md = [modes, torch.empty_like(modes)]
        copy = torch.cuda.Stream(dev)
        up = [torch.cuda.Event() for _ in range(2)]
        fit_done = [torch.cuda.Event() for _ in range(2)]
        down = [torch.cuda.Event() for _ in range(2)]
        steps = args.steps
        kk = 0
        call_in(d_in[0].copy_(h_in), d_lab[0], d_md[0])  # warm-up of this path
        barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(copy):
            d_in[0].copy_(h_in, non_blocking=True)
            up[0].record(copy)
        for i in range(steps):
            b = i % 2
            if i + 1 < steps:
                with torch.cuda.stream(copy):
                    # (the copy stream already waited for the fit that last
                    # read this buffer, before that fit's read-back)
                    d_in[1 - b].copy_(h_in, non_blocking=True)
                    up[1 - b].record(copy)
            stream.wait_event(up[b])
            if i >= 2:
                stream.wait_event(down[b])  # this buffer's previous read-back is done
            kk, _ = call_in(d_in[b], d_lab[b], d_md[b])
            fit_done[b].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(fit_done[b])
                h_labels[b].copy_(d_lab[b], non_blocking=True)
                h_modes[b][:kk].copy_(d_md[b][:kk], non_blocking=True)
                down[b].record(copy)
        copy.synchronize()
        stream.synchronize()
        barrier()
        secs = max_over_ranks(time.perf_counter() - t0, world, dev)
        return job_rate(n, steps, world, secs), int(h_in.numel() * h_in.element_size()), kk

    e2e_value, e2e_h2d, kk = run_e2e(torch.from_numpy(X).pin_memory(), call)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_h2d,
           "d2h_bytes_per_step": int(n * 4 + kk * d * 8),
           "input": "float64 features (n x d), gs_fit",
           "pipelined": ("the upload of step i + 1 and the read-back of step i "
                         "run on a second stream during step i's fit")}
    img = w.get("image")
    imgs = w.get("images")
    if img is not None or imgs is not None:
        if batched:
            pix = np.ascontiguousarray(np.concatenate([im.reshape(-1, im.shape[2]) for im in imgs], 0))
            h_img = torch.from_numpy(pix).pin_memory()

            def call_img(p, lab, md, gg=g):
                st, mo, infos = gridshift.gs_fit_image_batched(gg._ctx, p.data_ptr(), pix.shape[1],
                                                               offsets, lab.data_ptr(), md.data_ptr(),
                                                               md.shape[0])
                if st != gridshift.GS_OK:
                    raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(gg._ctx))
                return mo[-1], [x.as_dict() for x in infos]
            what = "uint8 images (n x 3), features built on the device, gs_fit_image_batched"
            how = e2e["pipelined"]
            v_img, h2d_img, kk = run_e2e(h_img, call_img)
        else:
            # the library's host-buffer call on a stream of `steps` images: it
            # uploads each image, fits it and reads labels and modes back,
            # the copies overlapping the fits inside the call
            h_img = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
            H, W, C = img.shape
            h_lab = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
            h_md = [torch.empty(modes.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
            cap = modes.shape[0]

            def stream_call(count):
                st, ks, _ = gridshift.gs_fit_images_host(
                    g._ctx, [h_img.data_ptr()] * count, H, W, C, w["xy_scale"],
                    [h_lab[i % 2].data_ptr() for i in range(count)],
                    [h_md[i % 2].data_ptr() for i in range(count)], cap)
                if st != gridshift.GS_OK:
                    raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(g._ctx))
                return ks

            stream_call(2)  # warm-up of this path
            barrier()
            t0 = time.perf_counter()
            ks = stream_call(args.steps)
            barrier()
            secs = max_over_ranks(time.perf_counter() - t0, world, dev)
            v_img, h2d_img, kk = job_rate(n, args.steps, world, secs), int(img.nbytes), ks[-1]
            what = (f"uint8 image ({H} x {W} x {C}) in page-locked host memory, one "
                    f"gs_fit_images_host call for the {args.steps} steps (features built on the "
                    "device; labels and modes read back into host memory)")
            how = ("inside the call: the upload of image i + 1 and the read-back of image i run "
                   "on a second stream while the neighbouring image is fitted")
        e2e = {"value": v_img, "unit": UNIT, "h2d_bytes_per_step": h2d_img,
               "d2h_bytes_per_step": int(n * 4 + kk * d * 8), "input": what,
               "pipelined": how,
               "features_path": {"value": e2e_value, "h2d_bytes_per_step": e2e_h2d,
                                 "input": e2e["input"]}}

    # -- roofline of the dominant kernel (the loop kernel: one launch per
    #    step), with the per-point launches beside it
    pk = peaks()
    roof = None
    if not batched:
        loop_ms = phase_ms["loop"] / max(phase_cnt["loop"], 1)
        cell_steps = (cell_iters + m0_total) // args.steps
        probe_steps = (cell_iters + k_total) // args.steps
        lb = loop_bytes(cell_steps, d, fp32)
        sb = loop_scope_bytes(probe_steps, d, fp32)
        # below split_min points the per-point passes run inside k_loop:
        # their bytes are k_loop's
        split = n >= g.tuning()["split_min"]
        inner = () if split else ("k_scatter", "k_sums", "labels_out")
        pp = n * sum(per_point_bytes(ph, d, elem) for ph in inner)
        lb += pp
        sb += pp
        achieved = sb / (loop_ms / 1e3) / 1e9
        tr = traffic(args.workload, args.precision, "k_loop", args.update)
        roof = {"kernel": "k_loop (update steps ii-v over the cell levels, numbering, modes)",
                "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"],
                "peak_source": f"{pk['source']} (MEASURED_PEAKS.json hbm_gbs)",
                "frac_of": pk["source"],
                "algorithmic_bytes_per_launch": sb,
                "algorithmic_count": ("scope count: per active cell and update step 3^d key "
                                      "sectors of 32 B, 2 payload sectors, centroid and key "
                                      "write, sort-and-reduce merge"
                                      + ("" if split else "; plus the per-point passes it runs "
                                         "(scatter 8 B, sums 8 + d x elem B, labels 8 B per "
                                         "point)")),
                "avg_launch_ms": loop_ms, "traffic": tr,
                "dram_count": {"bytes_per_launch": lb,
                               "achieved": lb / (loop_ms / 1e3) / 1e9,
                               "frac": lb / (loop_ms / 1e3) / 1e9 / pk["hbm_gbs"]},
                "traffic_frac": (tr / (loop_ms / 1e3) / 1e9 / pk["hbm_gbs"]) if tr else None,
                "per_point_kernels": {}}
        for ph, name in (("bin", "k_bin"),) + ((("k_scatter", "k_prep_scatter"),
                                                ("k_sums", "k_prep_sums"),
                                                ("labels_out", "k_labels_out")) if split else ()):
            ms = phase_ms[ph] / max(phase_cnt[ph], 1)
            by = n * per_point_bytes(ph, d, elem)
            roof["per_point_kernels"][name] = {
                "algorithmic_bytes_per_launch": by, "avg_launch_ms": ms,
                "achieved": by / (ms / 1e3) / 1e9 if ms > 0 else None,
                "frac": by / (ms / 1e3) / 1e9 / pk["hbm_gbs"] if ms > 0 else None,
                "traffic": traffic(args.workload, args.precision, name, args.update)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(args.warmup, 3),
                "ms_per_step": total_ms / args.steps, "median_ms_per_step": median_ms,
                "value_at_median": job_rate(n, 1, world, median_ms / 1e3),
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
                "data": "synthetic",
                "config": dict(workload_config(w, args.workload, args.precision, args.update),
                               tuning=g.tuning(), tuning_source=g.tuning_source),
                "e2e": e2e,
                "gpu_launches": int(launches),
                "roofline": roof,
                "active_cell_iterations_per_s": cell_iters * world / (total_ms / 1e3),
                "clocks": clk}
        if not batched:
            line["phases_ms_per_step"] = {p: phase_ms[p] / args.steps for p in phase_ms}
        if agreement is not None:
            line["agreement"] = agreement
        if sequential is not None:
            line["sequential"] = sequential
        if world == 1 and not args.no_cpu_baseline:
            refs = []
            line["cpu_baseline"] = cpu_baseline(w, update=args.update, results=refs)
            if last is not None and refs:
                try:
                    line["agreement"] = oracle_agreement(*last, refs[0], w["h"])
                except Exception as e:  # an informational field: never lose the line
                    line["agreement"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_track(args) -> int:
    """The tracking window step (Sec. 2.3, Algorithm 2) on a 1920x1080 RGB
    frame: R of a 600x600 search window around a moving disc, B = the disc's
    colour cells in the previous frame.  One step = one gs_track_window call
    (upload of B, the kernel, the results read back)."""
    import numpy as np
    import torch

    from paper_2206_02200_gb300 import gridshift, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H, W, h = 1080, 1920, 16.0
    frames, centres = synth.moving_object_frames(H, W, 2, seed=5, radius=150.0)
    f0 = frames[0].reshape(H * W, 3)
    yy, xx = np.divmod(np.arange(H * W), W)
    inside = (xx - centres[0, 0]) ** 2 + (yy - centres[0, 1]) ** 2 <= 150.0 ** 2
    B = np.unique(np.floor(f0[inside] / h).astype(np.int64), axis=0)
    rect = gridshift.window_rect(centres[0], 600.0, 600.0)
    npix = (min(rect[2], W) - max(rect[0], 0)) * (min(rect[3], H) - max(rect[1], 0))
    frame = torch.from_numpy(np.ascontiguousarray(frames[1].reshape(H * W, 3))).to(dev)
    g = gridshift.GridShift(3, h, 1)
    stream = torch.cuda.current_stream(dev)
    gridshift.gs_set_stream(g._ctx, stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def call():
        st, res, present = gridshift.gs_track_window(g._ctx, frame.data_ptr(), gridshift.GS_IN_F64,
                                                     W, H, B, *rect)
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(g._ctx))
        return res.as_dict()

    for _ in range(max(args.warmup, 3)):
        call()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    ev = []
    for _ in range(args.steps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = call()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    value = npix * args.steps / (total_ms / 1e3) / 1e6
    pk = peaks()
    line = {"metric": "tracking window Mpixels/s (Algorithm 2 window step)", "value": value,
            "unit": "Mpixels/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "track_window_1920x1080_d3", "window": [int(v) for v in rect],
                       "window_pixels": int(npix), "bins": int(B.shape[0]), "h": h,
                       "l2": "flushed between timed steps (256 MiB device write)",
                       "generator": "moving disc over a Voronoi background, seeded"},
            "roofline": {"kernel": "k_track", "bound": "hbm",
                         "achieved": npix * 3 * 8 / (total_ms / args.steps / 1e3) / 1e9,
                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": npix * 3 * 8 / (total_ms / args.steps / 1e3) / 1e9 / pk["hbm_gbs"],
                         "frac_of": pk["source"],
                         "note": "whole call (host upload of B, kernel, read-back) as the duration",
                         "traffic": None},
            "R": {"count": int(res["count"]), "mean": [res["mean_x"], res["mean_y"]]},
            "clocks": clk}
    if not args.no_cpu_baseline:
        import time
        from oracle import oracle
        f1 = frames[1].reshape(H * W, 3)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0 or reps == 0:
            oracle.track_window(f1, W, H, h, B, rect)
            reps += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": npix * reps / dt / 1e6, "unit": "Mpixels/s", "cores": 1,
                                "kind": "oracle", "sample": f"{reps} window steps"}
    print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_sweep(args) -> int:
    """A bandwidth sweep: one step = one gs_fit_sweep call over every h of the
    workload (the same points, B instances in one pass of the batched
    pipeline); beside it, the same B runs as B separate gs_fit calls.  Units:
    pixel-bandwidth pairs (B x n per step)."""
    import numpy as np
    import torch

    from paper_2206_02200_gb300 import gridshift

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = load_workload(args.workload)
    X, hs = w["points"], list(w["hs"])
    n, d = X.shape
    B = len(hs)
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty((B, n), dtype=torch.int32, device=dev)
    modes = torch.empty((65536, d), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    g = gridshift.GridShift(d, hs[0], w["max_iter"])
    gridshift.gs_set_stream(g._ctx, stream.cuda_stream)
    dt = gridshift.GS_IN_F64 if X.dtype == np.float64 else gridshift.GS_IN_F32

    def sweep_call(p=pts):
        st, mo, infos = gridshift.gs_fit_sweep(g._ctx, p.data_ptr(), dt, n, hs, labels.data_ptr(),
                                               modes.data_ptr(), modes.shape[0])
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(g._ctx))
        return mo, [x.as_dict() for x in infos]

    singles = []
    for h in hs:
        gg = gridshift.GridShift(d, h, w["max_iter"])
        gridshift.gs_set_stream(gg._ctx, stream.cuda_stream)
        singles.append(gg)

    def separate_calls():
        for b, gg in enumerate(singles):
            st, k, info = gridshift.gs_fit(gg._ctx, pts.data_ptr(), dt, n, labels[b].data_ptr(),
                                           modes.data_ptr(), modes.shape[0])
            if st != gridshift.GS_OK:
                raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(gg._ctx))

    for _ in range(max(args.warmup, 3)):
        sweep_call()
        separate_calls()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    ev, ev_sep = [], []
    launches = 0
    cell_iters = 0
    for _ in range(args.steps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mo, infos = sweep_call()
        b.record(stream)
        ev.append((a, b))
        launches += infos[0]["launches"]
        cell_iters += sum(x["cell_iters"] for x in infos)
        flush.fill_(2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        separate_calls()
        b.record(stream)
        ev_sep.append((a, b))
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sep_ms = [a.elapsed_time(b) for a, b in ev_sep]
    total_ms = sum(step_ms)
    value = job_rate(n * B, args.steps, 1, total_ms / 1e3)
    # end to end: the points from pinned host memory, labels and modes back
    h_pts = torch.from_numpy(X).pin_memory()
    h_labels = torch.empty((B, n), dtype=torch.int32).pin_memory()
    h_modes = torch.empty(modes.shape, dtype=torch.float64).pin_memory()
    d_pts = torch.empty_like(pts)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    kk = 0
    for _ in range(args.steps):
        d_pts.copy_(h_pts, non_blocking=True)
        mo, _ = sweep_call(d_pts)
        kk = mo[-1]
        h_labels.copy_(labels, non_blocking=True)
        h_modes[:kk].copy_(modes[:kk], non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    line = {"metric": "Mpixels/s of a bandwidth sweep (pixel-bandwidth pairs), one call vs "
                      "separate calls", "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_ms / args.steps,
            "median_ms_per_step": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.workload),
            "e2e": {"value": job_rate(n * B, args.steps, 1, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int(X.nbytes),
                    "d2h_bytes_per_step": int(B * n * 4 + kk * d * 8)},
            "gpu_launches": int(launches),
            "separate_calls": {"what": f"{B} gs_fit calls, one per h",
                               "ms_per_step": sum(sep_ms) / args.steps,
                               "value": job_rate(n * B, args.steps, 1, sum(sep_ms) / 1e3),
                               "unit": UNIT},
            "k_per_h": [x["k"] for x in infos], "iterations_per_h": [x["iterations"] for x in infos],
            "active_cell_iterations_per_s": cell_iters / (total_ms / 1e3),
            "roofline": None, "clocks": clk}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    for gg in singles:
        gg.close()
    g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="image_1080p_d5")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--update", choices=["parallel", "sequential"], default="parallel",
                    help="update form: Eq. 6 (parallel, default) or Eq. 5 (sequential; "
                         "float64, one point set per call)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", choices=["auto", "default"], default="auto",
                    help="launch choices: the autotuner's cached entry for the workload "
                         "(auto, default) or the library's built-in ones")
    ap.add_argument("--tune", action="append", default=[], metavar="KNOB=VALUE",
                    help="override one launch choice (gs_tuning field) after the above")
    args = ap.parse_args()
    if args.update == "sequential" and (args.precision != "fp64" or
                                        args.workload.startswith(("batch", "track", "sweep"))):
        ap.error("--update sequential runs in fp64 on workloads of one point set")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "track_1080p_d3":
        return run_track(args)
    if args.workload.startswith("sweep"):
        return run_sweep(args)
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
