"""Autotuner of the loop kernel's launch choices (gs_tuning).

The choices decide which lanes, tables and phases compute a GridShift run,
never its result: lanes per cell in the neighbour gather (few lanes, several
cells in flight per warp, or 32 lanes per cell, by level size), the load of
the level hash tables, whether probes pass the occupancy filter, the level
size below which one block finishes the run, the least cell count for the
pencil form of the first update, the least point count for running the
per-point passes as launches of their own, and how binning lists new cells.

``tune_workload`` measures them on one workload by coordinate descent from
the built-in choices (each knob swept over its candidates with the others
fixed, twice over), each setting timed as the median of several complete
runs with the L2 cache flushed between them, and keeps a change only when it
is faster by more than ``MIN_GAIN``.  Results are checked to be bit for bit
those of the built-in choices (FP64).  ``main`` writes the measurements to a
JSON cache (``tuning.json`` beside this file); ``GridShift(..., tuning="auto")``
reads the entry for its dimension, precision and size from it (``lookup``).

    python -m paper_2206_02200_gb300.autotune --workloads image_1080p_d5 gmm_10M_d6
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

from . import gridshift

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")

#: candidate values of every knob (the built-in choice is among them)
CANDIDATES = {
    "few_lanes_x4": [1, 2, 4, 8, 16, 64],
    "load_shift": [2, 1],
    "filter": [1, 0],
    "tail_enter": [0, 32, 64, 128, 192, 256],
    "pencil_min": [1024, 4096, 16384, 1 << 30],
    "split_min": [1 << 22, 0, (1 << 31) - 1],
    "bin_list": [1, 0],
    "bin_sums": [0, 1],
}
#: knobs that batched runs use (the tail and the pencil form are plain-run only)
BATCHED_KNOBS = ("few_lanes_x4", "load_shift", "filter", "split_min", "bin_list", "bin_sums")
MIN_GAIN = 0.01

_cache = None


def key_for(d: int, precision: int, n: int, batched: bool) -> str:
    """Cache key: dimension, precision, one point set or a batch, and the
    point count's power of two."""
    prec = "fp32" if precision == gridshift.GS_FP32_MIXED else "fp64"
    kind = "batch" if batched else "one"
    return f"d{d}_{prec}_{kind}_n2^{max(0, round(math.log2(max(n, 1))))}"


def load_cache(path: str = CACHE) -> dict:
    global _cache
    if _cache is None or path != CACHE:
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
        if path != CACHE:
            return data
        _cache = data
    return _cache


def lookup(d: int, precision: int, n: int, batched: bool = False, path: str = CACHE):
    """The cached entry for a call ({"key", "tuning", ...}): the same
    dimension, precision and kind, the nearest point-count bucket within a
    factor of four; None if there is none."""
    cache = load_cache(path)
    want = key_for(d, precision, n, batched)
    if want in cache:
        return dict(cache[want], key=want)
    prefix, bucket = want.rsplit("_n2^", 1)
    best = None
    for k, v in cache.items():
        p, b = k.rsplit("_n2^", 1)
        if p != prefix:
            continue
        dist = abs(int(b) - int(bucket))
        if dist <= 2 and (best is None or dist < best[0]):
            best = (dist, k, v)
    return dict(best[2], key=best[1]) if best else None


class _Runner:
    """Complete runs of one workload on one context, timed on the device."""

    def __init__(self, w: dict, precision: int, device):
        import numpy as np
        import torch
        self.torch = torch
        self.batched = "parts" in w
        if self.batched:
            X = np.ascontiguousarray(np.concatenate(w["parts"], 0))
            self.offsets = np.concatenate([[0], np.cumsum([len(p) for p in w["parts"]])]).tolist()
        else:
            X = w["points"]
        self.n, self.d = X.shape
        self.dev = device
        self.pts = torch.from_numpy(X).to(device)
        self.labels = torch.empty(self.n, dtype=torch.int32, device=device)
        self.modes = torch.empty((max(self.n // 16, 4096), self.d), dtype=torch.float64,
                                 device=device)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        self.g = gridshift.GridShift(self.d, w["h"], w["max_iter"], precision=precision)
        self.stream = torch.cuda.current_stream(device)
        gridshift.gs_set_stream(self.g._ctx, self.stream.cuda_stream)
        self.dt = gridshift.GS_IN_F64 if X.dtype == np.float64 else gridshift.GS_IN_F32

    def call(self):
        if self.batched:
            st, mo, _ = gridshift.gs_fit_batched(self.g._ctx, self.pts.data_ptr(), self.dt,
                                                 self.offsets, self.labels.data_ptr(),
                                                 self.modes.data_ptr(), self.modes.shape[0])
            k = mo[-1]
        else:
            st, k, _ = gridshift.gs_fit(self.g._ctx, self.pts.data_ptr(), self.dt, self.n,
                                        self.labels.data_ptr(), self.modes.data_ptr(),
                                        self.modes.shape[0])
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(self.g._ctx))
        self.k = k

    def time(self, tuning: dict, reps: int) -> float:
        """Median device time (ms) of `reps` runs with these choices."""
        torch = self.torch
        st = gridshift.gs_set_tuning(self.g._ctx, tuning)
        if st != gridshift.GS_OK:
            raise gridshift.GridShiftError(st, gridshift.gs_get_last_error(self.g._ctx))
        self.call()
        ts = []
        for i in range(reps):
            self.flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            self.call()
            b.record(self.stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def result(self):
        """Labels and modes of the last run (host copies)."""
        self.torch.cuda.synchronize(self.dev)
        return self.labels.cpu().numpy().copy(), self.modes[:self.k].cpu().numpy().copy()


def tune_workload(name: str, precision: int = gridshift.GS_FP64, reps: int = 7, rounds: int = 2,
                  device=None, log=None) -> dict:
    """Coordinate descent over CANDIDATES on one workload of synth.WORKLOADS;
    returns its cache entry (key, tuning, median_ms, default_ms, ...)."""
    import numpy as np
    import torch

    from . import synth
    dev = device or torch.device("cuda", 0)
    w = synth.WORKLOADS[name]()
    r = _Runner(w, precision, dev)
    knobs = BATCHED_KNOBS if r.batched else tuple(CANDIDATES)
    best = dict(gridshift.DEFAULT_TUNING)
    t_default = r.time(best, reps)
    ref_lab, ref_modes = r.result()
    t_best = t_default
    evals = 1
    for _ in range(rounds):
        changed = False
        for knob in knobs:
            for v in CANDIDATES[knob]:
                if v == best[knob]:
                    continue
                trial = dict(best, **{knob: v})
                t = r.time(trial, reps)
                evals += 1
                if precision == gridshift.GS_FP64:
                    lab, md = r.result()
                    if not (np.array_equal(lab, ref_lab) and
                            np.array_equal(md.view(np.int64), ref_modes.view(np.int64))):
                        raise RuntimeError(f"{name}: results changed under {trial}")
                if log:
                    log(f"{name} {trial} {t:.4f} ms (best {t_best:.4f})")
                if t < t_best * (1.0 - MIN_GAIN):
                    best, t_best, changed = trial, t, True
        if not changed:
            break
    # the winner timed again beside the built-in choices, interleaved
    t_def2, t_best2 = [], []
    for _ in range(3):
        t_def2.append(r.time(dict(gridshift.DEFAULT_TUNING), reps))
        t_best2.append(r.time(best, reps))
    r.g.close()
    return {"key": key_for(r.d, precision, r.n, r.batched), "workload": w["name"],
            "tuning": best, "median_ms": statistics.median(t_best2),
            "default_ms": statistics.median(t_def2), "evaluations": evals, "reps": reps,
            "gpu": torch.cuda.get_device_name(dev),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workloads", nargs="+", default=["image_321x481_d3", "image_1080p_d5",
                                                       "image_4k_d5", "batch_64_d3",
                                                       "gmm_10M_d6"])
    ap.add_argument("--precisions", nargs="+", choices=["fp64", "fp32"],
                    default=["fp64", "fp32"])
    ap.add_argument("--reps", type=int, default=7)
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--quiet", action="store_true")
    args = ap.parse_args(argv)
    cache = load_cache(args.out)
    for name in args.workloads:
        for p in args.precisions:
            prec = gridshift.GS_FP32_MIXED if p == "fp32" else gridshift.GS_FP64
            e = tune_workload(name, prec, args.reps, log=None if args.quiet else print)
            key = e.pop("key")
            cache[key] = e
            print(json.dumps({key: e}), flush=True)
            with open(args.out, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
