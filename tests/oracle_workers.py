"""Oracle runs for a process pool (started with the spawn method, so that no
worker inherits a CUDA context): each worker regenerates its input from the
seeded generators and returns the oracle's result, so no large array crosses
the pipe on the way in."""
from __future__ import annotations

import multiprocessing
import os


def _result(r: dict) -> dict:
    return {k: r[k] for k in ("labels", "modes", "keys", "counts", "iterations", "converged",
                              "m0", "k")}


def batch_item(args) -> dict:
    """Oracle run of instance i of image_batch(., seed0) with cell side h."""
    i, seed0, h, max_iter = args
    from oracle import oracle
    from paper_2206_02200_gb300 import synth
    return _result(oracle.fit(synth.image_batch_item(i, seed0), h, max_iter))


def workload(name: str) -> dict:
    """Oracle run of a named single-instance workload."""
    from oracle import oracle
    from paper_2206_02200_gb300 import synth
    w = synth.WORKLOADS[name]()
    return _result(oracle.fit(w["points"], w["h"], w["max_iter"]))


def pool(procs: int | None = None):
    """A spawn-method pool over the host's cores (the oracle is built first,
    so the workers only load it)."""
    from oracle import oracle
    oracle.build()
    n = procs or max(1, min(16, os.cpu_count() or 1))
    return multiprocessing.get_context("spawn").Pool(n)
