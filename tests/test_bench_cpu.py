"""bench.py's CPU-side contract: the reference arm (the oracle) on both update
forms, the argument checks, and the traffic lookup."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_sequential_line():
    r = _bench("--impl", "reference", "--workload", "image_321x481_d3", "--steps", "1",
               "--warmup", "0", "--update", "sequential")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["update"] == "sequential"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_sequential_needs_fp64_and_one_point_set():
    for extra in (["--precision", "fp32"], ["--workload", "batch_64_d3"]):
        r = _bench("--update", "sequential", *extra)
        assert r.returncode == 2 and "sequential" in r.stderr


def test_traffic_only_for_captured_parallel_kernels():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.traffic("image_1080p_d5", "fp64", "k_loop", "sequential") is None
    assert bench.traffic("no_such_workload", "fp64", "k_loop") is None


def test_scope_count_of_the_loop_kernel():
    # 1080p d=5 FP64: 3^5 key sectors, 2 payload sectors, the centroid and key
    # written (48 B) and the merge (48 B of sort passes, 2 x 44 B of payload)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.scope_bytes_per_cell_step(5, False) == 243 * 32 + 64 + 48 + 48 + 88
    assert bench.scope_bytes_per_cell_step(6, True) == 729 * 32 + 64 + 32 + 48 + 56
    assert bench.loop_scope_bytes(0, 3, False) == 0
    assert bench.loop_scope_bytes(7, 3, True) == 7 * bench.scope_bytes_per_cell_step(3, True)
    # DRAM counts: the loop kernel's rows and keys; the per-point launches
    assert bench.loop_bytes(10, 5, False) == 10 * (2 * 96 + 8)
    assert bench.per_point_bytes("k_sums", 5, 8) == 48
    assert bench.per_point_bytes("bin", 3, 4) == 16


def test_reference_arm_uses_every_core():
    r = _bench("--impl", "reference", "--workload", "image_321x481_d3", "--steps", "1",
               "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["cpu_baseline"]["cores"] == line["cpu_baseline"]["nproc"] >= 1


def test_oracle_agreement_of_the_fp64_line():
    # the FP64 line's comparison with the oracle: identical results read as
    # identical; one label, one mode bit or the cluster count off is reported
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from oracle import oracle
    from paper_2206_02200_gb300 import synth
    X = synth.image_features(synth.voronoi_image(40, 56, 5, 8.0, seed=3), xy_scale=0.1)
    ref = oracle.fit(X, 12.0, 50)
    k = int(ref["k"])
    same = bench.oracle_agreement(ref["labels"].copy(), ref["modes"][:k].copy(), k,
                                  ref["iterations"], ref, 12.0)
    assert same["labels_identical"] and same["modes_bit_identical"] and same["labels"] == 1.0
    assert same["k"] == same["k_ref"] == k and same["max_mode_error_h"] == 0.0
    lab = ref["labels"].copy()
    lab[7] = (lab[7] + 1) % k
    md = ref["modes"][:k].copy()
    md[0, 0] = np.nextafter(md[0, 0], np.inf)
    off = bench.oracle_agreement(lab, md, k, ref["iterations"], ref, 12.0)
    assert not off["labels_identical"] and off["labels"] == 1.0 - 1.0 / len(lab)
    assert not off["modes_bit_identical"] and 0.0 < off["max_mode_error_h"] < 1e-12
    fewer = bench.oracle_agreement(lab, md[:k - 1], k - 1, ref["iterations"], ref, 12.0)
    assert fewer["k"] == k - 1 and fewer["max_mode_error_h"] is None
