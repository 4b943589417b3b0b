"""gs_fit_batched: B independent point sets in one call.  Each instance's
labels (numbered from 0 within the instance), modes, iteration count,
convergence flag and counts must equal the oracle run on that instance alone,
bit for bit, as for gs_fit."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _check_batch(parts, h, max_iter=50, as_f32=False):
    X = np.concatenate([p for p in parts if len(p)], 0) if any(len(p) for p in parts) else \
        np.zeros((0, parts[0].shape[1]))
    offsets = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).tolist()
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if as_f32:
        pts = pts.float()
    with gridshift.GridShift(X.shape[1], h, max_iter) as g:
        labels, modes, infos = g.fit_batched(pts, offsets)
        torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    for b, p in enumerate(parts):
        Xo = p.astype(np.float32).astype(np.float64) if as_f32 else p
        ref = oracle.fit(Xo, h, max_iter) if len(p) else None
        info = infos[b]
        if ref is None:
            assert info["k"] == 0 and info["m0"] == 0 and modes[b].shape[0] == 0
            continue
        assert info["k"] == ref["k"] and info["m0"] == ref["m0"], b
        assert info["iterations"] == ref["iterations"], b
        assert bool(info["converged"]) == ref["converged"], b
        np.testing.assert_array_equal(lab[offsets[b]:offsets[b + 1]], ref["labels"])
        np.testing.assert_array_equal(modes[b].cpu().numpy().view(np.int64),
                                      ref["modes"].view(np.int64))
    return infos


def test_batch_of_uneven_images():
    rng = np.random.default_rng(8)
    parts = []
    for i in range(7):
        H, W = int(rng.integers(20, 90)), int(rng.integers(20, 120))
        img = synth.voronoi_image(H, W, int(rng.integers(3, 12)), 8.0, seed=100 + i)
        parts.append(synth.image_features(img))
    infos = _check_batch(parts, 16.0)
    # the instances stop after different numbers of updates
    assert len({i["iterations"] for i in infos}) > 1


def test_batch_d5_with_empty_and_single_point_instances():
    rng = np.random.default_rng(9)
    img = synth.voronoi_image(60, 80, 6, 10.0, seed=3, gradient=0.02)
    big = synth.image_features(img, xy_scale=0.1)
    parts = [big[:1000], np.zeros((0, 5)), big[1000:1001], big[1001:], np.zeros((0, 5))]
    _check_batch(parts, 12.0)


def test_batch_max_iter_cap_and_float32():
    parts = [synth.gmm_points(3000 + 500 * i, 3, 6, seed=20 + i) for i in range(5)]
    for mi in (0, 1, 2):
        _check_batch(parts, 4.0, max_iter=mi)
    _check_batch([p.astype(np.float32) for p in parts], 4.0, as_f32=True)


def test_batch_many_instances_and_sort_numbering():
    # 40 instances of 600 isolated lattice points: 24000 clusters in total,
    # numbered by the radix-sort path
    i, j = np.meshgrid(np.arange(20), np.arange(30), indexing="ij")
    base = np.stack([4.0 * i.ravel() + 0.5, 4.0 * j.ravel() + 0.5], 1)
    parts = [base + np.array([0.25 * (b % 3), 0.0]) for b in range(40)]
    infos = _check_batch(parts, 1.0)
    assert sum(i["k"] for i in infos) == 24000


def test_batched_single_instance_equals_gs_fit():
    X = synth.image_features(synth.voronoi_image(50, 70, 5, 8.0, seed=4))
    _check_batch([X], 16.0)
