"""Launch choices (gs_tuning) change which lanes, tables and phases compute a
run, never its result: under every extreme choice the FP64 path must still
equal the oracle bit for bit (exact sums, Sec. 2.1, Eq. 1-4)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CHOICES = [
    {"few_lanes_x4": 0},            # few lanes per cell at every level
    {"few_lanes_x4": 1 << 20},      # 32 lanes per cell at every level
    {"load_shift": 1},              # tables at load up to 1/2
    {"filter": 0},                  # every probe reads the table
    {"tail_enter": 0},              # no one-block tail
    {"tail_enter": 256},            # the largest tail
    {"pencil_min": 0},              # pencil form whenever the tail is not entered at once
    {"pencil_min": 1 << 30},        # no pencil form
    {"bin_list": 0},                # binning: one add per new cell
    {"split_min": 0},               # per-point passes as launches of their own
    {"split_min": (1 << 31) - 1},   # per-point passes inside the loop kernel
    {"few_lanes_x4": 1, "load_shift": 1, "filter": 0, "tail_enter": 32, "pencil_min": 1024,
     "split_min": 0},
]


def _check(X, h, tuning, max_iter=50):
    ref = oracle.fit(X, h, max_iter)
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    with gridshift.GridShift(X.shape[1], h, max_iter, tuning=tuning) as g:
        assert g.tuning() == dict(gridshift.DEFAULT_TUNING, **tuning)
        labels, modes, info = g.fit(pts)
        torch.cuda.synchronize()
    assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64), ref["modes"].view(np.int64))


@pytest.fixture(scope="module")
def image():
    return synth.image_features(synth.voronoi_image(240, 320, 14, 8.0, seed=21), xy_scale=0.1)


@pytest.mark.parametrize("tuning", CHOICES, ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_image_d5_under_every_choice(image, tuning):
    _check(image, 12.0, tuning)


@pytest.mark.parametrize("tuning", CHOICES[:4] + CHOICES[6:11],
                         ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_gmm_d6_under_choices(tuning):
    X = synth.gmm_points(60_000, 6, 20, seed=8).astype(np.float64)
    _check(X, 4.0, tuning)


@pytest.mark.parametrize("tuning", CHOICES[:4] + CHOICES[8:11],
                         ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_batched_under_choices(tuning):
    parts = synth.image_batch(4, 77, hmin=40, hmax=90, wmin=50, wmax=120)
    offsets = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).tolist()
    X = np.concatenate(parts, 0)
    with gridshift.GridShift(3, 16.0, 50, tuning=tuning) as g:
        labels, modes, infos = g.fit_batched(torch.from_numpy(X).cuda(), offsets)
        torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    for b, p in enumerate(parts):
        ref = oracle.fit(p, 16.0, 50)
        np.testing.assert_array_equal(lab[offsets[b]:offsets[b + 1]], ref["labels"])
        np.testing.assert_array_equal(modes[b].cpu().numpy().view(np.int64),
                                      ref["modes"].view(np.int64))


def test_auto_tuning_reads_the_cache():
    X = synth.image_features(synth.voronoi_image(120, 160, 9, 8.0, seed=4))
    with gridshift.GridShift(3, 16.0, 50, tuning="auto") as g:
        labels, modes, info = g.fit(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
        assert g.tuning_source
    ref = oracle.fit(X, 16.0, 50)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
