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
    {"bin_sums": 1},                          # exact sums in binning, in the loop kernel
    {"bin_sums": 1, "split_min": 0},          # ... labels as a launch of their own
    {"bin_sums": 1, "bin_list": 0},           # ... one add per new cell
    {"bin_sums": 0, "split_min": 0},          # counting sort and sums as launches of their own
]
SUM_CHOICES = CHOICES[12:]


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


@pytest.mark.parametrize("tuning", CHOICES[:4] + CHOICES[6:11] + SUM_CHOICES,
                         ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_gmm_d6_under_choices(tuning):
    X = synth.gmm_points(60_000, 6, 20, seed=8).astype(np.float64)
    _check(X, 4.0, tuning)


@pytest.mark.parametrize("tuning", CHOICES[:4] + CHOICES[8:11] + SUM_CHOICES,
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


@pytest.mark.parametrize("tuning", SUM_CHOICES, ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_sequential_under_sum_choices(image, tuning):
    # the sequential update (Eq. 5) starts from the same binning and cell sums
    ref = oracle.fit(image, 12.0, 50, update="sequential")
    with gridshift.GridShift(5, 12.0, 50, update=gridshift.GS_UPDATE_SEQUENTIAL,
                             tuning=tuning) as g:
        labels, modes, info = g.fit(torch.from_numpy(image).cuda())
        torch.cuda.synchronize()
    assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64), ref["modes"].view(np.int64))


@pytest.mark.parametrize("as_f32", [False, True], ids=["f64_input", "f32_input"])
@pytest.mark.parametrize("tuning", SUM_CHOICES, ids=lambda t: ",".join(f"{k}={v}" for k, v in t.items()))
def test_fp32_under_sum_choices(image, tuning, as_f32):
    # the float32 variant takes its initial cell means from either form of
    # the sums: the same bar as its other tests (one-to-one agreement, equal
    # cluster counts, modes within 1e-3 h of the oracle's)
    from paper_2206_02200_gb300 import agreement
    X = image.astype(np.float32).astype(np.float64) if as_f32 else image
    ref = oracle.fit(X, 12.0, 50)
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if as_f32:
        pts = pts.float()
    with gridshift.GridShift(5, 12.0, 50, precision=gridshift.GS_FP32_MIXED, tuning=tuning) as g:
        labels, modes, info = g.fit(pts)
        torch.cuda.synchronize()
    ag = agreement.agreement(labels.cpu().numpy(), ref["labels"], modes.cpu().numpy(),
                             ref["modes"], 12.0)
    assert ag["labels"] >= 0.999, ag
    assert info["k"] == ref["k"]
    assert ag["max_mode_error_h"] <= 1e-3, ag
