"""The float32 mixed-precision variant (GS_FP32_MIXED) against the float64
oracle.  The bar: clusters matched one to one (greedily by overlap, each
cluster of either side used once) cover at least 99.9% of the points, the
cluster counts agree, and the modes of every matched pair lie within
1e-3 * h of the oracle's (the float32 path is not bit-exact: its sums
are rounded float32 and merges add in any order)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import agreement, gridshift, synth
from tests import golden_io

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AGREE = 0.999
MODE_TOL = 1e-3  # in units of h


def _fit32(X, h, max_iter=50, as_f32=False):
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if as_f32:
        pts = pts.float()
    with gridshift.GridShift(X.shape[1], h, max_iter, precision=gridshift.GS_FP32_MIXED) as g:
        labels, modes, info = g.fit(pts)
        torch.cuda.synchronize()
    return labels.cpu().numpy(), modes.cpu().numpy(), info


def check32(X, h, max_iter=50, as_f32=False, k_slack=0):
    """The float32 path against the oracle: one-to-one label agreement of at
    least AGREE, the same number of clusters (up to k_slack), and every
    matched pair of modes within MODE_TOL * h."""
    Xo = X.astype(np.float32).astype(np.float64) if as_f32 else X
    ref = oracle.fit(Xo, h, max_iter)
    lab, md, info = _fit32(X, h, max_iter, as_f32)
    ag = agreement.agreement(lab, ref["labels"], md, ref["modes"], h)
    assert ag["labels"] >= AGREE, ag
    assert abs(info["k"] - ref["k"]) <= k_slack, (info["k"], ref["k"])
    assert ag["max_mode_error_h"] <= MODE_TOL, ag
    return ag["labels"], ag["max_mode_error_h"], info, ref


@pytest.mark.parametrize("case", golden_io.all_cases(), ids=lambda c: c["name"])
def test_golden_cases_fp32(case):
    X = case["points"]
    lab, md, info = _fit32(X, case["h"], case.get("max_iter", 50))
    assert list(lab) == case["labels"]
    for r, row in enumerate(case["modes"]):
        for a, v in enumerate(row):
            assert abs(md[r, a] - float(v)) <= 1e-6 * case["h"]


@pytest.mark.parametrize("d", [1, 2, 3, 5, 6, 8])
def test_random_blobs_fp32(d):
    rng = np.random.default_rng(500 + d)
    centres = rng.uniform(-40, 40, size=(5, d))
    X = centres[rng.integers(0, 5, 20000)] + rng.normal(0, 3.0, size=(20000, d))
    check32(X, 4.0)


def test_pencil_first_step_fp32():
    # enough level-0 cells (>= 4096) for the two-pass form of the first
    # update, on inputs that converge to few clusters (with thousands of
    # small clusters one float32 near-tie moves a cell and a mode with it)
    X = synth.image_features(synth.voronoi_image(480, 640, 20, 4.0, seed=9))
    _, _, _, ref = check32(X, 4.0)
    assert ref["m0"] >= 4096
    rng = np.random.default_rng(84)
    X = rng.uniform(0.0, 4.0, size=(15_000, 7))
    X[: 15_000 // 4] = rng.normal(3.0, 0.7, size=(15_000 // 4, 7))
    _, _, _, ref = check32(X, 1.0, max_iter=8)
    assert ref["m0"] >= 4096


def test_images_fp32():
    for (H, W, R, seed, xy) in [(120, 160, 9, 4, None), (250, 333, 15, 3, 0.1)]:
        img = synth.voronoi_image(H, W, R, 10.0, seed=seed, gradient=0.02)
        check32(synth.image_features(img, xy_scale=xy), 10.0 if xy else 16.0)


def test_gmm_float32_input_fp32():
    X = synth.gmm_points(300_000, 6, 40, seed=9)
    check32(X, 4.0, as_f32=True)


def test_max_iter_fp32():
    X = synth.image_features(synth.voronoi_image(120, 160, 9, 8.0, seed=4))
    for mi in (0, 1, 2):
        agree, err, info, ref = check32(X, 16.0, mi)
        assert info["iterations"] <= mi


def test_image_1080p_d5_fp32():
    w = synth.WORKLOADS["image_1080p_d5"]()
    agree, err, info, ref = check32(w["points"], w["h"], w["max_iter"])
    print(f"1080p fp32: label agreement {agree:.6f}, max mode error {err:.2e} h, "
          f"face rechecks {info['face_rechecks']}")


def test_batched_fp32():
    parts = synth.image_batch(5, 300, hmin=40, hmax=120, wmin=50, wmax=160)
    offsets = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).tolist()
    X = np.concatenate(parts, 0)
    with gridshift.GridShift(3, 16.0, 50, precision=gridshift.GS_FP32_MIXED) as g:
        labels, modes, infos = g.fit_batched(torch.from_numpy(X).cuda(), offsets)
        torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    for b, p in enumerate(parts):
        ref = oracle.fit(p, 16.0, 50)
        md = modes[b].cpu().numpy()
        ag = agreement.agreement(lab[offsets[b]:offsets[b + 1]], ref["labels"], md,
                                 ref["modes"], 16.0)
        assert ag["labels"] >= AGREE and ag["max_mode_error_h"] <= MODE_TOL, ag
        assert infos[b]["k"] == ref["k"] == len(md)


def test_switching_precision_on_one_context():
    X = synth.image_features(synth.voronoi_image(100, 140, 7, 8.0, seed=6))
    ref = oracle.fit(X, 16.0, 50)
    pts = torch.from_numpy(X).cuda()
    with gridshift.GridShift(3, 16.0, 50) as g:
        for prec in (gridshift.GS_FP64, gridshift.GS_FP32_MIXED, gridshift.GS_FP64):
            assert gridshift.gs_set_precision(g._ctx, prec) == gridshift.GS_OK
            labels, modes, info = g.fit(pts)
            torch.cuda.synchronize()
            if prec == gridshift.GS_FP64:
                np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
            else:
                ag = agreement.agreement(labels.cpu().numpy(), ref["labels"])
                assert ag["labels"] >= AGREE and info["k"] == ref["k"], ag
