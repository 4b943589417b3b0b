"""The sequential update (Sec. 2.2, Eq. 5; GS_UPDATE_SEQUENTIAL) through the
C ABI against the oracle's sequential form.

Both sides sweep the cells in ascending parity colour and form every sum
exactly, rounded once; an updated neighbour contributes its count times its
new centroid, exactly.  So the expected result is bit-identical: labels,
iteration count and float64 modes.  The hand-worked cases, tiny random
inputs with many points on cell faces, images (d = 3 and 5) and the step
limit are covered; every d from 1 to 8 runs at least once.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth
from tests import golden_io

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fit_seq(X, h, max_iter=50):
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    with gridshift.GridShift(X.shape[1], h, max_iter,
                             update=gridshift.GS_UPDATE_SEQUENTIAL) as g:
        labels, modes, info = g.fit(pts)
        torch.cuda.synchronize()
    return labels.cpu().numpy(), modes.cpu().numpy(), info


def check_seq(X, h, max_iter=50):
    ref = oracle.fit(X, h, max_iter, update="sequential")
    lab, md, info = _fit_seq(X, h, max_iter)
    assert info["k"] == ref["k"]
    assert info["m0"] == ref["m0"]
    assert info["iterations"] == ref["iterations"]
    assert bool(info["converged"]) == ref["converged"]
    assert info["inexact"] == 0
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(md.view(np.int64), ref["modes"].view(np.int64))
    return ref, info


@pytest.mark.parametrize("case", golden_io.sequential_cases(), ids=lambda c: c["name"])
def test_sequential_golden_cases_on_gpu(case):
    ref, _ = check_seq(case["points"], case["h"], case["max_iter"])
    assert ref["labels"].tolist() == case["labels"]
    assert ref["iterations"] == case["iterations"]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_sequential_random(d):
    rng = np.random.default_rng(700 + d)
    n = 3000 if d <= 5 else 1500
    C = rng.uniform(-6, 6, size=(4, d))
    X = C[rng.integers(0, 4, n)] + rng.normal(0, 1.2, size=(n, d))
    X[: n // 3] = np.round(X[: n // 3] * 4) / 4  # points on cell faces
    check_seq(X, 1.0 if d <= 4 else 2.0)


def test_sequential_differs_from_parallel():
    # E1's points: the parallel form merges keys 0 and 1 in its first update,
    # the sequential one only in its second
    X = np.array([[0.25], [0.75], [1.5], [4.25], [4.75], [7.5]])
    ref, info = check_seq(X, 1.0)
    assert info["iterations"] == 2
    par = oracle.fit(X, 1.0, 50)
    assert par["iterations"] == 1


def test_sequential_images():
    img = synth.voronoi_image(120, 160, 9, 8.0, seed=4)
    check_seq(synth.image_features(img), 16.0)
    img = synth.voronoi_image(96, 128, 7, 10.0, seed=5, gradient=0.02)
    check_seq(synth.image_features(img, xy_scale=0.1), 12.0)


def test_sequential_image_several_cells_per_group():
    # 7302 initial cells: more than the kernel's 2432 cell groups (152 blocks
    # of 512 threads, 32 lanes a cell), so groups take several cells per pass
    img = synth.voronoi_image(480, 640, 20, 10.0, seed=11)
    ref, info = check_seq(synth.image_features(img, xy_scale=0.1), 12.0)
    assert ref["m0"] > 2432


def test_sequential_max_iter():
    X = synth.image_features(synth.voronoi_image(60, 80, 5, 8.0, seed=6))
    for mi in (0, 1, 2, 3):
        ref, info = check_seq(X, 16.0, mi)
        assert info["iterations"] <= mi


def test_parallel_form_unchanged_on_the_same_context():
    # switching the form back gives the parallel result again
    X = synth.image_features(synth.voronoi_image(60, 80, 5, 8.0, seed=7))
    ref_p = oracle.fit(X, 16.0, 50)
    ref_s = oracle.fit(X, 16.0, 50, update="sequential")
    pts = torch.from_numpy(X).cuda()
    with gridshift.GridShift(3, 16.0, 50) as g:
        for form, ref in ((gridshift.GS_UPDATE_PARALLEL, ref_p),
                          (gridshift.GS_UPDATE_SEQUENTIAL, ref_s),
                          (gridshift.GS_UPDATE_PARALLEL, ref_p)):
            assert gridshift.gs_set_update(g._ctx, form) == gridshift.GS_OK
            labels, modes, info = g.fit(pts)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
            np.testing.assert_array_equal(modes.cpu().numpy(), ref["modes"])
