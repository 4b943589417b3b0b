"""The bandwidth sweep (gs_fit_sweep): B values of h over the same points in
one call, every instance bit-identical to the oracle run with that h
(Sec. 2.1, Eq. 1-4; the bandwidth study of Sec. 4.1 runs the method over a
range of h on the same data)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _sweep(X, hs, max_iter=50, f32=False):
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if f32:
        pts = pts.float()
    with gridshift.GridShift(X.shape[1], 1.0, max_iter) as g:
        labels, modes, infos = g.fit_sweep(pts, hs)
        torch.cuda.synchronize()
    return labels.cpu().numpy(), [m.cpu().numpy() for m in modes], infos


def _check(X, hs, max_iter=50, f32=False):
    lab, modes, infos = _sweep(X, hs, max_iter, f32)
    assert lab.shape == (len(hs), X.shape[0])
    Xo = X.astype(np.float32).astype(np.float64) if f32 else X
    for b, h in enumerate(hs):
        ref = oracle.fit(Xo, h, max_iter)
        assert infos[b]["k"] == ref["k"] and infos[b]["iterations"] == ref["iterations"], (b, h)
        assert infos[b]["m0"] == ref["m0"] and infos[b]["converged"] == int(ref["converged"])
        assert infos[b]["inexact"] == 0
        np.testing.assert_array_equal(lab[b], ref["labels"])
        np.testing.assert_array_equal(modes[b].view(np.int64), ref["modes"].view(np.int64))
    return infos


def test_sweep_bsds_sized_image():
    # a 321 x 481 RGB image over eight bandwidths from 8 to 32
    X = synth.image_features(synth.voronoi_image(321, 481, 12, 8.0, seed=1))
    _check(X, [8.0, 10.0, 12.0, 14.0, 16.0, 20.0, 24.0, 32.0])


def test_sweep_rgbxy_and_non_dyadic_bandwidths():
    X = synth.image_features(synth.voronoi_image(120, 160, 9, 10.0, seed=4, gradient=0.02),
                             xy_scale=0.1)
    _check(X, [7.3, 9.9, 12.0, 3.1415926])


def test_sweep_repeated_and_unsorted_bandwidths():
    X = synth.image_features(synth.voronoi_image(60, 80, 5, 6.0, seed=12))
    lab, modes, infos = _sweep(X, [16.0, 4.0, 16.0])
    np.testing.assert_array_equal(lab[0], lab[2])
    np.testing.assert_array_equal(modes[0].view(np.int64), modes[2].view(np.int64))
    _check(X, [16.0, 4.0, 16.0])


@pytest.mark.parametrize("d", [1, 2, 4, 6])
def test_sweep_blobs_in_several_dimensions(d):
    rng = np.random.default_rng(70 + d)
    centres = rng.uniform(-30, 30, size=(4, d))
    X = centres[rng.integers(0, 4, 3000)] + rng.normal(0, 2.5, size=(3000, d))
    _check(X, [2.0, 3.0, 5.0], max_iter=20)


def test_sweep_float32_input_and_step_limits():
    X = synth.gmm_points(20_000, 3, 12, seed=3)
    _check(X.astype(np.float64), [1.0, 2.0, 4.0], max_iter=2, f32=False)
    _check(X, [1.5, 3.0], max_iter=50, f32=True)


def test_sweep_of_one_bandwidth_is_the_plain_fit():
    X = synth.image_features(synth.voronoi_image(50, 70, 4, 8.0, seed=2))
    _check(X, [16.0])


def test_sweep_refuses_float32_state():
    X = synth.image_features(synth.voronoi_image(20, 30, 3, 8.0, seed=2))
    pts = torch.from_numpy(X).cuda()
    with gridshift.GridShift(3, 1.0, 10, precision=gridshift.GS_FP32_MIXED) as g:
        with pytest.raises(gridshift.GridShiftError):
            g.fit_sweep(pts, [8.0, 16.0])
