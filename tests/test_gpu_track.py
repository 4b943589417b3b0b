"""GPU tracking window step (Sec. 2.3, Algorithm 2) against the oracle: the
window step's results are exact integers and one IEEE division, so they must
match bit for bit."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cells(frame, h):
    return np.array([[oracle.floor_div(v, h) for v in c] for c in frame], dtype=np.int64)


def _gpu_window(frame, W, H, h, bins, rect, as_f32=False):
    d = frame.shape[1]
    t = torch.from_numpy(np.ascontiguousarray(frame)).cuda()
    if as_f32:
        t = t.float()
    with gridshift.GridShift(d, h, 1) as g:
        st, res, present = gridshift.gs_track_window(
            g._ctx, t.data_ptr(), gridshift.GS_IN_F32 if as_f32 else gridshift.GS_IN_F64, W, H,
            bins, *rect)
        msg = gridshift.gs_get_last_error(g._ctx)
    return st, res.as_dict(), present, msg


def _same(r, ref):
    for key in ("count", "sum_x", "sum_y", "min_x", "max_x", "min_y", "max_y"):
        assert r[key] == ref[key], key
    for key in ("mean_x", "mean_y"):
        if ref["count"]:
            assert np.float64(r[key]).view(np.int64) == np.float64(ref[key]).view(np.int64), key
        else:
            assert math.isnan(r[key])


@pytest.mark.parametrize("as_f32", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_window_step_matches_oracle(seed, as_f32):
    rng = np.random.default_rng(200 + seed)
    W, H, d = int(rng.integers(40, 300)), int(rng.integers(30, 200)), int(rng.integers(1, 5))
    h = float(rng.uniform(4, 20))
    frame = np.rint(rng.uniform(0, 255, size=(W * H, d)))
    frame[rng.random(W * H) < 0.2] += 0.5
    if as_f32:
        frame = frame.astype(np.float32).astype(np.float64)
    cells = _cells(frame[rng.choice(W * H, size=300)], h)
    B = np.concatenate([cells[:40], cells[:5], np.full((2, d), 10_000, dtype=np.int64)])
    for _ in range(3):
        x0, y0 = int(rng.integers(-20, W)), int(rng.integers(-20, H))
        rect = (x0, y0, x0 + int(rng.integers(0, W)), y0 + int(rng.integers(0, H)))
        st, r, present, msg = _gpu_window(frame, W, H, h, B, rect, as_f32)
        assert st == gridshift.GS_OK, msg
        ref, ref_present = oracle.track_window(frame, W, H, h, B, rect)
        _same(r, ref)
        np.testing.assert_array_equal(present, ref_present)


def test_window_step_edge_cases():
    rng = np.random.default_rng(7)
    W, H = 64, 48
    frame = np.rint(rng.uniform(0, 255, size=(W * H, 3)))
    B = _cells(frame[:50], 16.0)
    for rect in [(10, 10, 10, 20), (W, 0, W + 5, H), (-9, -9, 0, 0), (0, 0, W, H)]:
        for bins in [B, np.zeros((0, 3), dtype=np.int64)]:
            st, r, present, msg = _gpu_window(frame, W, H, 16.0, bins, rect)
            assert st == gridshift.GS_OK, msg
            ref, ref_present = oracle.track_window(frame, W, H, 16.0, bins, rect)
            _same(r, ref)
            np.testing.assert_array_equal(present, ref_present)
    # a non-finite colour inside the window is an error; outside it is not read
    frame[5 * W + 7, 1] = np.nan
    st, r, _, _ = _gpu_window(frame, W, H, 16.0, B, (0, 0, W, H))
    assert st == gridshift.GS_E_INVALID and r["count"] == -1
    st, r, _, msg = _gpu_window(frame, W, H, 16.0, B, (0, 10, W, H))
    assert st == gridshift.GS_OK, msg
