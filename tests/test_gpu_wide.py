"""Keys that the 63-bit packed key cannot hold (Sec. 2.1 keeps integer cell
keys of any size): key fields wider than 63 bits together, more than 2^22
cells along an axis, and d from 9 to 12.  Such runs go through the wide-key
pipeline; labels, iteration counts and float64 modes must equal the oracle's
bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fit(X, h, max_iter=50, f32=False, modes_cap=None):
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if f32:
        pts = pts.float()
    with gridshift.GridShift(X.shape[1], h, max_iter) as g:
        if modes_cap is None:
            labels, modes, info = g.fit(pts)
            torch.cuda.synchronize()
            return labels.cpu().numpy(), modes.cpu().numpy(), info
        lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
        md = torch.empty((max(modes_cap, 1), X.shape[1]), dtype=torch.float64, device="cuda")
        dt = gridshift.GS_IN_F32 if f32 else gridshift.GS_IN_F64
        st, k, info = gridshift.gs_fit(g._ctx, pts.data_ptr(), dt, X.shape[0], lab.data_ptr(),
                                       md.data_ptr(), modes_cap)
        torch.cuda.synchronize()
        return st, k, lab.cpu().numpy(), info


def _check(X, h, max_iter=50, f32=False):
    Xo = X.astype(np.float32).astype(np.float64) if f32 else X
    ref = oracle.fit(Xo, h, max_iter)
    lab, md, info = _fit(X, h, max_iter, f32)
    assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
    assert info["m0"] == ref["m0"] and info["converged"] == int(ref["converged"])
    assert info["inexact"] == 0
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(md.view(np.int64), ref["modes"].view(np.int64))
    return ref


def _key_bits(ref):
    span = ref["keys"].max(axis=0) - ref["keys"].min(axis=0)
    return int(np.sum(np.ceil(np.log2(span + 3))))


def test_keys_wider_than_63_bits():
    # the oracle's brute-force pin inputs: clusters millions of cells apart on
    # every axis (66 and 88 bits of packed key), some points on cell faces
    rng = np.random.default_rng(63)
    for d in (3, 4):
        C = rng.uniform(-2.0e6, 2.0e6, size=(4, d))
        X = C[rng.integers(0, 4, 50)] + rng.normal(0, 0.9, size=(50, d))
        X[:5] = np.round(X[:5] * 2) / 2
        ref = _check(X, 1.0)
        assert _key_bits(ref) > 63


def test_wide_keys_with_many_points_and_merges():
    rng = np.random.default_rng(5)
    C = rng.uniform(-1.0e7, 1.0e7, size=(30, 5))
    X = C[rng.integers(0, 30, 200_000)] + rng.normal(0, 1.0, size=(200_000, 5))
    ref = _check(X, 1.5)
    assert ref["m0"] > 1000 and ref["iterations"] >= 2


def test_more_than_2_22_cells_on_one_axis():
    rng = np.random.default_rng(22)
    X = rng.normal(0, 1.0, size=(3000, 2))
    X[:1500, 0] += 9.0e6  # 9 million cells apart along axis 0
    _check(X, 0.5)


@pytest.mark.parametrize("d", [9, 10, 12])
def test_dimensions_above_8(d):
    rng = np.random.default_rng(900 + d)
    centres = rng.uniform(-6, 6, size=(3, d))
    n = 400 if d < 12 else 60
    X = centres[rng.integers(0, 3, n)] + rng.normal(0, 0.7, size=(n, d))
    _check(X, 2.0, max_iter=10)


def test_wide_step_limits_and_float32_input():
    rng = np.random.default_rng(77)
    C = rng.uniform(-3.0e6, 3.0e6, size=(6, 4))
    X = C[rng.integers(0, 6, 5000)] + rng.normal(0, 3.0, size=(5000, 4))
    for mi in (0, 1, 2):
        _check(X, 1.0, max_iter=mi)
    _check(X.astype(np.float32), 2.0, f32=True)


def test_wide_short_modes_buffer_keeps_labels():
    rng = np.random.default_rng(3)
    C = rng.uniform(-2.0e6, 2.0e6, size=(5, 4))
    X = C[rng.integers(0, 5, 500)] + rng.normal(0, 0.5, size=(500, 4))
    ref = oracle.fit(X, 1.0, 50)
    st, k, lab, info = _fit(X, 1.0, modes_cap=1)
    assert st == gridshift.GS_E_CAPACITY and k == ref["k"]
    np.testing.assert_array_equal(lab, ref["labels"])


def test_wide_refuses_float32_state():
    X = np.random.default_rng(1).normal(0, 1, size=(100, 9))
    pts = torch.from_numpy(X).cuda()
    with gridshift.GridShift(9, 1.0, 10, precision=gridshift.GS_FP32_MIXED) as g:
        with pytest.raises(gridshift.GridShiftError):
            g.fit(pts)
