"""gs_fit_noalloc: the GridShift fit for callers that cannot allocate device
memory (a host program with a fixed GPU memory budget, a plug-in whose host
owns every allocation).  Its scratch is a static device array inside the
library, so two calls in a row must both match gs_fit, the second one starting
from whatever the first left in that array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _same_partition(a, b) -> bool:
    pairs = np.unique(np.stack([a, b], 1), axis=0)
    return len(pairs) == len(np.unique(a)) == len(np.unique(b))


def _fit_with_ctx(X, h, max_iter, dev):
    g = gridshift.GridShift(X.shape[1], h, max_iter)
    pts = torch.from_numpy(X).to(dev)
    labels, modes, info = g.fit(pts)
    torch.cuda.synchronize(dev)
    g.close()
    return labels.cpu().numpy(), modes.cpu().numpy(), info


def _fit_noalloc(pts, h, max_iter, labels, modes, dev):
    stream = torch.cuda.current_stream(dev).cuda_stream
    dt = gridshift.GS_IN_F64 if pts.dtype == torch.float64 else gridshift.GS_IN_F32
    st, k, info = gridshift.gs_fit_noalloc(pts.shape[1], h, max_iter, stream, pts.data_ptr(), dt,
                                           pts.shape[0], labels.data_ptr(), modes.data_ptr(),
                                           modes.shape[0])
    torch.cuda.synchronize(dev)
    return st, k, info


def _check(ref, got, h):
    lab_ref, md_ref, info_ref = ref
    lab, md, k, info = got
    assert k == info_ref["k"] and info.iterations == info_ref["iterations"]
    assert _same_partition(lab, lab_ref)
    assert np.max(np.abs(md[:k] - md_ref)) <= 1e-10 * h
    np.testing.assert_array_equal(lab, lab_ref)
    np.testing.assert_array_equal(md[:k].view(np.int64), md_ref.view(np.int64))


def test_noalloc_matches_gs_fit_twice_in_a_row():
    dev = torch.device("cuda:0")
    # two different inputs, so the second call starts from the first one's leftovers
    X1 = synth.image_features(synth.voronoi_image(321, 481, 12, 8.0, seed=1))
    X2 = synth.image_features(synth.voronoi_image(200, 300, 9, 10.0, seed=5, gradient=0.02),
                              xy_scale=0.1)
    cases = [(X1, 16.0), (X2, 12.0)]
    refs = [_fit_with_ctx(X, h, 50, dev) for X, h in cases]
    for (X, h), ref in zip(cases, refs):
        pts = torch.from_numpy(X).to(dev)
        labels = torch.full((X.shape[0],), -1, dtype=torch.int32, device=dev)
        modes = torch.zeros((4096, X.shape[1]), dtype=torch.float64, device=dev)
        st, k, info = _fit_noalloc(pts, h, 50, labels, modes, dev)
        assert st == gridshift.GS_OK, gridshift.gs_status_string(st)
        got = (labels.cpu().numpy(), modes.cpu().numpy(), k, info)
        _check(ref, got, h)
        # and directly against the oracle, bit for bit
        o = oracle.fit(X, h, 50)
        _check((o["labels"], o["modes"], {"k": o["k"], "iterations": o["iterations"]}), got, h)
    # and the first input again, after the second
    X, h = cases[0]
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty((X.shape[0],), dtype=torch.int32, device=dev)
    modes = torch.empty((4096, 3), dtype=torch.float64, device=dev)
    free_before = torch.cuda.mem_get_info(dev)[0]
    st, k, info = _fit_noalloc(pts, h, 50, labels, modes, dev)
    st2, k2, info2 = _fit_noalloc(pts, h, 50, labels, modes, dev)
    free_after = torch.cuda.mem_get_info(dev)[0]
    assert st == st2 == gridshift.GS_OK
    _check(refs[0], (labels.cpu().numpy(), modes.cpu().numpy(), k2, info2), h)
    assert free_after == free_before  # no device allocation by the calls


def test_noalloc_rejects_inputs_beyond_its_scratch():
    dev = torch.device("cuda:0")
    n = 17_000_000  # 4 bytes per point alone exceed the 64 MiB array
    pts = torch.zeros((n, 1), dtype=torch.float32, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    modes = torch.empty((1, 1), dtype=torch.float64, device=dev)
    st, k, info = _fit_noalloc(pts, 1.0, 10, labels, modes, dev)
    assert st == gridshift.GS_E_SCRATCH
    assert gridshift.gs_status_string(st) == "GS_E_SCRATCH"
    # too many distinct cells for the array: uniform noise in 4-D, tiny cells
    X = np.random.default_rng(0).uniform(0, 1000, size=(2_000_000, 4))
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty(X.shape[0], dtype=torch.int32, device=dev)
    modes = torch.empty((16, 4), dtype=torch.float64, device=dev)
    st, k, info = _fit_noalloc(pts, 1.0, 50, labels, modes, dev)
    assert st == gridshift.GS_E_SCRATCH
    # still usable afterwards
    test_noalloc_matches_gs_fit_twice_in_a_row()


@pytest.mark.parametrize("d", [3, 6])
def test_noalloc_with_nearly_one_cell_per_point(d):
    # as many cells as points and more than 4096 of them: the static tables
    # are sized for the points, so the pencil form of the first update (which
    # needs room for three times the cells) must step aside
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(40 + d)
    X = rng.uniform(0.0, 60.0 if d == 3 else 6.0, size=(5000, d))
    ref = _fit_with_ctx(X, 1.0, 8, dev)
    assert ref[2]["m0"] > 4096
    pts = torch.from_numpy(X).to(dev)
    labels = torch.full((X.shape[0],), -1, dtype=torch.int32, device=dev)
    modes = torch.zeros((8192, d), dtype=torch.float64, device=dev)
    st, k, info = _fit_noalloc(pts, 1.0, 8, labels, modes, dev)
    assert st == gridshift.GS_OK, gridshift.gs_status_string(st)
    _check(ref, (labels.cpu().numpy(), modes.cpu().numpy(), k, info), 1.0)
