"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares; argument checks that need no GPU behave as declared.
No compute call is made here (these run without a GPU)."""
from __future__ import annotations

import ctypes
import math
import glob
import os
import re

import numpy as np
import pytest

from paper_2206_02200_gb300 import _native, gridshift

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions() -> list:
    names = []
    for hdr in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(gs_\w+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _native.build()
    return gridshift.load(build_if_missing=False)


def test_header_declares_the_boundary():
    decl = _declared_functions()
    assert set(gridshift.EXPORTS) <= set(decl), decl


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings(lib):
    names = {gridshift.GS_OK: "GS_OK", gridshift.GS_E_INVALID: "GS_E_INVALID",
             gridshift.GS_E_NOMEM: "GS_E_NOMEM", gridshift.GS_E_KEYRANGE: "GS_E_KEYRANGE",
             gridshift.GS_E_CAPACITY: "GS_E_CAPACITY", gridshift.GS_E_CUDA: "GS_E_CUDA",
             gridshift.GS_E_INTERNAL: "GS_E_INTERNAL"}
    for code, name in names.items():
        assert gridshift.gs_status_string(code) == name


@pytest.mark.parametrize("d,h,max_iter", [(0, 1.0, 5), (13, 1.0, 5), (3, 0.0, 5), (3, -1.0, 5),
                                          (3, float("nan"), 5), (3, float("inf"), 5),
                                          (3, 1.0, -1)])
def test_create_rejects_bad_arguments(lib, d, h, max_iter):
    ctx = ctypes.c_void_p()
    st = lib.gs_create(d, h, max_iter, ctypes.byref(ctx))
    assert st == gridshift.GS_E_INVALID
    assert not ctx.value


def test_create_destroy_and_host_only_checks(lib):
    ctx = gridshift.gs_create(3, 16.0, 50)
    try:
        assert gridshift.gs_set_precision(ctx, 7) == gridshift.GS_E_INVALID
        assert gridshift.gs_get_last_error(ctx)
        assert gridshift.gs_set_precision(ctx, gridshift.GS_FP32_MIXED) == gridshift.GS_OK
        assert gridshift.gs_set_precision(ctx, gridshift.GS_FP64) == gridshift.GS_OK
        # n == 0 returns before any device work
        st, k, info = gridshift.gs_fit(ctx, 0, gridshift.GS_IN_F64, 0, 0, 0, 0)
        assert st == gridshift.GS_OK and k == 0 and info.converged == 1
        # bad arguments are rejected before any device work
        st, _, _ = gridshift.gs_fit(ctx, 0, gridshift.GS_IN_F64, -1, 0, 0, 0)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_fit(ctx, 0, 9, 10, 0, 0, 0)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_fit(ctx, 0, gridshift.GS_IN_F64, 10, 0, 0, 0)
        assert st == gridshift.GS_E_INVALID  # NULL points
        st = lib.gs_fit(ctx, None, 0, 0, None, None, 0, None, None)
        assert st == gridshift.GS_E_INVALID  # NULL k_out
        # batched: host-side checks, and an all-empty batch returns at once
        st, mo, infos = gridshift.gs_fit_batched(ctx, 0, gridshift.GS_IN_F64, [0, 0, 0], 0, 0, 0)
        assert st == gridshift.GS_OK and mo == [0, 0, 0]
        assert [i.converged for i in infos] == [1, 1]
        for bad in ([1, 2], [0, 5, 3], [0]):
            st, _, _ = gridshift.gs_fit_batched(ctx, 0, gridshift.GS_IN_F64, bad, 0, 0, 0)
            assert st == gridshift.GS_E_INVALID, bad
    finally:
        gridshift.gs_destroy(ctx)
    lib.gs_destroy(None)  # ignored


def test_update_form_host_only_checks(lib):
    ctx = gridshift.gs_create(2, 1.0, 10)
    try:
        assert gridshift.gs_set_update(ctx, 5) == gridshift.GS_E_INVALID
        assert gridshift.gs_get_last_error(ctx)
        assert gridshift.gs_set_update(ctx, gridshift.GS_UPDATE_SEQUENTIAL) == gridshift.GS_OK
        # the sequential form runs in GS_FP64 on one point set: other uses
        # are refused before any device work
        assert gridshift.gs_set_precision(ctx, gridshift.GS_FP32_MIXED) == gridshift.GS_OK
        st, _, _ = gridshift.gs_fit(ctx, 0, gridshift.GS_IN_F64, 0, 0, 0, 0)
        assert st == gridshift.GS_E_INVALID
        assert gridshift.gs_set_precision(ctx, gridshift.GS_FP64) == gridshift.GS_OK
        st, k, _ = gridshift.gs_fit(ctx, 0, gridshift.GS_IN_F64, 0, 0, 0, 0)
        assert st == gridshift.GS_OK and k == 0
        st, _, _ = gridshift.gs_fit_batched(ctx, 0, gridshift.GS_IN_F64, [0, 0, 0], 0, 0, 0)
        assert st == gridshift.GS_E_INVALID
        assert gridshift.gs_set_update(ctx, gridshift.GS_UPDATE_PARALLEL) == gridshift.GS_OK
        st, _, _ = gridshift.gs_fit_batched(ctx, 0, gridshift.GS_IN_F64, [0, 0, 0], 0, 0, 0)
        assert st == gridshift.GS_OK
    finally:
        gridshift.gs_destroy(ctx)
    assert lib.gs_set_update(None, 0) == gridshift.GS_E_INVALID


def test_tensor_front_end_rejects_unknown_forms(lib):
    pytest.importorskip("torch")
    for kw in ({"update": 9}, {"precision": 4}):
        with pytest.raises(gridshift.GridShiftError):
            gridshift.GridShift(3, 1.0, 10, **kw)
    with gridshift.GridShift(3, 1.0, 10, update=gridshift.GS_UPDATE_SEQUENTIAL) as g:
        assert g._ctx


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2206_02200_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if not path.endswith((".py", ".cu", ".cuh", ".h")):
            continue
        text = open(path).read()
        assert "import oracle" not in text and "from oracle" not in text, path
        assert "gs_oracle" not in text and "gso_" not in text, path


def test_track_window_host_only_checks(lib):
    # argument checks and empty windows return before any device work
    ctx = gridshift.gs_create(3, 16.0, 1)
    try:
        bins = np.zeros((2, 3), dtype=np.int64)
        st, res, present = gridshift.gs_track_window(ctx, 0, gridshift.GS_IN_F64, 64, 48, bins,
                                                     10, 10, 10, 20)  # zero-width window
        assert st == gridshift.GS_OK and res.count == 0 and present.tolist() == [0, 0]
        assert math.isnan(res.mean_x) and res.min_x > res.max_x
        st, res, _ = gridshift.gs_track_window(ctx, 0, gridshift.GS_IN_F64, 64, 48, bins,
                                               70, 0, 90, 48)  # right of the frame
        assert st == gridshift.GS_OK and res.count == 0
        st, _, _ = gridshift.gs_track_window(ctx, 0, gridshift.GS_IN_F64, -1, 48, bins, 0, 0, 1, 1)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_track_window(ctx, 0, 9, 64, 48, bins, 0, 0, 1, 1)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_track_window(ctx, 0, gridshift.GS_IN_F64, 64, 48, bins, 0, 0, 8, 8)
        assert st == gridshift.GS_E_INVALID  # NULL frame with a non-empty window
        out = gridshift.gs_track_result()
        assert lib.gs_track_window(ctx, None, 0, 4, 4, None, 1, 0, 0, 4, 4, ctypes.byref(out),
                                   None) == gridshift.GS_E_INVALID  # bins NULL with k > 0
    finally:
        gridshift.gs_destroy(ctx)


def test_window_rect():
    # W(o, l, w): the pixels within l/2 of o_x and w/2 of o_y
    assert gridshift.window_rect((10.5, 20.0), 5.0, 4.0) == (8, 18, 14, 23)
    assert gridshift.window_rect((0.0, 0.0), 1.0, 1.0) == (0, 0, 1, 1)
    assert gridshift.window_rect((3.2, 7.7), 0.2, 0.2) == (4, 8, 4, 8)  # no pixel inside


def test_noalloc_host_only_checks(lib):
    # argument checks and the per-point limit are decided before any device
    # call: 8 bytes a point plus 1 MiB must fit the 64 MiB static array
    F64 = gridshift.GS_IN_F64
    fake = 1 << 20  # never dereferenced: every case below returns first
    st, k, info = gridshift.gs_fit_noalloc(3, 1.0, 10, None, 0, F64, 0, 0, 0, 0)
    assert st == gridshift.GS_OK and k == 0 and info.converged == 1
    for args in ((0, 1.0, 10), (9, 1.0, 10), (3, 0.0, 10), (3, math.inf, 10), (3, 1.0, -1)):
        st, _, _ = gridshift.gs_fit_noalloc(*args, None, fake, F64, 10, fake, 0, 0)
        assert st == gridshift.GS_E_INVALID, args
    st, _, _ = gridshift.gs_fit_noalloc(3, 1.0, 10, None, fake, 7, 10, fake, 0, 0)
    assert st == gridshift.GS_E_INVALID  # dtype
    st, _, _ = gridshift.gs_fit_noalloc(3, 1.0, 10, None, 0, F64, 10, fake, 0, 0)
    assert st == gridshift.GS_E_INVALID  # NULL points
    limit = ((64 << 20) - (1 << 20)) // 8  # 8,257,536 points
    assert limit == 8_257_536
    st, _, _ = gridshift.gs_fit_noalloc(3, 1.0, 10, None, fake, F64, limit + 1, fake, 0, 0)
    assert st == gridshift.GS_E_SCRATCH



def test_sweep_host_only_checks(lib):
    F64 = gridshift.GS_IN_F64
    fake = 1 << 20  # never dereferenced: every case below returns first
    ctx = gridshift.gs_create(3, 16.0, 10)
    try:
        st, mo, infos = gridshift.gs_fit_sweep(ctx, 0, F64, 0, [4.0, 8.0], 0, 0, 0)
        assert st == gridshift.GS_OK and mo == [0, 0, 0] and [i.converged for i in infos] == [1, 1]
        for hs in ([], [1.0, 0.0], [math.nan], [-2.0], [math.inf, 1.0]):
            st, _, _ = gridshift.gs_fit_sweep(ctx, fake, F64, 10, hs, fake, 0, 0)
            assert st == gridshift.GS_E_INVALID, hs
        st, _, _ = gridshift.gs_fit_sweep(ctx, fake, F64, 1 << 30, [1.0, 2.0], fake, 0, 0)
        assert st == gridshift.GS_E_INVALID  # B x n >= 2^31
        st, _, _ = gridshift.gs_fit_sweep(ctx, 0, F64, 10, [1.0, 2.0], fake, 0, 0)
        assert st == gridshift.GS_E_INVALID  # NULL points
        assert gridshift.gs_set_precision(ctx, gridshift.GS_FP32_MIXED) == gridshift.GS_OK
        st, _, _ = gridshift.gs_fit_sweep(ctx, fake, F64, 10, [1.0, 2.0], fake, 0, 0)
        assert st == gridshift.GS_E_INVALID and "GS_FP64" in gridshift.gs_get_last_error(ctx)
    finally:
        gridshift.gs_destroy(ctx)


def test_wide_dimensions_host_only_checks(lib):
    # d up to 12 is accepted (the wide-key pipeline); batched runs, sweeps and
    # the tracking window step keep the packed key (d <= 8) and refuse first
    F64 = gridshift.GS_IN_F64
    fake = 1 << 20
    ctx = gridshift.gs_create(12, 1.0, 10)
    try:
        st, k, info = gridshift.gs_fit(ctx, 0, F64, 0, 0, 0, 0)
        assert st == gridshift.GS_OK and k == 0
        st, _, _ = gridshift.gs_fit_batched(ctx, fake, F64, [0, 5, 10], fake, 0, 0)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_fit_sweep(ctx, fake, F64, 10, [1.0, 2.0], fake, 0, 0)
        assert st == gridshift.GS_E_INVALID
        st, _, _ = gridshift.gs_track_window(ctx, fake, F64, 8, 8, np.zeros((1, 12), np.int64),
                                             0, 0, 4, 4)
        assert st == gridshift.GS_E_INVALID
    finally:
        gridshift.gs_destroy(ctx)


def test_image_entry_points_host_only_checks(lib):
    # argument checks of gs_fit_image / gs_fit_image_batched, made before any
    # device work
    ctx = gridshift.gs_create(5, 12.0, 50)
    try:
        # an empty image returns at once
        st, k, info = gridshift.gs_fit_image(ctx, 0, 0, 7, 3, 0.5, 0, 0, 0)
        assert st == gridshift.GS_OK and k == 0 and info.converged == 1
        for args in ((1, 1, 3, 0.0),      # d = 3 against the context's 5
                     (1, 1, 5, 0.5),      # d = 7
                     (-1, 4, 3, 0.5),     # negative height
                     (4, -1, 3, 0.5),     # negative width
                     (1 << 16, 1 << 16, 3, 0.5),  # 2^32 pixels
                     (1, 1, 0, 0.5), (1, 1, 9, 0.5),  # channels
                     (1, 1, 3, -1.0), (1, 1, 3, float("nan")), (1, 1, 3, float("inf"))):
            H, W, C, s = args
            st, _, _ = gridshift.gs_fit_image(ctx, 0, H, W, C, s, 0, 0, 0)
            assert st == gridshift.GS_E_INVALID, args
        # pixels but no output
        st, _, _ = gridshift.gs_fit_image(ctx, 1, 2, 2, 3, 0.5, 0, 0, 0)
        assert st == gridshift.GS_E_INVALID
        # the host-buffer stream of images: no image is no work; bad
        # arguments are rejected before any device work
        assert gridshift.gs_fit_images_host(ctx, [], 4, 4, 3, 0.5, [], [], 0)[0] == gridshift.GS_OK
        for args in (([1], 4, 4, 3, 0.0, [1]),      # d = 3 against 5
                     ([0], 4, 4, 3, 0.5, [1]),      # NULL image
                     ([1], 4, 4, 3, 0.5, [0]),      # NULL labels
                     ([1], -4, 4, 3, 0.5, [1]),     # negative height
                     ([1], 4, 4, 9, 0.5, [1])):     # channels
            imgs, H, W, C, sc, labs = args
            st, _, _ = gridshift.gs_fit_images_host(ctx, imgs, H, W, C, sc, labs, [], 0)
            assert st == gridshift.GS_E_INVALID, args
    finally:
        gridshift.gs_destroy(ctx)
    ctx = gridshift.gs_create(3, 12.0, 50)
    try:
        st, mo, infos = gridshift.gs_fit_image_batched(ctx, 0, 3, [0, 0, 0], 0, 0, 0)
        assert st == gridshift.GS_OK and mo == [0, 0, 0]
        for C, offsets in ((4, [0, 5]), (3, [1, 5]), (3, [0, 5, 4]), (0, [0, 5])):
            st, _, _ = gridshift.gs_fit_image_batched(ctx, 1, C, offsets, 1, 0, 0)
            assert st == gridshift.GS_E_INVALID, (C, offsets)
    finally:
        gridshift.gs_destroy(ctx)


def test_tuning_host_only_checks(lib, tmp_path):
    ctx = gridshift.gs_create(5, 12.0, 50)
    try:
        assert gridshift.gs_get_tuning(ctx) == gridshift.DEFAULT_TUNING
        t = {"few_lanes_x4": 16, "load_shift": 1, "filter": 0, "tail_enter": 256,
             "pencil_min": 0, "split_min": 5, "bin_list": 0, "bin_sums": 1}
        assert gridshift.gs_set_tuning(ctx, t) == gridshift.GS_OK
        assert gridshift.gs_get_tuning(ctx) == t
        for bad in ({"load_shift": 3}, {"load_shift": 0}, {"filter": 2}, {"tail_enter": 257},
                    {"tail_enter": -1}, {"few_lanes_x4": -1}, {"pencil_min": -5},
                    {"split_min": -1}, {"bin_list": 2}, {"bin_sums": 2}, {"bin_sums": -1}):
            assert gridshift.gs_set_tuning(ctx, bad) == gridshift.GS_E_INVALID, bad
            assert gridshift.gs_get_tuning(ctx) == t  # unchanged
        assert gridshift.gs_set_tuning(ctx, None) == gridshift.GS_OK
        assert gridshift.gs_get_tuning(ctx) == gridshift.DEFAULT_TUNING
    finally:
        gridshift.gs_destroy(ctx)


def test_autotune_cache_lookup(tmp_path):
    import json
    from paper_2206_02200_gb300 import autotune
    F64, F32 = gridshift.GS_FP64, gridshift.GS_FP32_MIXED
    assert autotune.key_for(5, F64, 2_073_600, False) == "d5_fp64_one_n2^21"
    assert autotune.key_for(3, F32, 47_465_008, True) == "d3_fp32_batch_n2^26"
    cache = {"d5_fp64_one_n2^21": {"tuning": {"filter": 0}},
             "d5_fp64_one_n2^23": {"tuning": {"filter": 1}},
             "d3_fp32_batch_n2^26": {"tuning": {"load_shift": 1}}}
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps(cache))
    e = autotune.lookup(5, F64, 2_073_600, False, path=str(path))
    assert e["key"] == "d5_fp64_one_n2^21" and e["tuning"] == {"filter": 0}
    assert autotune.lookup(5, F64, 1 << 23, False, path=str(path))["tuning"] == {"filter": 1}
    assert autotune.lookup(5, F64, 1 << 19, False, path=str(path))["key"] == "d5_fp64_one_n2^21"
    assert autotune.lookup(5, F64, 1 << 26, False, path=str(path)) is None  # too far
    assert autotune.lookup(5, F32, 2_073_600, False, path=str(path)) is None
    assert autotune.lookup(3, F32, 40_000_000, True, path=str(path))["tuning"] == {"load_shift": 1}
    for k, v in gridshift.DEFAULT_TUNING.items():
        assert v in autotune.CANDIDATES[k]
