"""The image entry points (gs_fit_image, gs_fit_image_batched) against the
oracle run on the same pixels' float64 features: the (r, g, b) or
(r, g, b, x, y) inputs of the paper's segmentation experiment (Sec. 4.2),
built on the device from the uint8 image.  In GS_FP64 the result is
bit-identical (labels, iterations, float64 modes); in float32 the usual bar
(one-to-one agreement >= 99.9%, equal cluster counts, modes within 1e-3 h)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import agreement, gridshift, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _features(img, xy_scale):
    """The pixels' float64 features, written out here (and equal to the
    synthetic workloads' own builder for three channels)."""
    H, W, C = img.shape
    cols = [img.reshape(H * W, C).astype(np.float64)]
    if xy_scale > 0:
        yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                             indexing="ij")
        cols += [xx.reshape(-1, 1) * xy_scale, yy.reshape(-1, 1) * xy_scale]
    X = np.ascontiguousarray(np.concatenate(cols, 1))
    if C == 3:
        np.testing.assert_array_equal(X, synth.image_features(img, xy_scale if xy_scale > 0
                                                              else None))
    return X


def _check(img, h, xy_scale, precision=gridshift.GS_FP64, max_iter=50):
    X = _features(img, xy_scale)
    ref = oracle.fit(X, h, max_iter)
    d = X.shape[1]
    with gridshift.GridShift(d, h, max_iter, precision=precision) as g:
        labels, modes, info = g.fit_image(torch.from_numpy(np.ascontiguousarray(img)).cuda(),
                                          xy_scale)
        torch.cuda.synchronize()
        # the same context on the features themselves
        l2, m2, i2 = g.fit(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
    lab, md = labels.cpu().numpy(), modes.cpu().numpy()
    if precision == gridshift.GS_FP64:
        assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
        np.testing.assert_array_equal(lab, ref["labels"])
        np.testing.assert_array_equal(md.view(np.int64), ref["modes"].view(np.int64))
    else:
        ag = agreement.agreement(lab, ref["labels"], md, ref["modes"], h)
        assert ag["labels"] >= 0.999 and info["k"] == ref["k"], ag
        assert ag["max_mode_error_h"] <= 1e-3, ag
    # gs_fit_image is gs_fit on the features, plus the feature build (which
    # also takes the key range from the pixels: the same plan, so the same
    # cells, window and statistics)
    np.testing.assert_array_equal(lab, l2.cpu().numpy())
    # (two launches with positions: the column and row products, then the rows)
    assert info["launches"] == i2["launches"] + (2 if xy_scale > 0 else 1)
    for key in ("m0", "inexact", "cell_iters", "iterations"):
        assert info[key] == i2[key], key


@pytest.mark.parametrize("xy_scale", [0.0, 0.1, 0.37])
def test_image_rgb_fp64(xy_scale):
    img = synth.voronoi_image(123, 211, 12, 8.0, seed=5)
    _check(img, 12.0, xy_scale)


def test_image_gradient_fp64_and_fp32():
    img = synth.voronoi_image(150, 173, 9, 6.0, seed=8, gradient=0.3)
    _check(img, 10.0, 0.1)
    _check(img, 10.0, 0.1, precision=gridshift.GS_FP32_MIXED)


@pytest.mark.parametrize("C,xy_scale", [(1, 0.5), (1, 0.0), (4, 0.0), (2, 1.0)])
def test_image_other_channel_counts(C, xy_scale):
    rng = np.random.default_rng(40 + C)
    base = synth.voronoi_image(97, 131, 7, 6.0, seed=C)
    img = np.ascontiguousarray(np.concatenate([base] * 2, axis=2)[:, :, :C])
    img[::5, ::7] = rng.integers(0, 256, size=img[::5, ::7].shape, dtype=np.uint8)
    _check(img, 16.0, xy_scale)


def test_image_full_1080p():
    # the bench's 1920x1080 workload through the image entry point: the same
    # result as gs_fit on its float64 features (which the full-size parity
    # tests pin to the oracle)
    w = synth.WORKLOADS["image_1080p_d5"]()
    with gridshift.GridShift(5, w["h"], w["max_iter"]) as g:
        labels, modes, info = g.fit_image(torch.from_numpy(w["image"]).cuda(), w["xy_scale"])
        l2, m2, i2 = g.fit(torch.from_numpy(w["points"]).cuda())
        torch.cuda.synchronize()
    np.testing.assert_array_equal(labels.cpu().numpy(), l2.cpu().numpy())
    np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64),
                                  m2.cpu().numpy().view(np.int64))
    for key in ("m0", "inexact", "cell_iters", "iterations", "k"):
        assert info[key] == i2[key], key


def test_image_batched_fp64():
    imgs = [synth.voronoi_image(h, w, r, 8.0, seed=s)
            for (h, w, r, s) in [(40, 60, 5, 1), (1, 1, 1, 2), (77, 50, 9, 3), (64, 64, 12, 4)]]
    pix = np.ascontiguousarray(np.concatenate([im.reshape(-1, 3) for im in imgs], 0))
    offsets = np.concatenate([[0], np.cumsum([im.shape[0] * im.shape[1] for im in imgs])]).tolist()
    with gridshift.GridShift(3, 16.0, 50) as g:
        labels, modes, infos = g.fit_image_batched(torch.from_numpy(pix).cuda(), offsets)
        torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    for b, im in enumerate(imgs):
        ref = oracle.fit(synth.image_features(im), 16.0, 50)
        np.testing.assert_array_equal(lab[offsets[b]:offsets[b + 1]], ref["labels"])
        np.testing.assert_array_equal(modes[b].cpu().numpy().view(np.int64),
                                      ref["modes"].view(np.int64))
        assert infos[b]["iterations"] == ref["iterations"]


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_images_host_stream(pinned):
    # a stream of same-size images in host memory with host outputs: every
    # image's labels and modes equal gs_fit_image's on the device
    imgs = [synth.voronoi_image(90, 140, r, 8.0, seed=s) for r, s in [(6, 1), (11, 2), (4, 3),
                                                                    (9, 4), (7, 5)]]
    H, W, C = imgs[0].shape
    n, cap = H * W, 4096
    with gridshift.GridShift(5, 12.0, 50) as g:
        ref = []
        for im in imgs:
            lab, md, info = g.fit_image(torch.from_numpy(im).cuda(), 0.2)
            torch.cuda.synchronize()
            ref.append((lab.cpu().numpy(), md.cpu().numpy(), info))
        if pinned:
            h_img = [torch.from_numpy(im).pin_memory() for im in imgs]
            h_lab = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in imgs]
            h_md = [torch.empty((cap, 5), dtype=torch.float64).pin_memory() for _ in imgs]
            ptr = lambda t: t.data_ptr()  # noqa: E731
            view = lambda t: t.numpy()  # noqa: E731
        else:
            h_img = [np.ascontiguousarray(im) for im in imgs]
            h_lab = [np.empty(n, dtype=np.int32) for _ in imgs]
            h_md = [np.empty((cap, 5), dtype=np.float64) for _ in imgs]
            ptr = lambda a: a.ctypes.data  # noqa: E731
            view = lambda a: a  # noqa: E731
        st, ks, infos = gridshift.gs_fit_images_host(g._ctx, [ptr(x) for x in h_img], H, W, C,
                                                     0.2, [ptr(x) for x in h_lab],
                                                     [ptr(x) for x in h_md], cap)
        assert st == gridshift.GS_OK, gridshift.gs_get_last_error(g._ctx)
        for i, (lab, md, info) in enumerate(ref):
            assert ks[i] == info["k"] and infos[i].iterations == info["iterations"]
            np.testing.assert_array_equal(view(h_lab[i]), lab)
            np.testing.assert_array_equal(view(h_md[i])[:ks[i]].view(np.int64), md.view(np.int64))
        # too few mode rows for one image: the others are still fitted
        small = min(ks) + 1
        st, ks2, _ = gridshift.gs_fit_images_host(g._ctx, [ptr(x) for x in h_img], H, W, C, 0.2,
                                                  [ptr(x) for x in h_lab],
                                                  [ptr(x) for x in h_md], small)
        assert ks2 == ks
        assert st == (gridshift.GS_E_CAPACITY if max(ks) > small else gridshift.GS_OK)
        for i, (lab, _, _) in enumerate(ref):
            np.testing.assert_array_equal(view(h_lab[i]), lab)
