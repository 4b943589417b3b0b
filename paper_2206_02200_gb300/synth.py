"""Seeded synthetic inputs for GridShift mode seeking.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle consume exactly
the same bits from it.

Workload shapes follow the paper's experiments:
  * segmentation images (Sec. 4.2): RGB pixels as features, optionally
    (R, G, B, x, y); the paper uses 481x321 BSDS500 images, which are stood in
    for here by Voronoi-region images with per-region colour, optional colour
    gradient and Gaussian noise, quantised to uint8 like a real photo;
  * clustering (Sec. 4.1, dataset table): millions of low-dimensional points,
    stood in for by a Gaussian mixture.

All generators use numpy's PCG64 (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "voronoi_image",
    "image_features",
    "gmm_points",
    "image_batch",
    "image_batch_item",
    "moving_object_frames",
    "WORKLOADS",
]


def _nearest_site(H: int, W: int, sites: np.ndarray, rows_per_chunk: int = 64) -> np.ndarray:
    """Index of the nearest site (squared Euclidean, ties -> lowest index) per pixel."""
    out = np.empty((H, W), dtype=np.int32)
    xs = np.arange(W, dtype=np.float64)
    sx = sites[:, 0][None, None, :]
    sy = sites[:, 1][None, None, :]
    for y0 in range(0, H, rows_per_chunk):
        y1 = min(H, y0 + rows_per_chunk)
        ys = np.arange(y0, y1, dtype=np.float64)
        dx = xs[None, :, None] - sx
        dy = ys[:, None, None] - sy
        dist = dx * dx + dy * dy
        out[y0:y1] = np.argmin(dist, axis=2)  # argmin returns the first minimum
    return out


def voronoi_image(H: int, W: int, regions: int, sigma: float, seed: int,
                  gradient: float = 0.0) -> np.ndarray:
    """H x W x 3 uint8 image made of ``regions`` Voronoi cells.

    Sites are uniform in [0, W) x [0, H); each region gets a base colour uniform
    in [0, 255]^3; with ``gradient`` > 0 each region also gets a 3x2 slope
    matrix with entries uniform in [-gradient, gradient] applied to the pixel's
    offset from its site; then i.i.d. N(0, sigma^2) noise per channel, clipping
    to [0, 255] and round-half-to-even to uint8.
    """
    rng = np.random.default_rng(seed)
    sites = np.stack([rng.uniform(0.0, W, regions), rng.uniform(0.0, H, regions)], axis=1)
    colours = rng.uniform(0.0, 255.0, size=(regions, 3))
    slopes = rng.uniform(-gradient, gradient, size=(regions, 3, 2)) if gradient > 0 else None
    lab = _nearest_site(H, W, sites)
    img = colours[lab]  # H x W x 3 float64
    if slopes is not None:
        yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                             indexing="ij")
        offx = xx - sites[lab, 0]
        offy = yy - sites[lab, 1]
        g = slopes[lab]  # H x W x 3 x 2
        img = img + g[..., 0] * offx[..., None] + g[..., 1] * offy[..., None]
    img = img + rng.normal(0.0, sigma, size=img.shape)
    img = np.clip(img, 0.0, 255.0)
    return np.rint(img).astype(np.uint8)  # rint rounds half to even


def image_features(img: np.ndarray, xy_scale: float | None = None) -> np.ndarray:
    """Row-major (y outer, x inner) n x d float64 features of an RGB image.

    d = 3 (R, G, B) when ``xy_scale`` is None, else d = 5 with
    (R, G, B, x * xy_scale, y * xy_scale) where x is the column and y the row.
    """
    H, W, _ = img.shape
    rgb = img.reshape(H * W, 3).astype(np.float64)
    if xy_scale is None:
        return np.ascontiguousarray(rgb)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    x = xx.reshape(-1) * xy_scale
    y = yy.reshape(-1) * xy_scale
    return np.ascontiguousarray(np.concatenate([rgb, x[:, None], y[:, None]], axis=1))


def moving_object_frames(H: int, W: int, T: int, seed: int, radius: float = 20.0,
                         speed: float = 3.0, sigma: float = 6.0) -> tuple:
    """T frames (T x H x W x 3 float64, uint8 values) of a disc of one colour
    moving in a straight line over a fixed Voronoi background (8 regions),
    with fresh i.i.d. N(0, sigma^2) noise per frame, and the disc's centre per
    frame (T x 2, (x, y)).  Stands in for a tracking sequence.

    The disc starts at a seed-drawn point in the middle of the image and moves
    ``speed`` pixels per frame in a seed-drawn direction; its colour is drawn
    at least 80 (max-norm) away from every background colour."""
    rng = np.random.default_rng(seed)
    sites = np.stack([rng.uniform(0.0, W, 8), rng.uniform(0.0, H, 8)], axis=1)
    bg = rng.uniform(0.0, 255.0, size=(8, 3))
    while True:
        obj = rng.uniform(0.0, 255.0, size=3)
        if np.min(np.max(np.abs(bg - obj[None, :]), axis=1)) >= 80.0:
            break
    lab = _nearest_site(H, W, sites)
    base = bg[lab]
    c0 = np.array([rng.uniform(0.35 * W, 0.65 * W), rng.uniform(0.35 * H, 0.65 * H)])
    ang = rng.uniform(0.0, 2.0 * np.pi)
    vel = speed * np.array([np.cos(ang), np.sin(ang)])
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    frames = np.empty((T, H, W, 3), dtype=np.float64)
    centres = np.empty((T, 2), dtype=np.float64)
    for t in range(T):
        c = c0 + t * vel
        centres[t] = c
        img = base.copy()
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 <= radius * radius
        img[inside] = obj
        img = img + rng.normal(0.0, sigma, size=img.shape)
        frames[t] = np.rint(np.clip(img, 0.0, 255.0))
    return frames, centres


def gmm_points(n: int, d: int, components: int, seed: int, lo: float = 0.0, hi: float = 100.0,
               sigma_lo: float = 1.0, sigma_hi: float = 3.0) -> np.ndarray:
    """n x d float32 points from an isotropic Gaussian mixture, shuffled.

    Means uniform in [lo, hi]^d, per-component sigma uniform in
    [sigma_lo, sigma_hi], weights Dirichlet(1), counts multinomial; points are
    drawn in float64, randomly permuted and rounded to float32.
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, size=(components, d))
    sig = rng.uniform(sigma_lo, sigma_hi, size=components)
    w = rng.dirichlet(np.ones(components))
    counts = rng.multinomial(n, w)
    comp = np.repeat(np.arange(components), counts)
    pts = means[comp] + sig[comp][:, None] * rng.standard_normal(size=(n, d))
    perm = rng.permutation(n)
    return np.ascontiguousarray(pts[perm].astype(np.float32))


def image_batch(count: int, seed0: int, hmin: int = 240, hmax: int = 1080, wmin: int = 320,
                wmax: int = 1920, rmin: int = 8, rmax: int = 60, sigma: float = 8.0):
    """List of ``count`` RGB feature arrays (d = 3) of uneven sizes.

    Image i uses seed ``seed0 + i``: its height, width and region count are
    drawn uniformly (inclusive) from that seed's stream, then the image itself.
    """
    return [image_batch_item(i, seed0, hmin, hmax, wmin, wmax, rmin, rmax, sigma)
            for i in range(count)]


def image_batch_item(i: int, seed0: int, hmin: int = 240, hmax: int = 1080, wmin: int = 320,
                     wmax: int = 1920, rmin: int = 8, rmax: int = 60,
                     sigma: float = 8.0) -> np.ndarray:
    """Instance i of ``image_batch(count, seed0, ...)`` alone (any count > i)."""
    return image_features(image_batch_image(i, seed0, hmin, hmax, wmin, wmax, rmin, rmax, sigma))


def image_batch_image(i: int, seed0: int, hmin: int = 240, hmax: int = 1080, wmin: int = 320,
                      wmax: int = 1920, rmin: int = 8, rmax: int = 60,
                      sigma: float = 8.0) -> np.ndarray:
    """The uint8 image behind ``image_batch_item(i, seed0, ...)``."""
    rng = np.random.default_rng(seed0 + i)
    H = int(rng.integers(hmin, hmax + 1))
    W = int(rng.integers(wmin, wmax + 1))
    R = int(rng.integers(rmin, rmax + 1))
    return voronoi_image(H, W, R, sigma, seed=seed0 + i + 7919 * (i + 1))


def _image_cfg(img, xy_scale, **kw):
    # the features, and the image they are built from (the image entry points)
    return dict(points=image_features(img, xy_scale=xy_scale), image=img,
                xy_scale=0.0 if xy_scale is None else xy_scale, **kw)


def _cfg_image_small():
    return _image_cfg(voronoi_image(321, 481, 12, 8.0, seed=1), None, h=16.0, max_iter=50,
                      name="voronoi_321x481_d3_h16")


def _cfg_1080p():
    return _image_cfg(voronoi_image(1080, 1920, 40, 10.0, seed=2), 0.1, h=12.0, max_iter=50,
                      name="voronoi_1920x1080_d5_h12")


def _cfg_4k():
    return _image_cfg(voronoi_image(2160, 3840, 120, 10.0, seed=3, gradient=0.02), 0.1, h=10.0,
                      max_iter=50, name="voronoi_gradient_3840x2160_d5_h10")


def _cfg_gmm():
    return dict(points=gmm_points(10_000_000, 6, 200, seed=5), h=4.0, max_iter=50,
                name="gmm_10M_d6_h4")


def _cfg_gmm_4m():
    # the same mixture at 4 million points: a profiling case whose tables
    # exceed L2 while the whole run holds a few GB of device memory
    return dict(points=gmm_points(4_000_000, 6, 200, seed=5), h=4.0, max_iter=50,
                name="gmm_4M_d6_h4")


def _cfg_batch64():
    images = [image_batch_image(i, 1000) for i in range(64)]
    return dict(parts=[image_features(im) for im in images], images=images, h=16.0, max_iter=50,
                name="voronoi_batch64_uneven_d3_h16")


def _cfg_sweep():
    # the 321x481 image over a range of bandwidths (the paper's bandwidth
    # study, Sec. 4.1, gives no values: eight from 8 to 32 here)
    return dict(points=image_features(voronoi_image(321, 481, 12, 8.0, seed=1)),
                hs=[8.0, 10.0, 12.0, 14.0, 16.0, 20.0, 24.0, 32.0], h=8.0, max_iter=50,
                name="voronoi_321x481_d3_sweep8_h8-32")


#: name -> zero-argument builder returning dict(points, h, max_iter, name);
#: batched workloads give dict(parts=[...], h, max_iter, name) instead, and
#: bandwidth sweeps dict(points, hs=[...], h, max_iter, name); image
#: workloads add the uint8 image and xy_scale (batches: the list of images)
WORKLOADS = {
    "image_321x481_d3": _cfg_image_small,
    "image_1080p_d5": _cfg_1080p,
    "image_4k_d5": _cfg_4k,
    "gmm_10M_d6": _cfg_gmm,
    "gmm_4M_d6": _cfg_gmm_4m,
    "batch_64_d3": _cfg_batch64,
    "sweep_321x481_d3": _cfg_sweep,
}
