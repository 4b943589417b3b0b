"""Python binding of libgridshift (the C ABI of include/gridshift.h).

Argument marshalling only: every step of GridShift runs in the CUDA library.
The low-level functions carry the C names (``gs_create``, ``gs_fit``, ...);
``GridShift`` wraps a context for torch tensors on a CUDA device.

There is no CPU fallback: if the library cannot be loaded, or no CUDA device is
visible, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

from . import _native

# Status codes (gs_status)
GS_OK = 0
GS_E_INVALID = 1
GS_E_NOMEM = 2
GS_E_KEYRANGE = 3
GS_E_CAPACITY = 4
GS_E_CUDA = 5
GS_E_INTERNAL = 6
GS_E_SCRATCH = 7

# Precisions (gs_precision) and input types (gs_dtype)
GS_FP64 = 0
GS_FP32_MIXED = 1
GS_IN_F64 = 0
GS_IN_F32 = 1

# Update forms (gs_update): Eq. 6 (parallel) and Eq. 5 (sequential)
GS_UPDATE_PARALLEL = 0
GS_UPDATE_SEQUENTIAL = 1

#: every symbol the header declares, in declaration order
EXPORTS = ("gs_create", "gs_set_precision", "gs_set_update", "gs_set_stream", "gs_fit",
           "gs_fit_batched", "gs_fit_image", "gs_fit_images_host", "gs_fit_image_batched",
           "gs_fit_sweep",
           "gs_set_tuning", "gs_get_tuning",
           "gs_set_timing", "gs_get_phase_times", "gs_fit_noalloc", "gs_track_window",
           "gs_get_last_error", "gs_status_string", "gs_destroy")

#: gs_phase names, in enum order (CUDA-event phases and the loop kernel's own
#: device-clock split)
PHASES = ("range", "bin", "loop", "sort", "k_offsets", "k_scatter", "k_sums", "k_level0",
          "k_update_first", "k_update_rest", "k_compact", "k_labels", "labels_out")


class gs_fit_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("m0", ctypes.c_int64), ("k", ctypes.c_int64), ("inexact", ctypes.c_int64),
                ("cell_iters", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("face_rechecks", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class gs_phase_times(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(PHASES)), ("count", ctypes.c_int32 * len(PHASES)),
                ("step_ms", (ctypes.c_double * 2) * 16)]

    def as_dict(self) -> dict:
        return {p: (float(self.ms[i]), int(self.count[i])) for i, p in enumerate(PHASES)}

    def steps(self) -> list:
        """[(update ms, compaction ms)] of the first 16 update steps."""
        return [(float(self.step_ms[i][0]), float(self.step_ms[i][1])) for i in range(16)]


class gs_tuning(ctypes.Structure):
    _fields_ = [("few_lanes_x4", ctypes.c_int32), ("load_shift", ctypes.c_int32),
                ("filter", ctypes.c_int32), ("tail_enter", ctypes.c_int32),
                ("pencil_min", ctypes.c_int32), ("split_min", ctypes.c_int32),
                ("bin_list", ctypes.c_int32), ("bin_sums", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


#: the library's built-in launch choices (gs_set_tuning with NULL)
DEFAULT_TUNING = {"few_lanes_x4": 4, "load_shift": 2, "filter": 1, "tail_enter": 128,
                  "pencil_min": 4096, "split_min": 1 << 22, "bin_list": 1, "bin_sums": 0}


class gs_track_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("sum_x", ctypes.c_int64), ("sum_y", ctypes.c_int64),
                ("mean_x", ctypes.c_double), ("mean_y", ctypes.c_double),
                ("min_x", ctypes.c_int64), ("max_x", ctypes.c_int64),
                ("min_y", ctypes.c_int64), ("max_y", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: (float(getattr(self, f)) if t is ctypes.c_double else int(getattr(self, f)))
                for f, t in self._fields_}


class GridShiftError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libgridshift.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _native.stale():
        _native.build()
    if not os.path.exists(_native.LIB):
        raise RuntimeError(f"libgridshift is not built ({_native.LIB} missing)")
    L = ctypes.CDLL(_native.LIB)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.gs_create.restype = i32
    L.gs_create.argtypes = [i32, ctypes.c_double, i32, ctypes.POINTER(vp)]
    L.gs_set_precision.restype = i32
    L.gs_set_precision.argtypes = [vp, i32]
    L.gs_set_update.restype = i32
    L.gs_set_update.argtypes = [vp, i32]
    L.gs_set_stream.restype = i32
    L.gs_set_stream.argtypes = [vp, vp]
    L.gs_fit.restype = i32
    L.gs_fit.argtypes = [vp, vp, i32, i64, vp, vp, i64, ctypes.POINTER(i64),
                         ctypes.POINTER(gs_fit_info)]
    L.gs_fit_batched.restype = i32
    L.gs_fit_batched.argtypes = [vp, vp, i32, ctypes.POINTER(i64), i32, vp, vp, i64,
                                 ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_fit_image.restype = i32
    L.gs_fit_image.argtypes = [vp, vp, i64, i64, i32, ctypes.c_double, vp, vp, i64,
                               ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_fit_images_host.restype = i32
    L.gs_fit_images_host.argtypes = [vp, i32, ctypes.POINTER(vp), i64, i64, i32, ctypes.c_double,
                                     ctypes.POINTER(vp), ctypes.POINTER(vp), i64,
                                     ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_fit_image_batched.restype = i32
    L.gs_fit_image_batched.argtypes = [vp, vp, i32, ctypes.POINTER(i64), i32, vp, vp, i64,
                                       ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_fit_sweep.restype = i32
    L.gs_fit_sweep.argtypes = [vp, vp, i32, i64, ctypes.POINTER(ctypes.c_double), i32, vp, vp,
                               i64, ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_set_tuning.restype = i32
    L.gs_set_tuning.argtypes = [vp, ctypes.POINTER(gs_tuning)]
    L.gs_get_tuning.restype = i32
    L.gs_get_tuning.argtypes = [vp, ctypes.POINTER(gs_tuning)]
    L.gs_set_timing.restype = i32
    L.gs_set_timing.argtypes = [vp, i32]
    L.gs_get_phase_times.restype = i32
    L.gs_get_phase_times.argtypes = [vp, ctypes.POINTER(gs_phase_times)]
    L.gs_fit_noalloc.restype = i32
    L.gs_fit_noalloc.argtypes = [i32, ctypes.c_double, i32, vp, vp, i32, i64, vp, vp, i64,
                                 ctypes.POINTER(i64), ctypes.POINTER(gs_fit_info)]
    L.gs_track_window.restype = i32
    L.gs_track_window.argtypes = [vp, vp, i32, i64, i64, vp, i64, i64, i64, i64, i64,
                                  ctypes.POINTER(gs_track_result), vp]
    L.gs_get_last_error.restype = i32
    L.gs_get_last_error.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    L.gs_status_string.restype = ctypes.c_char_p
    L.gs_status_string.argtypes = [i32]
    L.gs_destroy.restype = None
    L.gs_destroy.argtypes = [vp]
    _lib = L
    return L


# ---------------------------------------------------------------------------
# C names


def gs_create(d: int, h: float, max_iter: int) -> int:
    ctx = ctypes.c_void_p()
    st = load().gs_create(int(d), float(h), int(max_iter), ctypes.byref(ctx))
    if st != GS_OK:
        raise GridShiftError(st, f"gs_create(d={d}, h={h}, max_iter={max_iter})")
    return ctx.value


def gs_set_precision(ctx: int, precision: int) -> int:
    return load().gs_set_precision(ctx, int(precision))


def gs_set_update(ctx: int, update: int) -> int:
    return load().gs_set_update(ctx, int(update))


def gs_set_stream(ctx: int, stream: int | None) -> int:
    return load().gs_set_stream(ctx, stream or None)


def gs_fit(ctx: int, points_ptr: int, dtype: int, n: int, labels_ptr: int, modes_ptr: int,
           modes_cap: int):
    """Raw call; returns (status, k, gs_fit_info)."""
    k = ctypes.c_int64(0)
    info = gs_fit_info()
    st = load().gs_fit(ctx, points_ptr or None, int(dtype), int(n), labels_ptr or None,
                       modes_ptr or None, int(modes_cap), ctypes.byref(k), ctypes.byref(info))
    return st, int(k.value), info


def gs_fit_image(ctx: int, pixels_ptr: int, height: int, width: int, channels: int,
                 xy_scale: float, labels_ptr: int, modes_ptr: int, modes_cap: int):
    """Raw call; returns (status, k, gs_fit_info)."""
    k = ctypes.c_int64(0)
    info = gs_fit_info()
    st = load().gs_fit_image(ctx, pixels_ptr or None, int(height), int(width), int(channels),
                             float(xy_scale), labels_ptr or None, modes_ptr or None,
                             int(modes_cap), ctypes.byref(k), ctypes.byref(info))
    return st, int(k.value), info


def gs_fit_images_host(ctx: int, image_ptrs, height: int, width: int, channels: int,
                       xy_scale: float, label_ptrs, mode_ptrs, modes_cap: int):
    """Raw call on host buffers (lists of addresses, one per image; page-locked
    memory lets the copies overlap the fits).  Returns (status, k list,
    list of gs_fit_info)."""
    count = len(image_ptrs)
    arr = ctypes.c_void_p * max(count, 1)
    imgs = arr(*[int(p) for p in image_ptrs])
    labs = arr(*[int(p) for p in label_ptrs])
    mds = arr(*[int(p) if p else None for p in mode_ptrs]) if mode_ptrs else None
    ks = (ctypes.c_int64 * max(count, 1))()
    infos = (gs_fit_info * max(count, 1))()
    st = load().gs_fit_images_host(ctx, int(count), imgs, int(height), int(width), int(channels),
                                   float(xy_scale), labs, mds, int(modes_cap), ks, infos)
    return st, list(ks)[:count], list(infos)[:count]


def gs_fit_image_batched(ctx: int, pixels_ptr: int, channels: int, offsets, labels_ptr: int,
                         modes_ptr: int, modes_cap: int):
    """Raw call; offsets: B + 1 pixel offsets.  Returns (status, mode_offsets list,
    list of gs_fit_info)."""
    B = len(offsets) - 1
    off = (ctypes.c_int64 * (B + 1))(*[int(o) for o in offsets])
    mo = (ctypes.c_int64 * (B + 1))()
    infos = (gs_fit_info * max(B, 1))()
    st = load().gs_fit_image_batched(ctx, pixels_ptr or None, int(channels), off, int(B),
                                     labels_ptr or None, modes_ptr or None, int(modes_cap),
                                     mo, infos)
    return st, list(mo), list(infos)[:B]


def gs_track_window(ctx: int, frame_ptr: int, dtype: int, width: int, height: int, bins,
                    x0: int, y0: int, x1: int, y1: int):
    """Raw call; bins: host k x d int64 array.  Returns (status, gs_track_result,
    present uint8[k])."""
    import numpy as np
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64))
    k = b.shape[0] if b.ndim == 2 else 0
    present = np.zeros(max(k, 1), dtype=np.uint8)
    res = gs_track_result()
    st = load().gs_track_window(ctx, frame_ptr or None, int(dtype), int(width), int(height),
                                b.ctypes.data if k else None, int(k), int(x0), int(y0), int(x1),
                                int(y1), ctypes.byref(res), present.ctypes.data)
    return st, res, present[:k]


def gs_fit_batched(ctx: int, points_ptr: int, dtype: int, offsets, labels_ptr: int,
                   modes_ptr: int, modes_cap: int):
    """Raw call; offsets: B + 1 host integers.  Returns (status, mode_offsets
    list of B + 1, list of B gs_fit_info)."""
    B = len(offsets) - 1
    off = (ctypes.c_int64 * (B + 1))(*[int(v) for v in offsets])
    mo = (ctypes.c_int64 * (B + 1))()
    infos = (gs_fit_info * max(B, 1))()
    st = load().gs_fit_batched(ctx, points_ptr or None, int(dtype), off, int(B), labels_ptr or None,
                               modes_ptr or None, int(modes_cap), mo, infos)
    return st, [int(v) for v in mo], [infos[i] for i in range(B)]


def gs_fit_sweep(ctx: int, points_ptr: int, dtype: int, n: int, hs, labels_ptr: int,
                 modes_ptr: int, modes_cap: int):
    """Raw call; hs: B host floats.  Returns (status, mode_offsets list of B + 1,
    list of B gs_fit_info)."""
    B = len(hs)
    hv = (ctypes.c_double * max(B, 1))(*[float(v) for v in hs])
    mo = (ctypes.c_int64 * (B + 1))()
    infos = (gs_fit_info * max(B, 1))()
    st = load().gs_fit_sweep(ctx, points_ptr or None, int(dtype), int(n), hv, int(B),
                             labels_ptr or None, modes_ptr or None, int(modes_cap), mo, infos)
    return st, [int(v) for v in mo], [infos[i] for i in range(B)]


def gs_set_tuning(ctx: int, tuning: dict | None) -> int:
    """Raw call; tuning: dict of gs_tuning fields (missing ones take the
    defaults), or None for the built-in choices."""
    if tuning is None:
        return load().gs_set_tuning(ctx, None)
    t = gs_tuning(**{k: int(v) for k, v in dict(DEFAULT_TUNING, **tuning).items()})
    return load().gs_set_tuning(ctx, ctypes.byref(t))


def gs_get_tuning(ctx: int) -> dict:
    t = gs_tuning()
    st = load().gs_get_tuning(ctx, ctypes.byref(t))
    if st != GS_OK:
        raise GridShiftError(st, "gs_get_tuning")
    return t.as_dict()


def gs_set_timing(ctx: int, enable: bool) -> int:
    return load().gs_set_timing(ctx, 1 if enable else 0)


def gs_get_phase_times(ctx: int, steps: bool = False):
    """{phase: (device ms, launch groups)} of the context's last gs_fit; with
    steps=True also the per-step split [(update ms, compaction ms)]."""
    out = gs_phase_times()
    st = load().gs_get_phase_times(ctx, ctypes.byref(out))
    if st != GS_OK:
        raise GridShiftError(st, "gs_get_phase_times")
    return (out.as_dict(), out.steps()) if steps else out.as_dict()


def gs_fit_noalloc(d: int, h: float, max_iter: int, stream: int | None, points_ptr: int,
                   dtype: int, n: int, labels_ptr: int, modes_ptr: int, modes_cap: int):
    """gs_fit with all scratch in the library's static device array; returns
    (status, k, gs_fit_info).  For callers that cannot allocate device memory."""
    k = ctypes.c_int64(0)
    info = gs_fit_info()
    st = load().gs_fit_noalloc(int(d), float(h), int(max_iter), stream or None,
                               points_ptr or None, int(dtype), int(n), labels_ptr or None,
                               modes_ptr or None, int(modes_cap), ctypes.byref(k),
                               ctypes.byref(info))
    return st, int(k.value), info


def gs_get_last_error(ctx: int) -> str:
    buf = ctypes.create_string_buffer(1024)
    load().gs_get_last_error(ctx, buf, len(buf))
    return buf.value.decode(errors="replace")


def gs_status_string(status: int) -> str:
    return load().gs_status_string(int(status)).decode()


def status_string(status: int) -> str:
    try:
        return gs_status_string(status)
    except Exception:  # pragma: no cover
        return f"status {status}"


def gs_destroy(ctx: int) -> None:
    if ctx:
        load().gs_destroy(ctx)


# ---------------------------------------------------------------------------
# Tensor front end


class GridShift:
    """A GridShift context (cell side h, at most max_iter updates) for d-dim points.

    ``fit(points)`` takes an n x d float64 or float32 CUDA tensor and returns
    (labels int32[n], modes float64[k x d], info dict), all on the points'
    device, computed on the current torch stream.  ``update`` selects the
    parallel (Eq. 6, default) or sequential (Eq. 5) update form.
    """

    def __init__(self, d: int, h: float, max_iter: int = 50, precision: int = GS_FP64,
                 update: int = GS_UPDATE_PARALLEL, tuning=None):
        import torch  # noqa: F401  (device memory and streams)
        self.d, self.h, self.max_iter = int(d), float(h), int(max_iter)
        self.precision = int(precision)
        self._ctx = gs_create(self.d, self.h, self.max_iter)
        st = gs_set_precision(self._ctx, precision)
        if st == GS_OK:
            st = gs_set_update(self._ctx, update)
        if st == GS_OK and isinstance(tuning, dict):
            st = gs_set_tuning(self._ctx, tuning)
        if st != GS_OK:
            msg = gs_get_last_error(self._ctx)
            gs_destroy(self._ctx)
            self._ctx = None
            raise GridShiftError(st, msg)
        self._modes_cap = 1024
        # "auto": the autotuner's cached choice for each call's size (see
        # autotune.py), looked up per point count
        self._auto = tuning == "auto"
        self._auto_n = None
        self.tuning_source = "given" if isinstance(tuning, dict) else "built-in"

    def _apply_auto_tuning(self, n: int, batched: bool = False) -> None:
        if not self._auto or self._auto_n == (n, batched):
            return
        from . import autotune
        entry = autotune.lookup(self.d, self.precision, n, batched)
        st = gs_set_tuning(self._ctx, entry["tuning"] if entry else None)
        if st != GS_OK:
            raise GridShiftError(st, gs_get_last_error(self._ctx))
        self.tuning_source = entry["key"] if entry else "built-in (no cache entry)"
        self._auto_n = (n, batched)

    def tuning(self) -> dict:
        """The launch choices the context uses now."""
        return gs_get_tuning(self._ctx)

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            gs_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_timing(self, enable: bool) -> None:
        gs_set_timing(self._ctx, enable)

    def phase_times(self) -> dict:
        return gs_get_phase_times(self._ctx)

    def fit_into(self, points, labels, modes):
        """Runs gs_fit with caller-provided output tensors; returns (status, k, info)."""
        import torch
        if points.dtype == torch.float64:
            dt = GS_IN_F64
        elif points.dtype == torch.float32:
            dt = GS_IN_F32
        else:
            raise TypeError("points must be float64 or float32")
        if not points.is_cuda or not points.is_contiguous() or points.dim() != 2:
            raise ValueError("points must be a contiguous n x d CUDA tensor")
        if points.shape[1] != self.d:
            raise ValueError(f"points have d={points.shape[1]}, context has d={self.d}")
        stream = torch.cuda.current_stream(points.device).cuda_stream
        gs_set_stream(self._ctx, stream)
        self._apply_auto_tuning(points.shape[0])
        cap = 0 if modes is None else modes.shape[0]
        return gs_fit(self._ctx, points.data_ptr(), dt, points.shape[0], labels.data_ptr(),
                      0 if modes is None else modes.data_ptr(), cap)

    def fit_sweep(self, points, hs):
        """GridShift on the same points for every bandwidth in hs (one call).
        points: n x d CUDA tensor.  Returns (labels int32[B, n] numbered per
        bandwidth, list of B modes tensors, list of B info dicts)."""
        import torch
        if points.dtype == torch.float64:
            dt = GS_IN_F64
        elif points.dtype == torch.float32:
            dt = GS_IN_F32
        else:
            raise TypeError("points must be float64 or float32")
        if not points.is_cuda or not points.is_contiguous() or points.dim() != 2:
            raise ValueError("points must be a contiguous n x d CUDA tensor")
        n, B = points.shape[0], len(hs)
        with torch.cuda.device(points.device):
            gs_set_stream(self._ctx, torch.cuda.current_stream(points.device).cuda_stream)
            labels = torch.empty((B, n), dtype=torch.int32, device=points.device)
            while True:
                modes = torch.empty((self._modes_cap, self.d), dtype=torch.float64,
                                    device=points.device)
                st, mo, infos = gs_fit_sweep(self._ctx, points.data_ptr(), dt, n, hs,
                                             labels.data_ptr(), modes.data_ptr(), modes.shape[0])
                if st == GS_E_CAPACITY:
                    self._modes_cap = max(2 * self._modes_cap, mo[-1])
                    continue
                if st != GS_OK:
                    raise GridShiftError(st, gs_get_last_error(self._ctx))
                return (labels, [modes[mo[b]:mo[b + 1]] for b in range(len(mo) - 1)],
                        [i.as_dict() for i in infos])

    def fit_batched(self, points, offsets):
        """GridShift on each instance of a concatenated batch.  points: n x d
        CUDA tensor, offsets: B + 1 integers.  Returns (labels int32[n] numbered
        per instance, list of B modes tensors, list of B info dicts)."""
        import torch
        if points.dtype == torch.float64:
            dt = GS_IN_F64
        elif points.dtype == torch.float32:
            dt = GS_IN_F32
        else:
            raise TypeError("points must be float64 or float32")
        if not points.is_cuda or not points.is_contiguous() or points.dim() != 2:
            raise ValueError("points must be a contiguous n x d CUDA tensor")
        n = points.shape[0]
        self._apply_auto_tuning(n, batched=True)
        with torch.cuda.device(points.device):
            gs_set_stream(self._ctx, torch.cuda.current_stream(points.device).cuda_stream)
            labels = torch.empty(n, dtype=torch.int32, device=points.device)
            while True:
                modes = torch.empty((self._modes_cap, self.d), dtype=torch.float64,
                                    device=points.device)
                st, mo, infos = gs_fit_batched(self._ctx, points.data_ptr(), dt, offsets,
                                               labels.data_ptr(), modes.data_ptr(),
                                               modes.shape[0])
                if st == GS_E_CAPACITY:
                    self._modes_cap = max(2 * self._modes_cap, mo[-1])
                    continue
                if st != GS_OK:
                    raise GridShiftError(st, gs_get_last_error(self._ctx))
                return (labels, [modes[mo[b]:mo[b + 1]] for b in range(len(mo) - 1)],
                        [i.as_dict() for i in infos])

    def fit_image(self, image, xy_scale: float = 0.0):
        """GridShift on the pixels of an image (Sec. 4.2): image is a height x
        width x channels uint8 CUDA tensor; each pixel is the point of its
        channel values, followed by (x, y) * xy_scale when xy_scale > 0.  The
        features are built on the device.  Returns (labels int32[height *
        width] in pixel order, modes, info)."""
        import torch
        if image.dtype != torch.uint8 or not image.is_cuda or not image.is_contiguous() \
                or image.dim() != 3:
            raise ValueError("image must be a contiguous height x width x channels uint8 "
                             "CUDA tensor")
        H, W, C = image.shape
        n = H * W
        with torch.cuda.device(image.device):
            gs_set_stream(self._ctx, torch.cuda.current_stream(image.device).cuda_stream)
            self._apply_auto_tuning(n)
            labels = torch.empty(n, dtype=torch.int32, device=image.device)
            while True:
                modes = torch.empty((self._modes_cap, self.d), dtype=torch.float64,
                                    device=image.device)
                st, k, info = gs_fit_image(self._ctx, image.data_ptr(), H, W, C, xy_scale,
                                           labels.data_ptr(), modes.data_ptr(), modes.shape[0])
                if st == GS_E_CAPACITY:
                    self._modes_cap = max(2 * self._modes_cap, k)
                    continue
                if st != GS_OK:
                    raise GridShiftError(st, gs_get_last_error(self._ctx))
                return labels, modes[:k], info.as_dict()

    def fit_image_batched(self, pixels, offsets):
        """GridShift on the pixels of several images (channel values only):
        pixels is an n x channels uint8 CUDA tensor of the images' pixels
        concatenated, offsets B + 1 pixel offsets.  Returns (labels int32[n]
        numbered per image, list of B modes tensors, list of B info dicts)."""
        import torch
        if pixels.dtype != torch.uint8 or not pixels.is_cuda or not pixels.is_contiguous() \
                or pixels.dim() != 2:
            raise ValueError("pixels must be a contiguous n x channels uint8 CUDA tensor")
        n, C = pixels.shape
        self._apply_auto_tuning(n, batched=True)
        with torch.cuda.device(pixels.device):
            gs_set_stream(self._ctx, torch.cuda.current_stream(pixels.device).cuda_stream)
            labels = torch.empty(n, dtype=torch.int32, device=pixels.device)
            while True:
                modes = torch.empty((self._modes_cap, self.d), dtype=torch.float64,
                                    device=pixels.device)
                st, mo, infos = gs_fit_image_batched(self._ctx, pixels.data_ptr(), C, offsets,
                                                     labels.data_ptr(), modes.data_ptr(),
                                                     modes.shape[0])
                if st == GS_E_CAPACITY:
                    self._modes_cap = max(2 * self._modes_cap, mo[-1])
                    continue
                if st != GS_OK:
                    raise GridShiftError(st, gs_get_last_error(self._ctx))
                return (labels, [modes[mo[b]:mo[b + 1]] for b in range(len(mo) - 1)],
                        [i.as_dict() for i in infos])

    def fit(self, points):
        import torch
        n = points.shape[0]
        with torch.cuda.device(points.device):
            labels = torch.empty(n, dtype=torch.int32, device=points.device)
            while True:
                modes = torch.empty((self._modes_cap, self.d), dtype=torch.float64,
                                    device=points.device)
                st, k, info = self.fit_into(points, labels, modes)
                if st == GS_E_CAPACITY:
                    self._modes_cap = max(2 * self._modes_cap, k)
                    continue
                if st != GS_OK:
                    raise GridShiftError(st, gs_get_last_error(self._ctx))
                return labels, modes[:k], info.as_dict()


def fit(points, h: float, max_iter: int = 50):
    """One-shot GridShift on an n x d CUDA tensor: (labels, modes, info)."""
    with GridShift(points.shape[1], h, max_iter) as g:
        return g.fit(points)


# ---------------------------------------------------------------------------
# GridShift-based object tracking (Sec. 2.3, Algorithm 2).  The window step
# runs on the GPU (gs_track_window); the loop around it is host logic.

def window_rect(o, length: float, width: float):
    """Pixel rectangle (x0, y0, x1, y1) of the window W(o, length, width): the
    pixels with |x - o_x| <= length / 2 and |y - o_y| <= width / 2."""
    import math
    return (math.ceil(o[0] - length / 2), math.ceil(o[1] - width / 2),
            math.floor(o[0] + length / 2) + 1, math.floor(o[1] + width / 2) + 1)
