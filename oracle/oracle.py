"""ctypes front end of the C oracle (gs_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
legs may import this module.  The product library never does.

``build()`` compiles gs_oracle.c with gcc into oracle/_build/ (plain -O2,
no FP contraction); ``fit()`` runs one GridShift instance (parallel update of
Eq. 6, or the sequential one of Eq. 5); ``fit_batched()`` runs several
independent instances one after another.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_HDR = os.path.join(_HERE, "gs_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgs_oracle.so")

_lib = None


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("m0", ctypes.c_int64), ("k", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or older than its sources."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)
             or os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        for fn in (L.gso_fit, L.gso_fit_sequential):
            fn.restype = ctypes.c_int
            fn.argtypes = [P(ctypes.c_double), ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                           ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int64,
                           P(ctypes.c_int64), P(ctypes.c_uint64), P(ctypes.c_int64),
                           P(ctypes.c_double), P(_Info)]
        L.gso_floor_div.restype = ctypes.c_int64
        L.gso_floor_div.argtypes = [ctypes.c_double, ctypes.c_double]
        L.gso_exact_sum.restype = ctypes.c_double
        L.gso_exact_sum.argtypes = [P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int64]
        L.gso_exact_mean.restype = ctypes.c_double
        L.gso_exact_mean.argtypes = [P(ctypes.c_double), ctypes.c_int64, ctypes.c_uint64]
        L.gso_track_window.restype = ctypes.c_int
        L.gso_track_window.argtypes = [P(ctypes.c_double), ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_double, P(ctypes.c_int64),
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64, P(ctypes.c_int64),
                                       P(ctypes.c_uint8)]
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def fit(points, h: float, max_iter: int = 50, trace: bool = False,
        update: str = "parallel") -> dict:
    """Run the oracle on an n x d array (any real dtype; converted to float64 exactly).

    ``update`` is "parallel" (Eq. 6: every cell reads the state before the
    update) or "sequential" (Eq. 5: a sweep in ascending parity colour, then
    key, that reads the neighbours it has already updated).

    Returns dict(labels, modes, keys, counts, iterations, converged, m0, k,
    m_hist[, trace]).
    """
    if update not in ("parallel", "sequential"):
        raise ValueError("update must be 'parallel' or 'sequential'")
    X = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    if X.ndim != 2:
        raise ValueError("points must be n x d")
    n, d = X.shape
    cap = max(n, 1)
    labels = np.zeros(n, dtype=np.int32)
    modes = np.zeros((cap, d), dtype=np.float64)
    keys = np.zeros((cap, d), dtype=np.int64)
    cnt = np.zeros(cap, dtype=np.uint64)
    m_hist = np.zeros(max_iter + 1, dtype=np.int64)
    tr = np.zeros((max(max_iter, 1), 2, d), dtype=np.float64) if trace else None
    info = _Info()
    fn = lib().gso_fit if update == "parallel" else lib().gso_fit_sequential
    rc = fn(_ptr(X, ctypes.c_double), n, d, float(h), int(max_iter),
                       _ptr(labels, ctypes.c_int32), _ptr(modes, ctypes.c_double), cap,
                       _ptr(keys, ctypes.c_int64), _ptr(cnt, ctypes.c_uint64),
                       _ptr(m_hist, ctypes.c_int64), _ptr(tr, ctypes.c_double),
                       ctypes.byref(info))
    if rc != 0:
        raise RuntimeError(f"oracle {update} fit failed with code {rc}")
    k = int(info.k)
    it = int(info.iterations)
    out = dict(labels=labels, modes=modes[:k].copy(), keys=keys[:k].copy(),
               counts=cnt[:k].copy(), iterations=it, converged=bool(info.converged),
               m0=int(info.m0), k=k, m_hist=m_hist[:it + 1].copy())
    if trace:
        out["trace"] = tr[:it].copy()
    return out


def fit_batched(point_sets, h: float, max_iter: int = 50) -> list:
    """Independent oracle runs, one per instance."""
    return [fit(P, h, max_iter) for P in point_sets]


def floor_div(x: float, h: float) -> int:
    return int(lib().gso_floor_div(float(x), float(h)))


def exact_sum(v, w=None) -> float:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    wa = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.uint32))
    return float(lib().gso_exact_sum(_ptr(v, ctypes.c_double), _ptr(wa, ctypes.c_uint32), v.size))


def exact_mean(v, D: int) -> float:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    return float(lib().gso_exact_mean(_ptr(v, ctypes.c_double), v.size, int(D)))


# ---------------------------------------------------------------------------
# GridShift-based object tracking (Sec. 2.3, Algorithm 2)

def track_window(frame, width: int, height: int, h: float, bins, rect) -> tuple:
    """R of one search window (gso_track_window): returns (dict with count,
    sum_x, sum_y, mean_x, mean_y, min_x, max_x, min_y, max_y; present uint8[k]).
    The mean is the exact integer sum divided by the count, one IEEE division
    (NaN for an empty R)."""
    f = np.ascontiguousarray(np.asarray(frame, dtype=np.float64).reshape(int(height) * int(width), -1))
    d = f.shape[1]
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64).reshape(-1, d))
    k = b.shape[0]
    out = np.zeros(7, dtype=np.int64)
    present = np.zeros(max(k, 1), dtype=np.uint8)
    st = lib().gso_track_window(_ptr(f, ctypes.c_double), int(width), int(height), d, float(h),
                                _ptr(b, ctypes.c_int64), k, int(rect[0]), int(rect[1]),
                                int(rect[2]), int(rect[3]), _ptr(out, ctypes.c_int64),
                                _ptr(present, ctypes.c_uint8))
    if st != 0:
        raise ValueError("a colour in the window has no exact cell")
    cnt = int(out[0])
    r = dict(count=cnt, sum_x=int(out[1]), sum_y=int(out[2]),
             mean_x=float(out[1]) / cnt if cnt else float("nan"),
             mean_y=float(out[2]) / cnt if cnt else float("nan"),
             min_x=int(out[3]), max_x=int(out[4]), min_y=int(out[5]), max_y=int(out[6]))
    return r, present[:k]
