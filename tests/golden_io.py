"""Reader of the hand-worked fixtures under tests/golden/."""
from __future__ import annotations

import glob
import os
from fractions import Fraction

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path: str) -> dict:
    lines = [ln.split("#", 1)[0].strip() for ln in open(path)]
    lines = [ln for ln in lines if ln]
    out: dict = {"name": os.path.basename(path)}
    i = 0
    while i < len(lines):
        head, *rest = lines[i].split()
        if head in ("points", "modes"):
            rows = []
            i += 1
            while i < len(lines) and lines[i].split()[0] not in (
                    "labels", "iterations", "converged", "m_hist", "modes", "points", "h",
                    "max_iter", "tol_ulp"):
                rows.append(lines[i].split())
                i += 1
            if head == "points":
                out["points"] = np.array([[float(Fraction(v)) for v in r] for r in rows])
            else:
                out["modes"] = [[Fraction(v) for v in r] for r in rows]
            continue
        if head == "h":
            out["h"] = float(Fraction(rest[0]))
        elif head in ("max_iter", "iterations", "converged", "tol_ulp"):
            out[head] = int(rest[0])
        elif head in ("labels", "m_hist"):
            out[head] = [int(v) for v in rest]
        i += 1
    return out


def all_cases() -> list:
    """The hand-worked cases of the parallel update (Eq. 6)."""
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]


def sequential_cases() -> list:
    """The hand-worked cases of the sequential update (Eq. 5)."""
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "sequential", "*.txt")))]


def step_limit_cases() -> list:
    """Hand-worked cases stopped by max_iter (parallel update)."""
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "step_limit", "*.txt")))]
