"""Agreement of two clusterings of the same points, up to renaming of labels.

Used to state how closely the float32 mixed-precision path reproduces the
float64 result: labels are matched one to one (each cluster of either side
used at most once), greedily by overlap, largest overlap first; the agreement
is the fraction of points whose two labels form a matched pair.  Splitting a
cluster into pieces therefore costs the points of every piece but the
matched one.  Modes are compared on every matched pair.

Pure numpy on host arrays; none of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

__all__ = ["match_clusters", "agreement"]


def match_clusters(lab: np.ndarray, ref_lab: np.ndarray):
    """Greedy one-to-one matching of the labels of ``lab`` to those of
    ``ref_lab`` (same length): pairs sorted by overlap (descending; ties by
    the smaller label pair), each label of either side used at most once.
    Returns (pairs, overlaps): matched (ours, theirs) label pairs and the
    number of points each pair shares."""
    lab = np.asarray(lab, dtype=np.int64).ravel()
    ref_lab = np.asarray(ref_lab, dtype=np.int64).ravel()
    if lab.shape != ref_lab.shape:
        raise ValueError("label arrays differ in length")
    if lab.size == 0:
        return [], []
    pairs, counts = np.unique(np.stack([lab, ref_lab], 1), axis=0, return_counts=True)
    order = np.lexsort((pairs[:, 1], pairs[:, 0], -counts))
    used_a, used_b = set(), set()
    out, ov = [], []
    for i in order.tolist():
        a, b = int(pairs[i, 0]), int(pairs[i, 1])
        if a in used_a or b in used_b:
            continue
        used_a.add(a)
        used_b.add(b)
        out.append((a, b))
        ov.append(int(counts[i]))
    return out, ov


def agreement(lab, ref_lab, modes=None, ref_modes=None, h: float = 1.0) -> dict:
    """Label agreement under the one-to-one matching, the cluster counts of
    both sides, and (when modes are given: k x d arrays in label order) the
    largest max-norm distance between matched modes in units of h."""
    lab = np.asarray(lab).ravel()
    ref_lab = np.asarray(ref_lab).ravel()
    pairs, ov = match_clusters(lab, ref_lab)
    n = lab.size
    k = int(np.unique(lab).size) if n else 0
    k_ref = int(np.unique(ref_lab).size) if n else 0
    out = {"labels": (sum(ov) / n) if n else 1.0, "k": k, "k_ref": k_ref,
           "matched": len(pairs)}
    if modes is not None and ref_modes is not None:
        err = 0.0
        for a, b in pairs:
            err = max(err, float(np.max(np.abs(np.asarray(modes[a]) - np.asarray(ref_modes[b])))))
        out["max_mode_error_h"] = err / h
    return out
