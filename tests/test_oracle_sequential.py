"""Pins of the oracle's sequential update (Sec. 2.2, Eq. 5: Algorithm 1 writes
each cell's new centroid in place, so cells later in the sweep read it).

The sweep order is the oracle's reading of an order the paper leaves to the
hash table: ascending parity colour (bit d-1-a of the colour is k_a mod 2),
then ascending key.  The pins:
  * hand-worked examples (tests/golden/sequential/), within a few ulp of the
    exact rational result;
  * an independent brute force (Python Fractions, O(m^2) neighbour search,
    the colour order written as a sort on parity tuples) on tiny inputs,
    bit for bit;
  * cells of one colour are never neighbours, so any order inside a colour
    gives the same result; the order of the colours does matter;
  * closed forms shared with the parallel form (one cell, separated clusters)
    and the invariants of Sec. 2.1 and Theorem 2.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from tests import golden_io


def _bf_floor(x: float, h: float) -> int:
    return math.floor(Fr(x) / Fr(h))


def colour_order(keys, d: int, axis0_major: bool = True) -> list:
    """Cells sorted by their tuple of key parities (axis 0 first, or last),
    then by key."""
    axes = range(d) if axis0_major else range(d - 1, -1, -1)
    return sorted(keys, key=lambda k: (tuple(k[a] % 2 for a in axes), k))


def _bf_sweep(cells: dict, d: int, order: list):
    """One sequential update: cells in `order`; a neighbour updated earlier
    contributes count x new centroid, any other its stored sum."""
    new = {}
    any_nb = False
    for j in order:
        D = 0
        N = [Fr(0)] * d
        for q in cells:
            if max(abs(q[a] - j[a]) for a in range(d)) <= 1:
                D += cells[q][0]
                for a in range(d):
                    N[a] += cells[q][0] * Fr(new[q][a]) if q in new else Fr(cells[q][1][a])
                if q != j:
                    any_nb = True
        new[j] = [float(N[a] / D) for a in range(d)]
    return new, any_nb


def brute_force_sequential(X: np.ndarray, h: float, max_iter: int, order_fn=None) -> dict:
    n, d = X.shape
    order_fn = order_fn or (lambda keys: colour_order(keys, d))
    pts_key = [tuple(_bf_floor(float(v), h) for v in row) for row in X]
    cells: dict = {}
    for i, k in enumerate(pts_key):
        c = cells.setdefault(k, [0, [Fr(0)] * d])
        c[0] += 1
        for a in range(d):
            c[1][a] += Fr(float(X[i, a]))
    cells = {k: [c, [float(s) for s in S]] for k, (c, S) in cells.items()}
    where = {k: k for k in cells}
    m_hist = [len(cells)]
    t = 0
    converged = False
    while True:
        cen, any_nb = _bf_sweep(cells, d, order_fn(list(cells)))
        if not any_nb:
            converged = True
            break
        if t == max_iter:
            break
        groups: dict = {}
        for j, s in cen.items():
            groups.setdefault(tuple(_bf_floor(v, h) for v in s), []).append(j)
        new = {}
        moved = {}
        for nk, members in groups.items():
            cnt = sum(cells[j][0] for j in members)
            S = [float(sum(cells[j][0] * Fr(cen[j][a]) for j in members)) for a in range(d)]
            new[nk] = [cnt, S]
            for j in members:
                moved[j] = nk
        where = {k0: moved[k] for k0, k in where.items()}
        cells = new
        t += 1
        m_hist.append(len(cells))
    order = sorted(cells)
    rank = {k: r for r, k in enumerate(order)}
    labels = np.array([rank[where[k]] for k in pts_key], dtype=np.int32)
    modes = np.array([[cells[k][1][a] / cells[k][0] for a in range(d)] for k in order])
    return dict(labels=labels, modes=modes, iterations=t, converged=converged, m_hist=m_hist,
                keys=np.array(order, dtype=np.int64).reshape(len(order), d),
                counts=np.array([cells[k][0] for k in order]))


def _same(r, b):
    return (r["iterations"] == b["iterations"] and r["converged"] == b["converged"]
            and r["m_hist"].tolist() == b["m_hist"] and np.array_equal(r["labels"], b["labels"])
            and np.array_equal(r["keys"], b["keys"])
            and np.array_equal(r["counts"].astype(np.int64), b["counts"])
            and np.array_equal(r["modes"], b["modes"]))


# ---------------------------------------------------------------------------
# Hand-worked fixtures


@pytest.mark.parametrize("case", golden_io.sequential_cases(), ids=lambda c: c["name"])
def test_sequential_golden(case):
    r = oracle.fit(case["points"], case["h"], case["max_iter"], update="sequential")
    assert r["labels"].tolist() == case["labels"]
    assert r["iterations"] == case["iterations"]
    assert int(r["converged"]) == case["converged"]
    assert r["m_hist"].tolist() == case["m_hist"]
    want = case["modes"]
    assert r["modes"].shape == (len(want), len(want[0]))
    for got_row, want_row in zip(r["modes"], want):
        for g, w in zip(got_row, want_row):
            assert abs(Fr(float(g)) - w) <= case["tol_ulp"] * Fr(math.ulp(float(w))), (g, w)


def test_sequential_differs_from_parallel_on_e1():
    # the parallel form merges keys 0 and 1 in its first update (E1); the
    # sequential one does not
    X = np.array([[0.25], [0.75], [1.5], [4.25], [4.75], [7.5]])
    par = oracle.fit(X, 1.0, 50)
    seq = oracle.fit(X, 1.0, 50, update="sequential")
    assert par["m_hist"].tolist() == [4, 3] and seq["m_hist"].tolist() == [4, 4, 3]
    assert par["modes"][0, 0] == float(Fr(5, 6))
    assert seq["modes"][0, 0] != par["modes"][0, 0]


def test_sequential_colour_order_is_pinned():
    # S2 and S3 tell the colour order from key order and from the colour
    # order with the axes' bits reversed: both alternatives give another run
    for name, alt in [("s2_1d_chain.txt", lambda keys: sorted(keys)),
                      ("s3_2d_colour_order.txt", lambda keys: colour_order(keys, 2, False))]:
        case = golden_io.load(f"{golden_io.GOLDEN_DIR}/sequential/{name}")
        r = oracle.fit(case["points"], case["h"], 50, update="sequential")
        b = brute_force_sequential(case["points"], case["h"], 50)
        assert _same(r, b)
        other = brute_force_sequential(case["points"], case["h"], 50, order_fn=alt)
        assert not _same(r, other)


# ---------------------------------------------------------------------------
# Brute force on tiny inputs (bit-exact)


def _tiny_inputs():
    rng = np.random.default_rng(2206)
    cases = []
    for trial in range(30):
        d = 1 + trial % 3
        n = int(rng.integers(1, 50))
        h = float(rng.choice([1.0, 0.75, 2.5]))
        kind = trial % 3
        if kind == 0:  # continuous, a few clusters, some negative values
            C = rng.uniform(-4, 4, size=(3, d))
            X = C[rng.integers(0, 3, n)] + rng.normal(0, 0.8, size=(n, d))
        elif kind == 1:  # dyadic grid values: many points exactly on faces
            X = rng.integers(-8, 9, size=(n, d)) / 4.0
        else:  # integers with a coarse cell
            X = rng.integers(0, 12, size=(n, d)).astype(np.float64)
            h = 2.0
        cases.append((X, h, int(rng.choice([0, 1, 2, 50]))))
    return cases


@pytest.mark.parametrize("X,h,max_iter", _tiny_inputs())
def test_sequential_brute_force_matches(X, h, max_iter):
    r = oracle.fit(X, h, max_iter, update="sequential")
    b = brute_force_sequential(X, h, max_iter)
    assert _same(r, b)


def test_order_inside_a_colour_is_free():
    # two distinct cells of one colour differ by an even, non-zero amount on
    # some axis: they never see each other, so shuffling the cells inside
    # each colour leaves every bit of the run unchanged
    rng = np.random.default_rng(31)
    for d in (1, 2, 3):
        X = rng.normal(0, 2.5, size=(60, d))

        def shuffled(keys, d=d):
            out = []
            by = {}
            for k in colour_order(keys, d):
                by.setdefault(tuple(k[a] % 2 for a in range(d)), []).append(k)
            for par in sorted(by):
                grp = by[par]
                out.extend(grp[i] for i in rng.permutation(len(grp)))
            return out

        r = oracle.fit(X, 1.0, 50, update="sequential")
        assert _same(r, brute_force_sequential(X, 1.0, 50, order_fn=shuffled))


# ---------------------------------------------------------------------------
# Closed forms and invariants


def test_sequential_closed_forms():
    rng = np.random.default_rng(8)
    # one cell: no update, the mode is the mean
    X = 5.0 * (7 + rng.uniform(0, 1, size=(300, 3)))
    r = oracle.fit(X, 5.0, 50, update="sequential")
    assert r["iterations"] == 0 and r["converged"] and r["k"] == 1
    for a in range(3):
        assert r["modes"][0, a] == math.fsum(X[:, a]) / 300
    # clusters two or more cells apart: nothing moves, both forms agree
    centers = np.array([[0, 0], [2, 0], [0, 5], [-3, -3]])
    lab = rng.integers(0, 4, 200)
    X = centers[lab] + rng.uniform(0, 1, size=(200, 2))
    par = oracle.fit(X, 1.0, 50)
    seq = oracle.fit(X, 1.0, 50, update="sequential")
    assert seq["iterations"] == 0 and _same(seq, {**par, "m_hist": par["m_hist"].tolist(),
                                                   "counts": par["counts"].astype(np.int64)})
    # two adjacent 1-D cells a < b: b reads a's new centroid,
    # s_b = (c_a s_a + S_b) / (c_a + c_b) with s_a = (S_a + S_b) / (c_a + c_b)
    X = np.array([[0.125], [0.25], [0.5], [1.75]])
    r = oracle.fit(X, 1.0, 1, update="sequential")
    s_a = (Fr(0.875) + Fr(1.75)) / 4
    s_b = (3 * Fr(float(s_a)) + Fr(1.75)) / 4
    assert r["iterations"] == 1 and r["k"] == 1  # both keys are 0
    want = (3 * Fr(float(s_a)) + Fr(float(s_b))) / 4
    assert abs(Fr(float(r["modes"][0, 0])) - want) <= Fr(math.ulp(float(want)))


def test_sequential_max_iter_and_empty():
    r = oracle.fit(np.zeros((0, 2)), 1.0, 10, update="sequential")
    assert r["k"] == 0
    X = np.array([[0.5], [1.5], [2.5]])
    r = oracle.fit(X, 1.0, 0, update="sequential")
    assert r["iterations"] == 0 and not r["converged"] and r["k"] == 3
    with pytest.raises(ValueError):
        oracle.fit(X, 1.0, 1, update="gauss")


@pytest.mark.parametrize("d,h,seed", [(2, 0.6, 0), (3, 1.0, 1), (4, 2.0, 2)])
def test_sequential_invariants(d, h, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 10, size=(5, d))
    X = C[rng.integers(0, 5, 2000)] + rng.normal(0, 0.7, size=(2000, d))
    r = oracle.fit(X, h, 50, trace=True, update="sequential")
    n = X.shape[0]
    assert int(r["counts"].sum()) == n
    assert np.all(np.diff(r["m_hist"]) <= 0)
    keys = [tuple(k) for k in r["keys"]]
    assert keys == sorted(set(keys))
    assert np.array_equal(np.bincount(r["labels"], minlength=r["k"]),
                          r["counts"].astype(np.int64))
    lo = np.floor(X.min(axis=0) / h)
    hi = np.floor(X.max(axis=0) / h)
    assert np.all(r["keys"] >= lo) and np.all(r["keys"] <= hi)  # convex combinations
    if r["converged"]:
        K = r["keys"]
        for i in range(len(K)):
            dist = np.max(np.abs(K - K[i]), axis=1)
            dist[i] = 99
            assert dist.min() >= 2  # Theorem 2
    tr = r["trace"]
    scale = np.abs(X).max() * n
    for t in range(r["iterations"]):
        assert np.all(np.abs(tr[t, 0] - tr[t, 1]) <= r["m_hist"][t] * scale * 2.0 ** -52)
