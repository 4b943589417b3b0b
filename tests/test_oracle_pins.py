"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself.  The pins are:
  * hand-worked examples (tests/golden/, each citing the paper's Sec. 2.1,
    Eq. 1-4 and Algorithm 1), checked to within one rounding of the exact
    rational result;
  * an independent brute force written with Python Fractions and an O(m^2)
    neighbour search (no hashing, no sorting by key), on tiny random inputs;
  * the first update equals grid-kernel mean shift on the raw points
    (supplementary Sec. "Grid KDE": g(.) = 1 iff the cell keys are within one
    cell in every axis);
  * closed forms: one cell, all cells mutually adjacent, separated clusters;
  * invariants: total count, sum conservation across merges (Eq. 4),
    non-increasing active-cell count (Sec. 2.1), unique sorted keys, pairwise
    key distance >= 2 at convergence (Theorem 2), label histogram = counts;
  * the shrink rate of the centroids on a Gaussian sample (Theorem 3), with
    the constant derived from the three-cell window.
"""
from __future__ import annotations

import math
from fractions import Fraction
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from tests import golden_io

# ---------------------------------------------------------------------------
# Independent brute force (Python Fractions, O(m^2) neighbour search).


def _bf_floor(x: float, h: float) -> int:
    return math.floor(Fr(x) / Fr(h))


def _bf_step_centroids(cells: dict, d: int):
    """Parallel update (Eq. 1-2, Eq. 6) by exhaustive pairwise search."""
    keys = list(cells)
    out = {}
    any_nb = False
    for j in keys:
        D = 0
        N = [Fr(0)] * d
        for q in keys:
            if max(abs(q[a] - j[a]) for a in range(d)) <= 1:
                D += cells[q][0]
                for a in range(d):
                    N[a] += Fr(cells[q][1][a])
                if q != j:
                    any_nb = True
        out[j] = [float(N[a] / D) for a in range(d)]
    return out, any_nb


def brute_force(X: np.ndarray, h: float, max_iter: int) -> dict:
    n, d = X.shape
    pts_key = [tuple(_bf_floor(float(v), h) for v in row) for row in X]
    cells: dict = {}
    for i, k in enumerate(pts_key):
        c = cells.setdefault(k, [0, [Fr(0)] * d])
        c[0] += 1
        for a in range(d):
            c[1][a] += Fr(float(X[i, a]))
    cells = {k: [c, [float(s) for s in S]] for k, (c, S) in cells.items()}
    where = {k: k for k in cells}  # initial key -> current key
    m_hist = [len(cells)]
    t = 0
    converged = False
    while True:
        cen, any_nb = _bf_step_centroids(cells, d)
        if not any_nb:
            converged = True
            break
        if t == max_iter:
            break
        groups: dict = {}
        for j, s in cen.items():
            nk = tuple(_bf_floor(v, h) for v in s)
            groups.setdefault(nk, []).append(j)
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


# ---------------------------------------------------------------------------
# Hand-worked fixtures


@pytest.mark.parametrize("case", golden_io.all_cases(), ids=lambda c: c["name"])
def test_golden_examples(case):
    r = oracle.fit(case["points"], case["h"], case["max_iter"])
    assert r["labels"].tolist() == case["labels"]
    assert r["iterations"] == case["iterations"]
    assert int(r["converged"]) == case["converged"]
    assert r["m_hist"].tolist() == case["m_hist"]
    want = case["modes"]
    assert r["modes"].shape == (len(want), len(want[0]))
    for got_row, want_row in zip(r["modes"], want):
        for g, w in zip(got_row, want_row):
            # within one rounding of the exact rational value
            assert abs(Fr(float(g)) - w) <= Fr(math.ulp(float(w))), (g, w)


@pytest.mark.parametrize("case", golden_io.step_limit_cases(), ids=lambda c: c["name"])
def test_golden_step_limit(case):
    test_golden_examples(case)
    assert not oracle.fit(case["points"], case["h"], case["max_iter"])["converged"]


def test_golden_chain_is_not_plain_mean():
    # E2: the converged mode 97/48 differs from the mean of the points (2.0);
    # an implementation that merged everything at once would return 2.0.
    case = golden_io.load(golden_io.GOLDEN_DIR + "/e2_1d_chain.txt")
    r = oracle.fit(case["points"], case["h"], 50)
    assert r["modes"][0, 0] == float(Fr(97, 48))
    assert r["modes"][0, 0] != 2.0


# ---------------------------------------------------------------------------
# Brute force on tiny random inputs (bit-exact)


def _tiny_inputs():
    rng = np.random.default_rng(12345)
    cases = []
    for trial in range(40):
        d = 1 + trial % 4
        n = int(rng.integers(1, 60))
        h = float(rng.choice([1.0, 0.75, 2.5, 0.3]))
        kind = trial % 3
        if kind == 0:  # continuous, a few clusters, some negative values
            C = rng.uniform(-4, 4, size=(3, d))
            X = C[rng.integers(0, 3, n)] + rng.normal(0, 0.8, size=(n, d))
        elif kind == 1:  # dyadic grid values: many points exactly on faces
            X = rng.integers(-8, 9, size=(n, d)) / 4.0
        else:  # integers, like 8-bit pixel values, with a coarse cell
            X = rng.integers(0, 12, size=(n, d)).astype(np.float64)
            h = 2.0
        cases.append((X, h, int(rng.choice([0, 1, 2, 50]))))
    return cases


@pytest.mark.parametrize("X,h,max_iter", _tiny_inputs())
def test_brute_force_matches(X, h, max_iter):
    r = oracle.fit(X, h, max_iter)
    b = brute_force(X, h, max_iter)
    assert r["iterations"] == b["iterations"]
    assert r["converged"] == b["converged"]
    assert r["m_hist"].tolist() == b["m_hist"]
    assert np.array_equal(r["labels"], b["labels"])
    assert np.array_equal(r["keys"], b["keys"])
    assert np.array_equal(r["counts"].astype(np.int64), b["counts"])
    assert np.array_equal(r["modes"], b["modes"])  # bit-exact


def test_wide_key_ranges_match_brute_force():
    # keys far apart on every axis: a packed key of these cells would need
    # more than 63 bits (d = 4 axes spanning 2^22 cells each); the oracle
    # keeps one int64 per axis and must still match the brute force
    rng = np.random.default_rng(63)
    for d in (3, 4):
        C = rng.uniform(-2.0e6, 2.0e6, size=(4, d))
        X = C[rng.integers(0, 4, 50)] + rng.normal(0, 0.9, size=(50, d))
        X[:5] = np.round(X[:5] * 2) / 2  # some points on cell faces
        r = oracle.fit(X, 1.0, 50)
        b = brute_force(X, 1.0, 50)
        span = r["keys"].max(axis=0) - r["keys"].min(axis=0)
        assert np.sum(np.ceil(np.log2(span + 3))) > 63
        assert r["iterations"] == b["iterations"] and r["m_hist"].tolist() == b["m_hist"]
        assert np.array_equal(r["labels"], b["labels"])
        assert np.array_equal(r["keys"], b["keys"])
        assert np.array_equal(r["modes"], b["modes"])


def test_brute_force_order_independent():
    # The result does not depend on the order of the points (Eq. 1-4 define
    # sums only); the oracle's exact sums make that hold bit for bit.
    rng = np.random.default_rng(7)
    X = rng.normal(0, 3, size=(300, 2))
    r1 = oracle.fit(X, 1.3, 50)
    perm = rng.permutation(300)
    r2 = oracle.fit(X[perm], 1.3, 50)
    assert np.array_equal(r1["modes"], r2["modes"])
    assert np.array_equal(r1["labels"][perm], r2["labels"])


# ---------------------------------------------------------------------------
# First update = grid-kernel mean shift on raw points


def test_first_update_is_grid_kernel_mean_shift():
    # Dyadic inputs with few bits: every cell sum is exact in FP64, so one
    # update of the cell state equals, exactly, the mean of the raw points whose
    # key is within one cell of the cell's key (g = 1, supplementary Grid KDE).
    rng = np.random.default_rng(99)
    for d in (1, 2, 3):
        X = rng.integers(-40, 40, size=(80, d)) / 8.0
        h = 1.5
        keys = np.array([[_bf_floor(v, h) for v in row] for row in X])
        cells = {}
        for i, k in enumerate(map(tuple, keys)):
            c = cells.setdefault(k, [0, [Fr(0)] * d])
            c[0] += 1
            for a in range(d):
                c[1][a] += Fr(float(X[i, a]))
        cells = {k: [c, [float(s) for s in S]] for k, (c, S) in cells.items()}
        cen, _ = _bf_step_centroids(cells, d)
        for j, s in cen.items():
            near = np.max(np.abs(keys - np.array(j)), axis=1) <= 1
            want = [float(sum(Fr(float(v)) for v in X[near, a]) / int(near.sum()))
                    for a in range(d)]
            assert s == want
        # and the oracle after one update holds, per new cell, the sum of
        # count-weighted centroids of its members
        r = oracle.fit(X, h, 1)
        groups = {}
        for j, s in cen.items():
            groups.setdefault(tuple(_bf_floor(v, h) for v in s), []).append(j)
        if r["iterations"] == 1:
            assert sorted(groups) == [tuple(k) for k in r["keys"]]
            for row, k in enumerate(sorted(groups)):
                cnt = sum(cells[j][0] for j in groups[k])
                assert int(r["counts"][row]) == cnt


# ---------------------------------------------------------------------------
# Closed forms


def test_single_cell_is_mean():
    rng = np.random.default_rng(3)
    for d in (1, 3, 6):
        X = 5.0 * (7 + rng.uniform(0, 1, size=(500, d)))  # all in key 7 for h = 5
        r = oracle.fit(X, 5.0, 50)
        assert r["iterations"] == 0 and r["converged"] and r["k"] == 1
        assert np.all(r["labels"] == 0)
        for a in range(d):
            assert r["modes"][0, a] == math.fsum(X[:, a]) / 500


def test_all_adjacent_cells_merge_in_one_update():
    rng = np.random.default_rng(4)
    for d in (1, 2, 4):
        h = 2.0
        X = h * (3 + rng.integers(0, 16, size=(200, d)) / 8.0)  # keys 3 or 4 in each axis
        keys = np.floor(X / h)
        assert set(np.unique(keys)) <= {3.0, 4.0}
        r = oracle.fit(X, h, 50)
        assert r["k"] == 1 and r["converged"]
        assert r["iterations"] == (1 if len(np.unique(keys, axis=0)) > 1 else 0)
        n = X.shape[0]
        for a in range(d):
            s = float(sum(Fr(float(v)) for v in X[:, a]) / n)  # common centroid
            want = float(n * Fr(s)) / n
            assert r["modes"][0, a] == want


def test_separated_clusters_do_not_move():
    rng = np.random.default_rng(5)
    d, h = 3, 1.0
    centers = np.array([[0, 0, 0], [2, 0, 0], [0, 5, 2], [-3, -3, -3], [2, 2, 2]])
    lab = rng.integers(0, len(centers), 400)
    X = centers[lab] + rng.uniform(0, 1, size=(400, d))
    r = oracle.fit(X, h, 50)
    assert r["iterations"] == 0 and r["converged"]
    order = sorted(range(len(centers)), key=lambda c: tuple(centers[c]))
    rank = {c: i for i, c in enumerate(order)}
    assert np.array_equal(r["labels"], np.array([rank[c] for c in lab]))
    for c in range(len(centers)):
        for a in range(d):
            assert r["modes"][rank[c], a] == math.fsum(X[lab == c, a]) / int((lab == c).sum())


def test_empty_and_degenerate():
    r = oracle.fit(np.zeros((0, 3)), 1.0, 10)
    assert r["k"] == 0 and r["labels"].size == 0
    r = oracle.fit(np.full((10, 2), 3.25), 0.5, 10)
    assert r["k"] == 1 and r["iterations"] == 0 and np.all(r["modes"] == 3.25)
    # max_iter = 0: no update is applied; the binning is returned
    X = np.array([[0.5], [1.5], [2.5]])
    r = oracle.fit(X, 1.0, 0)
    assert r["iterations"] == 0 and not r["converged"] and r["k"] == 3


# ---------------------------------------------------------------------------
# Invariants on medium inputs


@pytest.mark.parametrize("d,h,seed", [(2, 0.6, 0), (3, 1.0, 1), (5, 2.0, 2)])
def test_invariants(d, h, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 10, size=(6, d))
    X = C[rng.integers(0, 6, 3000)] + rng.normal(0, 0.7, size=(3000, d))
    r = oracle.fit(X, h, 50, trace=True)
    n = X.shape[0]
    assert int(r["counts"].sum()) == n
    assert np.all(np.diff(r["m_hist"]) <= 0)  # m_{t+1} <= m_t
    keys = [tuple(k) for k in r["keys"]]
    assert keys == sorted(set(keys))  # unique, ascending
    hist = np.bincount(r["labels"], minlength=r["k"])
    assert np.array_equal(hist, r["counts"].astype(np.int64))
    lo = np.floor(X.min(axis=0) / h)
    hi = np.floor(X.max(axis=0) / h)
    assert np.all(r["keys"] >= lo) and np.all(r["keys"] <= hi)  # convexity
    if r["converged"]:
        K = r["keys"]
        for i in range(len(K)):
            dist = np.max(np.abs(K - K[i]), axis=1)
            dist[i] = 99
            assert dist.min() >= 2  # Theorem 2
    # Eq. 4: a merge conserves the total of count-weighted centroids; each
    # merged sum is rounded once, so the totals agree to that rounding.
    tr = r["trace"]
    scale = np.abs(X).max() * n
    for t in range(r["iterations"]):
        assert np.all(np.abs(tr[t, 0] - tr[t, 1]) <= r["m_hist"][t] * scale * 2.0 ** -52)


# ---------------------------------------------------------------------------
# Convergence rate on a Gaussian sample (Theorem 3, a loose check)


def _centroid_spread(r):
    c = r["counts"].astype(np.float64)
    m = r["modes"]
    mu = (c[:, None] * m).sum(0) / c.sum()
    return np.sqrt((c[:, None] * (m - mu) ** 2).sum(0) / c.sum())


@pytest.mark.parametrize("s,h,d", [(8.0, 1.0, 1), (5.0, 1.0, 1), (6.0, 2.0, 1), (5.0, 1.0, 2)])
def test_gaussian_shrink_rate(s, h, d):
    # Theorem 3: on a Gaussian sample the cell centroids shrink towards the
    # mean at every update, s' = s / (1 + c h^2 / s^2).  For s >> h the
    # leading-order constant follows from the update itself: a cell's new
    # centroid is the mean of the three-cell window around it (variance
    # (3h)^2 / 12 = 3/4 h^2 about its centre), so it moves by -(3/4) h^2 x / s^2,
    # while the cell means it starts from already sit -(1/12) h^2 x / s^2 from
    # the cell centres: c = 3/4 - 1/12 = 2/3 relative to the spread of the cell
    # means (the theorem prints 2.25 h^2).  A wrong window (a dropped or extra
    # term, a shifted neighbourhood) moves c far from 2/3.
    rng = np.random.default_rng(583 + int(10 * s) + d)
    X = rng.normal(0, s, size=(60000, d))
    spreads = [_centroid_spread(oracle.fit(X, h, t)) for t in range(4)]
    c = (spreads[0] / spreads[1] - 1) * spreads[0] ** 2 / h ** 2
    assert np.all(np.abs(c - 2.0 / 3.0) < 0.03), c
    for t in range(3):
        assert np.all(spreads[t + 1] < spreads[t])  # shrinks at every update


# ---------------------------------------------------------------------------
# Exact helpers


def test_floor_div_exact():
    rng = np.random.default_rng(11)
    hs = [0.1, 0.3, 1.0, 12.0, 10.0, 1e-3, 7.25]
    for _ in range(3000):
        h = float(rng.choice(hs))
        q = int(rng.integers(-1000, 1000))
        x = q * h
        for v in (x, np.nextafter(x, -np.inf), np.nextafter(x, np.inf),
                  float(rng.uniform(-100, 100))):
            assert oracle.floor_div(float(v), h) == math.floor(Fr(float(v)) / Fr(h))
    # cases where x / h rounds up to an integer but the exact quotient is below
    assert oracle.floor_div(0.3, 0.1) == 2
    assert math.floor(0.3 / 0.1) == 2 and oracle.floor_div(3 * 0.1, 0.1) == 3


def test_exact_sum_and_mean():
    rng = np.random.default_rng(12)
    for _ in range(200):
        v = rng.normal(0, 1, 50) * 10.0 ** rng.integers(-8, 8, 50)
        w = rng.integers(1, 1000, 50).astype(np.uint32)
        want = float(sum(Fr(float(a)) * int(b) for a, b in zip(v, w)))
        assert oracle.exact_sum(v, w) == want
        assert oracle.exact_sum(v) == math.fsum(v)
        D = int(rng.integers(1, 2 ** 31))
        assert oracle.exact_mean(v, D) == float(sum(Fr(float(a)) for a in v) / D)
    # cancellation and ties to even
    assert oracle.exact_sum([1e300, 1.0, -1e300]) == 1.0
    assert oracle.exact_sum([2.0 ** 53, 1.0]) == 2.0 ** 53
    assert oracle.exact_sum([2.0 ** 53, 1.0, 2.0 ** -60]) == 2.0 ** 53 + 2


# ---------------------------------------------------------------------------
# GridShift-based tracking (Sec. 2.3, Algorithm 2): the window step R and the
# tracker loop of the oracle, against exact rational arithmetic and closed
# forms.

def _cell(c, h):
    return [math.floor(Fraction(float(v)) / Fraction(float(h))) for v in c]


def _window_brute(frame, W, H, h, bins, rect):
    """R by exact rationals: count, sums, extent, present."""
    x0, y0 = max(rect[0], 0), max(rect[1], 0)
    x1, y1 = min(rect[2], W), min(rect[3], H)
    keys = [tuple(b) for b in np.asarray(bins, dtype=np.int64).tolist()]
    present = [0] * len(keys)
    xs, ys = [], []
    for y in range(y0, y1):
        for x in range(x0, x1):
            kc = tuple(_cell(frame[y * W + x], h))
            hit = False
            for j, b in enumerate(keys):
                if b == kc:
                    present[j] = 1
                    hit = True
            if hit:
                xs.append(x)
                ys.append(y)
    return xs, ys, present


def test_track_window_hand_example():
    # 4 x 3 frame, one channel, value of pixel (x, y) = 4 y + x; h = 2, so the
    # cell of a value v is floor(v / 2).  B = {1, 4}: cell 1 holds values 2, 3
    # (pixels (2,0), (3,0)), cell 4 holds 8, 9 (pixels (0,2), (1,2)).  R is
    # those four pixels: sum x = 2+3+0+1 = 6, sum y = 0+0+2+2 = 4, mean
    # (1.5, 1.0), x extent 0..3, y extent 0..2, both cells present.
    frame = np.arange(12, dtype=np.float64).reshape(12, 1)
    r, present = oracle.track_window(frame, 4, 3, 2.0, [[1], [4]], (0, 0, 4, 3))
    assert (r["count"], r["sum_x"], r["sum_y"]) == (4, 6, 4)
    assert (r["mean_x"], r["mean_y"]) == (1.5, 1.0)
    assert (r["min_x"], r["max_x"], r["min_y"], r["max_y"]) == (0, 3, 0, 2)
    assert present.tolist() == [1, 1]
    # the window x in [1, 3), y in [0, 3) keeps (2,0) and (1,2) only; cell 6
    # (values 12, 13) holds no pixel
    r, present = oracle.track_window(frame, 4, 3, 2.0, [[1], [4], [6]], (1, 0, 3, 3))
    assert (r["count"], r["sum_x"], r["sum_y"]) == (2, 3, 2)
    assert present.tolist() == [1, 1, 0]


def test_track_window_whole_frame_closed_form():
    # B = every cell of the frame and the window = the frame: R is every
    # pixel, whose mean position is the frame's centre ((W-1)/2, (H-1)/2)
    rng = np.random.default_rng(5)
    W, H, h = 13, 9, 7.5
    frame = rng.uniform(-50, 50, size=(W * H, 3))
    B = np.unique(np.array([_cell(c, h) for c in frame], dtype=np.int64), axis=0)
    r, present = oracle.track_window(frame, W, H, h, B, (-5, -5, W + 5, H + 5))
    assert r["count"] == W * H
    assert (r["mean_x"], r["mean_y"]) == ((W - 1) / 2, (H - 1) / 2)
    assert (r["min_x"], r["max_x"], r["min_y"], r["max_y"]) == (0, W - 1, 0, H - 1)
    assert present.all()
    # an empty B, or a window outside the frame, gives an empty R
    r, present = oracle.track_window(frame, W, H, h, np.zeros((0, 3), np.int64), (0, 0, W, H))
    assert r["count"] == 0 and math.isnan(r["mean_x"]) and r["min_x"] > r["max_x"]
    r, present = oracle.track_window(frame, W, H, h, B, (W, 0, W + 4, H))
    assert r["count"] == 0 and not present.any()


@pytest.mark.parametrize("seed", range(4))
def test_track_window_against_exact_rationals(seed):
    rng = np.random.default_rng(100 + seed)
    W, H, d = int(rng.integers(5, 14)), int(rng.integers(5, 14)), int(rng.integers(1, 4))
    h = float(rng.uniform(3, 12))
    frame = np.rint(rng.uniform(0, 60, size=(W * H, d))) + (rng.random((W * H, d)) < 0.3) * 0.5
    cells = np.array([_cell(c, h) for c in frame], dtype=np.int64)
    B = cells[rng.choice(len(cells), size=6)]
    B = np.concatenate([B, B[:2], [[999] * d]])  # duplicates and an absent cell
    rect = (int(rng.integers(-3, W)), int(rng.integers(-3, H)), 0, 0)
    rect = (rect[0], rect[1], rect[0] + int(rng.integers(0, W + 4)), rect[1] + int(rng.integers(0, H + 4)))
    r, present = oracle.track_window(frame, W, H, h, B, rect)
    xs, ys, pres = _window_brute(frame, W, H, h, B, rect)
    assert r["count"] == len(xs) and r["sum_x"] == sum(xs) and r["sum_y"] == sum(ys)
    if xs:
        assert r["mean_x"] == sum(xs) / len(xs) and r["mean_y"] == sum(ys) / len(ys)
        assert (r["min_x"], r["max_x"], r["min_y"], r["max_y"]) == (min(xs), max(xs), min(ys), max(ys))
    assert present.tolist() == pres
