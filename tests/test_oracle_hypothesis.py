"""Property-based pins of the oracle: generated tiny point sets (dyadic and
general values, negative coordinates, points on cell faces, repeated points)
must give bit for bit what the independent Fraction brute forces give, for
the parallel update (Eq. 6) and the sequential one (Eq. 5).  Derandomised, so
every run checks the same examples."""
from __future__ import annotations

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import oracle  # noqa: E402
from tests.test_oracle_pins import brute_force  # noqa: E402
from tests.test_oracle_sequential import brute_force_sequential  # noqa: E402

_coord = st.one_of(
    st.integers(-24, 24).map(lambda k: k / 4.0),  # dyadic: many values on faces
    st.floats(-6.0, 6.0, allow_nan=False, allow_infinity=False, width=64),
)


@st.composite
def point_sets(draw):
    d = draw(st.integers(1, 3))
    n = draw(st.integers(1, 24))
    pts = [[draw(_coord) for _ in range(d)] for _ in range(n)]
    if n > 2 and draw(st.booleans()):
        pts[-1] = list(pts[0])  # a repeated point
    h = draw(st.sampled_from([1.0, 0.75, 2.5, 0.5]))
    max_iter = draw(st.sampled_from([0, 1, 3, 50]))
    return np.array(pts, dtype=np.float64), h, max_iter


def _same(r, b) -> bool:
    return (r["iterations"] == b["iterations"] and r["converged"] == b["converged"]
            and r["m_hist"].tolist() == b["m_hist"] and np.array_equal(r["labels"], b["labels"])
            and np.array_equal(r["keys"], b["keys"])
            and np.array_equal(r["counts"].astype(np.int64), b["counts"])
            and np.array_equal(r["modes"], b["modes"]))


_SETTINGS = settings(max_examples=120, derandomize=True, deadline=None, database=None)


@_SETTINGS
@given(point_sets())
def test_parallel_form_matches_brute_force(case):
    X, h, max_iter = case
    assert _same(oracle.fit(X, h, max_iter), brute_force(X, h, max_iter))


@_SETTINGS
@given(point_sets())
def test_sequential_form_matches_brute_force(case):
    X, h, max_iter = case
    assert _same(oracle.fit(X, h, max_iter, update="sequential"),
                 brute_force_sequential(X, h, max_iter))
