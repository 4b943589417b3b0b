"""The one-to-one label agreement used to state how closely the float32 path
reproduces the float64 result (host code, no GPU)."""
from __future__ import annotations

import numpy as np

from paper_2206_02200_gb300 import agreement


def test_renaming_is_full_agreement():
    rng = np.random.default_rng(0)
    ref = rng.integers(0, 7, 1000)
    perm = rng.permutation(7)
    ag = agreement.agreement(perm[ref], ref)
    assert ag["labels"] == 1.0 and ag["k"] == ag["k_ref"] == 7 and ag["matched"] == 7


def test_split_clusters_lose_their_pieces():
    # every reference cluster split in two halves: the best-overlap measure
    # would still say 1.0; the one-to-one matching keeps one half of each
    ref = np.repeat(np.arange(4), 100)
    ours = np.repeat(np.arange(8), 50)
    ag = agreement.agreement(ours, ref)
    assert ag["labels"] == 0.5
    assert ag["k"] == 8 and ag["k_ref"] == 4 and ag["matched"] == 4


def test_merged_clusters_lose_the_smaller_part():
    ref = np.array([0] * 60 + [1] * 30 + [2] * 10)
    ours = np.array([0] * 90 + [1] * 10)
    ag = agreement.agreement(ours, ref)
    assert ag["labels"] == 0.7
    pairs, ov = agreement.match_clusters(ours, ref)
    assert pairs == [(0, 0), (1, 2)] and ov == [60, 10]


def test_greedy_takes_the_largest_overlap_first():
    ref = np.array([0] * 5 + [1] * 5)
    ours = np.array([0] * 6 + [1] * 4)
    pairs, ov = agreement.match_clusters(ours, ref)
    assert pairs == [(0, 0), (1, 1)] and ov == [5, 4]


def test_modes_compared_on_matched_pairs_only():
    ref = np.array([0, 0, 1, 1, 1])
    ours = np.array([1, 1, 0, 0, 0])
    ref_modes = np.array([[0.0, 0.0], [10.0, 10.0]])
    modes = np.array([[10.0, 10.5], [0.25, 0.0]])
    ag = agreement.agreement(ours, ref, modes, ref_modes, h=2.0)
    assert ag["labels"] == 1.0
    assert ag["max_mode_error_h"] == 0.25


def test_empty():
    ag = agreement.agreement(np.array([], dtype=np.int32), np.array([], dtype=np.int32))
    assert ag["labels"] == 1.0 and ag["k"] == ag["k_ref"] == 0
