"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The FP64 path forms every sum exactly and rounds once, as the oracle does, so
the expected result is bit-identical: the same labels (canonical numbering by
ascending final cell key), the same iteration count and the same float64
modes.  The tolerance the FP64 path is held to is the partition up to renaming
and modes within 1e-10 * h; both are asserted, and bit-identity is asserted on
top of it.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle
from paper_2206_02200_gb300 import gridshift, synth
from tests import golden_io

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu_fit(X, h, max_iter=50, as_f32=False, stream=None):
    dev = torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    if as_f32:
        t = t.float()
    with torch.cuda.stream(stream) if stream is not None else _null():
        labels, modes, info = gridshift.fit(t, h, max_iter)
        torch.cuda.current_stream().synchronize()
    return labels.cpu().numpy(), modes.cpu().numpy(), info


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def _same_partition(a, b) -> bool:
    """True if label arrays a and b describe the same partition (up to renaming)."""
    if a.shape != b.shape:
        return False
    if a.size == 0:
        return True
    pairs = np.unique(np.stack([a, b], 1), axis=0)
    return (len(pairs) == len(np.unique(a)) == len(np.unique(b)))


def check_parity(X, h, max_iter=50, as_f32=False, stream=None):
    Xo = X.astype(np.float32).astype(np.float64) if as_f32 else X
    ref = oracle.fit(Xo, h, max_iter)
    lab, md, info = _gpu_fit(X, h, max_iter, as_f32=as_f32, stream=stream)
    assert info["k"] == ref["k"]
    assert info["m0"] == ref["m0"]
    assert info["iterations"] == ref["iterations"]
    assert bool(info["converged"]) == ref["converged"]
    assert info["inexact"] == 0
    # the stated tolerance: same partition, modes within 1e-10 h
    assert _same_partition(lab, ref["labels"])
    assert md.shape == ref["modes"].shape
    if md.size:
        assert np.max(np.abs(md - ref["modes"])) <= 1e-10 * h
    # what exact arithmetic gives: bit-identical labels and modes
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(md.view(np.int64), ref["modes"].view(np.int64))
    return ref, info


# ---------------------------------------------------------------------------
# hand-worked examples


@pytest.mark.parametrize("case", golden_io.all_cases(), ids=lambda c: c["name"])
def test_golden_cases_on_gpu(case):
    X = case["points"]
    lab, md, info = _gpu_fit(X, case["h"], case.get("max_iter", 50))
    assert list(lab) == case["labels"]
    assert info["iterations"] == case["iterations"]
    for r, row in enumerate(case["modes"]):
        for a, v in enumerate(row):
            assert abs(md[r, a] - float(v)) <= 4 * np.spacing(abs(float(v)))
    check_parity(X, case["h"], case.get("max_iter", 50))


# ---------------------------------------------------------------------------
# random inputs: every dimension, ragged sizes, negative coordinates


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n", [1, 7, 1000, 33_333])
def test_random_blobs(d, n):
    rng = np.random.default_rng(1000 * d + n)
    centres = rng.uniform(-40, 40, size=(5, d))
    X = centres[rng.integers(0, 5, n)] + rng.normal(0, 3.0, size=(n, d))
    check_parity(X, 4.0)


@pytest.mark.parametrize("seed", range(6))
def test_uniform_noise_many_cells(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5000, 60000))
    d = int(rng.integers(1, 5))
    X = rng.uniform(-100, 100, size=(n, d))
    check_parity(X, float(rng.uniform(2, 9)))


@pytest.mark.parametrize("d,n,side", [(3, 60_000, 25.0), (4, 60_000, 12.0), (5, 60_000, 12.0),
                                        (6, 60_000, 6.0), (7, 15_000, 4.0), (8, 12_000, 3.0)])
def test_pencil_first_step(d, n, side):
    # enough level-0 cells (>= 4096) for the two-pass form of the first update,
    # dense enough that most neighbourhoods are full, with edges on every axis
    rng = np.random.default_rng(77 + d)
    X = rng.uniform(0.0, side, size=(n, d))
    X[: n // 4] = rng.normal(3.0, 0.7, size=(n // 4, d))
    check_parity(X, 1.0, max_iter=8)


@pytest.mark.parametrize("seed", [0, 2])
def test_long_runs_label_by_pointer_jumping(seed):
    # more than 16 update steps: labels through pointer jumping rather than a
    # walk of the chain of merges
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.normal(0, 30, size=(3000, 2)), rng.normal(100, 30, size=(3000, 2))])
    ref, _ = check_parity(X, 2.0)
    assert ref["iterations"] > 16


def test_unaligned_input():
    # points starting 8 bytes (float64) or 4 bytes (float32) past a 16-byte
    # boundary take the scalar load paths
    rng = np.random.default_rng(77)
    X = rng.normal(0, 6, size=(20001, 3))
    ref = oracle.fit(X, 2.0, 50)
    for dt, Xd in ((torch.float64, X), (torch.float32, X.astype(np.float32))):
        buf = torch.empty(X.size + 1, dtype=dt, device="cuda")
        pts = buf[1:].view(X.shape)
        pts.copy_(torch.from_numpy(np.ascontiguousarray(Xd)))
        assert pts.data_ptr() % 16 != 0
        labels, modes, info = gridshift.fit(pts, 2.0, 50)
        torch.cuda.synchronize()
        exp = ref if dt == torch.float64 else oracle.fit(Xd.astype(np.float64), 2.0, 50)
        np.testing.assert_array_equal(labels.cpu().numpy(), exp["labels"])
        np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64),
                                      exp["modes"].view(np.int64))


def test_binning_table_regrows():
    # about one cell per point: far more cells than a fresh context's first
    # binning table holds (n / 32 + 65536), so binning overflows and the
    # table grows, twice, before the loop kernel runs
    rng = np.random.default_rng(31)
    X = rng.uniform(0, 4000, size=(600_000, 2))
    ref = oracle.fit(X, 1.0, 10)
    assert ref["m0"] > 400_000
    g = gridshift.GridShift(2, 1.0, 10)
    labels, modes, info = g.fit(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert info["m0"] == ref["m0"] and info["k"] == ref["k"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64), ref["modes"].view(np.int64))
    # the same context on a small input afterwards
    check_ctx_reuse(g)
    g.close()


def test_float32_input():
    X = synth.gmm_points(200_000, 6, 40, seed=9)
    ref, _ = check_parity(X.astype(np.float64), 4.0)
    lab, md, info = _gpu_fit(X, 4.0, as_f32=True)
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(md.view(np.int64), ref["modes"].view(np.int64))


@pytest.mark.parametrize("max_iter", [0, 1, 2, 3])
def test_max_iter_cap(max_iter):
    X = synth.image_features(synth.voronoi_image(120, 160, 9, 8.0, seed=4))
    ref, info = check_parity(X, 16.0, max_iter)
    assert info["iterations"] <= max_iter


def test_small_images_span_tiles_and_ragged_tails():
    for (H, W, R, seed) in [(37, 53, 3, 1), (97, 131, 7, 2), (250, 333, 15, 3)]:
        img = synth.voronoi_image(H, W, R, 10.0, seed=seed, gradient=0.02)
        check_parity(synth.image_features(img, xy_scale=0.1), 10.0)
        check_parity(synth.image_features(img), 16.0)


# ---------------------------------------------------------------------------
# full-size workloads


def test_image_321x481_d3_full():
    w = synth.WORKLOADS["image_321x481_d3"]()
    check_parity(w["points"], w["h"], w["max_iter"])


def test_image_1080p_d5_full():
    w = synth.WORKLOADS["image_1080p_d5"]()
    check_parity(w["points"], w["h"], w["max_iter"])


def test_gmm_1M_d6():
    X = synth.gmm_points(1_000_000, 6, 200, seed=5)
    check_parity(X, 4.0, 50, as_f32=True)


# ---------------------------------------------------------------------------
# more clusters than the loop kernel numbers itself (16384): the final cells
# are numbered by a radix sort of their keys instead


def _lattice_pairs(side: int, with_partner: bool):
    """side x side sites 4 cells apart; with_partner adds a point in the next
    cell along axis 0, so each pair merges in one update."""
    i, j = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    base = np.stack([4.0 * i.ravel() + 0.5, 4.0 * j.ravel() + 0.5], 1)
    if not with_partner:
        return base
    return np.concatenate([base, base + np.array([1.0, 0.0])], 0)


def test_many_clusters_numbered_by_sort():
    X = _lattice_pairs(150, with_partner=False)          # 22500 isolated cells, 0 updates
    ref, info = check_parity(X, 1.0)
    assert ref["k"] == 22500 and ref["iterations"] == 0
    X = _lattice_pairs(150, with_partner=True)           # 45000 cells merge into 22500
    ref, info = check_parity(X, 1.0)
    assert ref["k"] == 22500 and ref["iterations"] == 1


def test_cluster_count_at_the_numbering_threshold():
    for side in (127, 128, 129):                         # k = 16129, 16384, 16641
        ref, info = check_parity(_lattice_pairs(side, with_partner=True), 1.0)
        assert ref["k"] == side * side


# ---------------------------------------------------------------------------
# edge cases and errors


def test_empty_and_single_point():
    lab, md, info = _gpu_fit(np.zeros((0, 3)), 1.0)
    assert lab.shape == (0,) and md.shape == (0, 3) and info["k"] == 0
    check_parity(np.array([[1.5, -2.25, 3.0]]), 1.0)


def test_identical_points_and_exact_faces():
    check_parity(np.full((5000, 2), 3.0), 1.0)          # all on one face corner
    X = np.repeat(np.arange(0, 20, 1.0)[:, None], 3, axis=1)
    check_parity(X, 1.0)                                 # every point on a face


def test_nonfinite_input_is_rejected():
    g = gridshift.GridShift(2, 1.0, 10)
    for bad in (np.nan, -np.nan, np.inf, -np.inf):
        X = np.zeros((100, 2))
        X[37, 1] = bad
        with pytest.raises(gridshift.GridShiftError) as e:
            g.fit(torch.from_numpy(X).cuda())
        assert e.value.status == gridshift.GS_E_INVALID
    # every value non-finite (a NaN whose bits are all ones, both signs)
    for bits in (0x7FFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF):
        X = np.full((64, 2), bits, dtype=np.uint64).view(np.float64)
        with pytest.raises(gridshift.GridShiftError) as e:
            g.fit(torch.from_numpy(X).cuda())
        assert e.value.status == gridshift.GS_E_INVALID
    # the context stays usable
    check_ctx_reuse(g)
    g.close()


def test_nonfinite_float32_input_is_rejected():
    # float32 input: the key range reads the values in their own width
    g = gridshift.GridShift(3, 1.0, 10)
    for bad in (np.nan, -np.nan, np.inf, -np.inf):
        X = np.zeros((1001, 3), dtype=np.float32)
        X[500, 2] = bad
        with pytest.raises(gridshift.GridShiftError) as e:
            g.fit(torch.from_numpy(X).cuda())
        assert e.value.status == gridshift.GS_E_INVALID
    for bits in (0x7FFFFFFF, 0xFFFFFFFF):
        X = np.full((33, 3), bits, dtype=np.uint32).view(np.float32)
        with pytest.raises(gridshift.GridShiftError) as e:
            g.fit(torch.from_numpy(X).cuda())
        assert e.value.status == gridshift.GS_E_INVALID
    g.close()


@pytest.mark.parametrize("as_f32", [False, True], ids=["f64", "f32"])
@pytest.mark.parametrize("aligned", [True, False], ids=["aligned", "unaligned"])
def test_key_range_signs_zeros_and_tiny_values(as_f32, aligned):
    # signed zeros, negative and positive values, and float32 subnormals: the
    # per-axis extremes (order codes, largest magnitude) set the packing and
    # the fixed-point window; an unaligned array takes the one-value-per-load
    # reads of the key range and binning
    rng = np.random.default_rng(71)
    n, d = 4099, 3
    X = rng.normal(0.0, 3.0, size=(n, d))
    X[::7, 0] = 0.0
    X[1::7, 0] = -0.0
    X[2::5, 1] = -X[2::5, 1]
    X[:, 2] = rng.uniform(-1e-36, 1e-36, size=n)  # cells 0 and -1, a fine fixed-point unit
    X[::3, 2] = rng.uniform(-1e-38, 1e-38, size=len(X[::3, 2]))  # float32 subnormals
    X[::13, 2] = -0.0
    if as_f32:
        X = X.astype(np.float32).astype(np.float64)
    ref = oracle.fit(X, 1.5, 50)
    buf = torch.zeros(n * d + 1, dtype=torch.float32 if as_f32 else torch.float64, device="cuda")
    off = 0 if aligned else 1
    pts = buf[off:off + n * d].view(n, d)
    pts.copy_(torch.from_numpy(X.astype(np.float32) if as_f32 else X))
    labels, modes, info = gridshift.fit(pts, 1.5, 50)
    torch.cuda.synchronize()
    assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64), ref["modes"].view(np.int64))


def check_ctx_reuse(g):
    X = np.random.default_rng(1).normal(0, 5, size=(3000, 2))
    labels, modes, info = g.fit(torch.from_numpy(X).cuda())
    ref = oracle.fit(X, 1.0, 10)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])


def test_key_range_error():
    # 10^15 cells along the axis: more than the packed key's 2^22, so gs_fit
    # takes the wide-key pipeline and still equals the oracle
    X = np.array([[0.0], [1e12]])
    check_parity(X, 1e-3)
    # a batched run keeps the packed key and refuses
    with gridshift.GridShift(1, 1e-3, 50) as g:
        with pytest.raises(gridshift.GridShiftError) as e:
            g.fit_batched(torch.from_numpy(np.concatenate([X, X])).cuda(), [0, 2, 4])
        assert e.value.status == gridshift.GS_E_KEYRANGE
    # |x / h| of 4e15 or more has no exact integer cell on either pipeline
    for Y in (np.array([[0.0], [1e13]]), np.zeros((3, 10))):
        Y = Y.copy()
        Y[-1, 0] = 1e13
        with pytest.raises(gridshift.GridShiftError) as e:
            _gpu_fit(Y, 1e-3)
        assert e.value.status == gridshift.GS_E_KEYRANGE


@pytest.mark.parametrize("d,width", [(1, 200_000.0), (2, 40_000.0)])
def test_face_table_above_device_capacity(d, width):
    # more than 2^16 face-table entries in all: the plan is made on the host
    X = np.random.default_rng(11).uniform(0.0, width, size=(4000, d))
    check_parity(X, 1.0)
    X[:2000] = X[:2000] * 1e-3 + 5.0  # and a dense corner that merges
    check_parity(X, 1.0)


def test_capacity_error_leaves_labels_valid():
    X = synth.image_features(synth.voronoi_image(64, 64, 8, 8.0, seed=3))
    ref = oracle.fit(X, 16.0, 50)
    assert ref["k"] > 1
    g = gridshift.GridShift(3, 16.0, 50)
    pts = torch.from_numpy(X).cuda()
    labels = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    modes = torch.empty((1, 3), dtype=torch.float64, device="cuda")
    st, k, info = g.fit_into(pts, labels, modes)
    torch.cuda.synchronize()
    assert st == gridshift.GS_E_CAPACITY and k == ref["k"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    g.close()


def test_context_reuse_across_sizes_and_streams():
    g = gridshift.GridShift(5, 12.0, 50)
    s = torch.cuda.Stream()
    for (H, W, seed) in [(300, 400, 1), (40, 50, 2), (500, 600, 3), (40, 50, 2)]:
        X = synth.image_features(synth.voronoi_image(H, W, 10, 10.0, seed=seed), xy_scale=0.1)
        ref = oracle.fit(X, 12.0, 50)
        with torch.cuda.stream(s):
            pts = torch.from_numpy(X).cuda()
            labels, modes, info = g.fit(pts)
            s.synchronize()
        np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
        np.testing.assert_array_equal(modes.cpu().numpy().view(np.int64),
                                      ref["modes"].view(np.int64))
    g.close()
