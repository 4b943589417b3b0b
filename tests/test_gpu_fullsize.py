"""Full-size parity with the oracle on the two largest image configurations:
the 3840x2160 gradient image (d = 5, h = 10) and the batch of 64 uneven
images (d = 3, h = 16, 47,465,008 pixels).  FP64: bit-identical labels,
iteration counts and float64 modes (Sec. 2.1, Eq. 1-4; exact sums rounded
once).  FP32 mixed: clusters matched one to one cover at least 99.9% of the
points, the cluster counts agree and matched modes lie within 1e-3 h.

The oracle runs in a spawn-method process pool over the host's cores while
the GPU works (about a minute of host time for the batch, 20-30 s for the 4K
image)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2206_02200_gb300 import agreement, gridshift, synth
from tests import oracle_workers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AGREE = 0.999
MODE_TOL = 1e-3
BATCH_SEED0 = 1000  # the seeds of the 64-image batch workload


@pytest.fixture(scope="module")
def oracle_results():
    """The oracle's results for the 4K image and every batch instance, computed
    in a process pool while the tests run."""
    p = oracle_workers.pool()
    big = p.apply_async(oracle_workers.workload, ("image_4k_d5",))
    items = p.map_async(oracle_workers.batch_item,
                        [(i, BATCH_SEED0, 16.0, 50) for i in range(64)])
    p.close()
    got = {}

    def get(name):
        if name not in got:
            got[name] = big.get() if name == "4k" else items.get()
        return got[name]

    yield get
    p.terminate()
    p.join()


def _fit(X, h, prec):
    pts = torch.from_numpy(X).cuda()
    with gridshift.GridShift(X.shape[1], h, 50, precision=prec) as g:
        labels, modes, info = g.fit(pts)
        torch.cuda.synchronize()
    return labels.cpu().numpy(), modes.cpu().numpy(), info


@pytest.fixture(scope="module")
def image_4k():
    return synth.WORKLOADS["image_4k_d5"]()


@pytest.fixture(scope="module")
def batch64():
    w = synth.WORKLOADS["batch_64_d3"]()
    parts = w["parts"]
    offsets = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).tolist()
    return parts, offsets


def _fit_batched(parts, offsets, prec):
    X = np.ascontiguousarray(np.concatenate(parts, 0))
    with gridshift.GridShift(3, 16.0, 50, precision=prec) as g:
        labels, modes, infos = g.fit_batched(torch.from_numpy(X).cuda(), offsets)
        torch.cuda.synchronize()
    return labels.cpu().numpy(), [m.cpu().numpy() for m in modes], infos


def test_image_4k_fp64_bit_identical(image_4k, oracle_results):
    lab, md, info = _fit(image_4k["points"], image_4k["h"], gridshift.GS_FP64)
    ref = oracle_results("4k")
    assert info["k"] == ref["k"] and info["iterations"] == ref["iterations"]
    assert info["m0"] == ref["m0"] and info["inexact"] == 0
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(md[:ref["k"]].view(np.int64), ref["modes"].view(np.int64))


def test_image_4k_fp32(image_4k, oracle_results):
    lab, md, info = _fit(image_4k["points"], image_4k["h"], gridshift.GS_FP32_MIXED)
    ref = oracle_results("4k")
    ag = agreement.agreement(lab, ref["labels"], md, ref["modes"], image_4k["h"])
    print(f"4K fp32 against the oracle: {ag}")
    assert ag["labels"] >= AGREE and ag["max_mode_error_h"] <= MODE_TOL, ag
    assert info["k"] == ref["k"], (info["k"], ref["k"])


def test_batch64_fp64_every_instance_bit_identical(batch64, oracle_results):
    parts, offsets = batch64
    lab, modes, infos = _fit_batched(parts, offsets, gridshift.GS_FP64)
    refs = oracle_results("batch")
    for b, ref in enumerate(refs):
        assert infos[b]["k"] == ref["k"] and infos[b]["iterations"] == ref["iterations"], b
        assert infos[b]["m0"] == ref["m0"] and infos[b]["converged"] == int(ref["converged"]), b
        np.testing.assert_array_equal(lab[offsets[b]:offsets[b + 1]], ref["labels"])
        np.testing.assert_array_equal(modes[b].view(np.int64), ref["modes"].view(np.int64))


def test_batch64_fp32_every_instance(batch64, oracle_results):
    parts, offsets = batch64
    lab, modes, infos = _fit_batched(parts, offsets, gridshift.GS_FP32_MIXED)
    refs = oracle_results("batch")
    worst = 1.0
    for b, ref in enumerate(refs):
        ag = agreement.agreement(lab[offsets[b]:offsets[b + 1]], ref["labels"], modes[b],
                                 ref["modes"], 16.0)
        worst = min(worst, ag["labels"])
        assert ag["labels"] >= AGREE and ag["max_mode_error_h"] <= MODE_TOL, (b, ag)
        assert infos[b]["k"] == ref["k"], (b, infos[b]["k"], ref["k"])
    print(f"batch fp32: worst instance label agreement {worst:.6f}")
