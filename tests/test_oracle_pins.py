"""The CPU oracle against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(lib, pin):
    pin(lib)


def test_batch_matches_single(lib):
    fst, strs = synth.make_config("c2", scale=0.004, strings=12)
    o = oracle.Fst(fst, lib)
    vb = o.viterbi_batch(strs.ids, strs.offsets, nthreads=3)
    fbb = o.fb_batch(strs.ids, strs.offsets, nthreads=4)
    fb1 = o.fb_batch(strs.ids, strs.offsets, nthreads=1)
    tot = np.zeros(o.A)
    for b in range(strs.count):
        x = strs.get(b)
        v = o.viterbi(x)
        assert v["best"] == vb["best"][b]
        assert np.array_equal(v["path"], vb["paths"][strs.offsets[b]:strs.offsets[b + 1]])
        f = o.forward_backward(x)
        assert f["logz"] == fbb["logz"][b]
        tot += f["counts"]
    assert np.allclose(tot, fbb["counts"], rtol=1e-12, atol=1e-12)
    assert np.allclose(fb1["counts"], fbb["counts"], rtol=1e-12, atol=1e-12)


def test_weighted_batch_counts(lib):
    fst, strs = synth.make_config("c1", scale=0.1, strings=5)
    o = oracle.Fst(fst, lib)
    w = np.array([0.5, -1.0, 2.0, 0.0, 3.0])
    fb = o.fb_batch(strs.ids, strs.offsets, nthreads=2, weights=w)
    ref = sum(w[b] * o.forward_backward(strs.get(b))["counts"] for b in range(strs.count))
    assert np.allclose(fb["counts"], ref, atol=1e-12)


def test_invalid_inputs_rejected(lib):
    fst = synth.fig1_fst()
    o = oracle.Fst(fst, lib)
    with pytest.raises(RuntimeError):
        o.viterbi(np.array([0, 7], np.int32))  # symbol out of range
    fst.weight[2] = np.nan
    with pytest.raises(RuntimeError):
        oracle.Fst(fst, lib).viterbi(np.array([0], np.int32))


def test_no_path_status(lib):
    fst = synth.fig1_fst()
    o = oracle.Fst(fst, lib)
    v = o.viterbi(np.array([1, 1], np.int32))
    assert v["status"] == oracle.NO_PATH and np.all(v["path"] == -1)
    fb = o.forward_backward(np.array([1, 1], np.int32))
    assert fb["status"] == oracle.NO_PATH and fb["logz"] == -np.inf
    assert np.all(fb["counts"] == 0)
