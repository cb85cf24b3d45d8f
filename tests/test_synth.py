"""The seeded synthetic workloads match the recipe they stand for: sizes,
label and out-degree laws, weights that are -log of per-state Dirichlet
distributions, one start state, ~10% final states, and random-walk strings
that every FST accepts.  These inputs feed both the oracle and the GPU path,
so a drift here would change every measured figure."""
import numpy as np
import pytest

from paper_1701_03038_gb300 import synth


def test_seeded_and_reproducible():
    a1, s1 = synth.make_config("c2", scale=0.01, strings=20)
    a2, s2 = synth.make_config("c2", scale=0.01, strings=20)
    for x, y in ((a1.src, a2.src), (a1.dst, a2.dst), (a1.ilabel, a2.ilabel), (a1.weight, a2.weight),
                 (s1.ids, s2.ids), (s1.offsets, s2.offsets)):
        assert np.array_equal(x, y)
    b1, _ = synth.make_config("c2", scale=0.01, strings=20, seed_offset=1)
    assert not np.array_equal(a1.weight, b1.weight)


@pytest.mark.parametrize("name,scale", [("c1", 1.0), ("c2", 0.01), ("c3", 0.002), ("c4", 0.01), ("c5", 0.0005)])
def test_sizes_weights_starts_finals(name, scale):
    cfg = synth.CONFIGS[name]
    fa, strs = synth.make_config(name, scale=scale, strings=8)
    q = max(8, int(round(cfg["num_states"] * scale)))
    assert fa.num_states == q
    assert fa.num_arcs == max(16, int(round(cfg["num_arcs"] * scale)))
    for arr, hi in ((fa.src, q), (fa.dst, q), (fa.ilabel, fa.num_isyms), (fa.olabel, fa.num_osyms)):
        assert arr.min() >= 0 and arr.max() < hi
    # costs are -log p with p a distribution over each state's outgoing arcs
    p = np.exp(-fa.weight.astype(np.float64))
    mass = np.bincount(fa.src, weights=p, minlength=q)
    has_out = np.bincount(fa.src, minlength=q) > 0
    assert np.allclose(mass[has_out], 1.0, atol=1e-5)
    # one start state (0, weight 0); about 10% final states with weight 0
    assert np.flatnonzero(np.isfinite(fa.start_weight)).tolist() == [0] and fa.start_weight[0] == 0
    fin = np.isfinite(fa.final_weight)
    assert fin.sum() == max(1, q // 10) or abs(fin.mean() - 0.1) < 0.02
    assert (fa.final_weight[fin] == 0).all()
    lens = np.diff(strs.offsets)
    assert lens.min() >= cfg["len_lo"] and lens.max() <= cfg["len_hi"]


def _accepts(fa, x):
    live = {0}
    for a in x:
        nxt = set()
        for k in np.flatnonzero(fa.ilabel == a):
            if int(fa.src[k]) in live:
                nxt.add(int(fa.dst[k]))
        live = nxt
    return any(np.isfinite(fa.final_weight[q]) for q in live)


def test_walk_strings_are_accepted():
    fa, strs = synth.make_config("c2", scale=0.005, strings=12)
    for b in range(strs.count):
        assert _accepts(fa, strs.get(b))


def test_zipf_labels_follow_rank_order():
    fa, _ = synth.make_config("c2", scale=0.02, strings=1)
    counts = np.bincount(fa.ilabel, minlength=fa.num_isyms)
    # the most frequent symbols are the lowest ranks, with ~1/r frequencies
    assert counts[0] > counts[1] > counts[3] > counts[9]
    ratio = counts[0] / max(counts[9], 1)
    assert 5 < ratio < 20
