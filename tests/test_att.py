"""The OpenFst / AT&T text format (Sec. 6: the paper's implementations read
it): the worked example of Figs. 1-2 written as text, round trips of random
FSTs, and the inputs the reader must refuse."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import att, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fig1_text():
    """Figs. 1-2 as AT&T text with symbol tables, built from the golden arrays."""
    with open(os.path.join(GOLDEN, "fig1.json")) as fh:
        g = json.load(fh)
    R = g["R"]
    lines = []
    for a in range(len(R) - 1):
        for k in range(R[a], R[a + 1]):
            cost = -np.log(g["P"][k]) + 0.0
            lines.append(f"{g['S'][k]} {g['T'][k]} {g['input_symbols'][a]} {g['O'][k]} {cost:.9g}")
    for s, p in g["final_states"].items():
        lines.append(f"{s} {-np.log(p) + 0.0:.9g}")
    isyms = "\n".join(["<eps> 0"] + [f"{s} {i + 1}" for i, s in enumerate(g["input_symbols"])])
    osyms = "\n".join(["<eps> 0"] + [f"{s} {i + 1}" for i, s in enumerate(g["output_symbols"])])
    return "\n".join(lines) + "\n", isyms, osyms, g


def test_fig1_text_decodes_as_the_paper_says():
    text, isyms_txt, osyms_txt, g = _fig1_text()
    isyms, osyms = att.read_symbols(isyms_txt), att.read_symbols(osyms_txt)
    fa = att.read_att(text, isyms, osyms)
    assert fa.num_states == g["num_states"]
    assert list(fa.src) == g["S"] and list(fa.dst) == g["T"]
    assert np.isfinite(fa.start_weight).sum() == 1 and fa.start_weight[g["start_state"]] == 0
    o = oracle.Fst(fa)
    x = att.encode(g["input"], isyms)
    v = o.viterbi(x)
    assert list(v["path"]) == g["expected"]["viterbi_arcs"]
    inv = {i: s for s, i in osyms.items()}
    assert [inv[int(k)] for k in v["olabels"]] == g["expected"]["viterbi_output"]
    assert abs(np.exp(float(v["best"])) - g["expected"]["viterbi_probability"]) < 1e-6
    assert abs(np.exp(o.forward_backward(x)["logz"]) - g["expected"]["total_weight_Z"]) < 1e-6


def _canon(fa):
    key = np.lexsort((fa.weight, fa.olabel, fa.ilabel, fa.dst, fa.src))
    return [a[key] for a in (fa.src, fa.dst, fa.ilabel, fa.olabel, fa.weight)]


def test_round_trip_random_fsts():
    rng = np.random.default_rng(3)
    for _ in range(40):
        fa = synth.tiny_fst(rng, multi_start=False)
        if not (fa.src == 0).any() and not np.isfinite(fa.final_weight[0]):
            with pytest.raises(ValueError, match="no line can name it"):
                att.write_att(fa)  # a start state with no arcs and no final weight
            continue
        text = att.write_att(fa)
        fb = att.read_att(text, num_isyms=fa.num_isyms, num_states=fa.num_states)
        for a, b in zip(_canon(fa), _canon(fb)):
            assert np.array_equal(a, b)
        assert np.array_equal(fa.start_weight, fb.start_weight)
        assert np.array_equal(fa.final_weight, fb.final_weight)
        # the first line names the start state
        assert int(text.split()[0]) == int(np.flatnonzero(np.isfinite(fa.start_weight))[0])
        x = rng.integers(0, fa.num_isyms, size=4).astype(np.int32)
        oa, ob = oracle.Fst(fa), oracle.Fst(fb)
        assert oa.viterbi(x)["best"] == ob.viterbi(x)["best"]
        assert oa.forward_backward(x)["logz"] == pytest.approx(ob.forward_backward(x)["logz"], rel=1e-12, abs=0)


def test_acceptor_and_default_weights():
    fa = att.read_att("0 1 2\n1 2 3 0.5\n2\n", acceptor=True)
    assert list(fa.ilabel) == [2, 3] and list(fa.olabel) == [2, 3]
    assert list(fa.weight) == [0.0, 0.5] and fa.final_weight[2] == 0.0
    assert fa.num_isyms == 4 and fa.num_states == 3


@pytest.mark.parametrize("text,kw,msg", [
    ("0 1 0 1 0.5\n1\n", dict(epsilon=0), "epsilon"),
    ("0 1 <eps> a\n1\n", dict(isyms={"<eps>": 0, "a": 1}, osyms={"<eps>": 0, "a": 1}), "epsilon"),
    ("0 1 b a\n1\n", dict(isyms={"a": 1}, osyms={"a": 1}), "not in the symbol table"),
    ("0 1 2\n", {}, "expected"),
    ("0 1 2 3 nan\n", {}, "not a cost"),
    ("0 -1 2 3\n", {}, "negative state"),
    ("x 1 2 3\n", {}, "not an integer"),
    ("", {}, "empty"),
])
def test_rejected_inputs(text, kw, msg):
    with pytest.raises(ValueError, match=msg):
        att.read_att(text, **kw)


def test_writer_refuses_what_the_format_cannot_hold():
    fa = synth.fig1_fst()
    fa.start_weight[1] = 0.0  # two start states
    with pytest.raises(ValueError, match="one start state"):
        att.write_att(fa)
