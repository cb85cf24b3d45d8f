"""Inputs beyond a plain string, on the device: an FST read from OpenFst /
AT&T text (the format the paper's implementations read, Sec. 6), and
acyclic input lattices composed with the FST (Sec. 6.1), against the
oracle's string decoders and its lattice Viterbi / forward-backward."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import att, synth

from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal, ensure_built
import pins
from test_att import _fig1_text

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_att_text_decodes_on_the_device():
    # the worked example of Figs. 1-2 written as AT&T text, read by
    # Fst.from_att and decoded by the kernels: the paper's best path, output
    # "the cat </s>", probability 0.48 and Z = 0.56
    from paper_1701_03038_gb300.fst import Fst
    text, isyms_txt, osyms_txt, g = _fig1_text()
    isyms, osyms = att.read_symbols(isyms_txt), att.read_symbols(osyms_txt)
    f = Fst.from_att(text, isyms, osyms)
    fa = att.read_att(text, isyms, osyms)
    o = oracle.Fst(fa)
    x = att.encode(g["input"], isyms)
    score, path, olab, st = f.viterbi(x)
    assert_viterbi_equal(score, path, olab, st, o.viterbi(x))
    assert list(path) == g["expected"]["viterbi_arcs"]
    inv = {i: s for s, i in osyms.items()}
    assert [inv[int(k)] for k in olab] == g["expected"]["viterbi_output"]
    lz, cnt, _ = f.forward_backward(x)
    assert abs(math.exp(lz) - g["expected"]["total_weight_Z"]) < 1e-6
    assert_counts_close(cnt, o.forward_backward(x)["counts"])
    # random FSTs through a text round trip decode as the originals
    rng = np.random.default_rng(5)
    for _ in range(10):
        fa = synth.tiny_fst(rng, multi_start=False)
        if not (fa.src == 0).any() and not np.isfinite(fa.final_weight[0]):
            continue
        f2 = Fst.from_att(att.write_att(fa))
        o2 = oracle.Fst(att.read_att(att.write_att(fa)))
        for _ in range(3):
            x = rng.integers(0, fa.num_isyms, size=int(rng.integers(0, 6))).astype(np.int32)
            if x.size and x.max() >= f2.num_isyms:
                continue
            s2, p2, ol2, st2 = f2.viterbi(x)
            assert_viterbi_equal(s2, p2, ol2, st2, o2.viterbi(x))


def _check_lattice(f, o, lat):
    args = (lat.N, lat.frm, lat.to, lat.label, lat.weight)
    lv = oracle.lattice_viterbi(o, lat)
    s, edges, arcs, st = f.lattice_viterbi(*args)
    assert st == lv["status"]
    assert np.float32(s) == lv["best"] or (math.isinf(lv["best"]) and s == lv["best"]), (s, lv["best"])
    if st == oracle.OK:
        assert np.array_equal(edges, lv["edges"]) and np.array_equal(arcs, lv["arcs"])
    lfb = oracle.lattice_forward_backward(o, lat)
    lz, cnt, epost, st2 = f.lattice_forward_backward(*args)
    assert st2 == lfb["status"]
    assert_logz_close(lz, lfb["logz"])
    assert_counts_close(cnt, lfb["counts"])
    assert_counts_close(epost, lfb["edge_post"])
    return lv["status"] == oracle.OK


def test_linear_lattices_decode_as_strings():
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=6)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    for b in range(strs.count):
        x = strs.get(b)
        lat = oracle.Lattice.from_string(x)
        s, edges, arcs, st = f.lattice_viterbi(lat.N, lat.frm, lat.to, lat.label, lat.weight)
        s2, p2, _, st2 = f.viterbi(x)
        assert st == st2 and s == s2 and np.array_equal(arcs, p2)
        assert _check_lattice(f, o, lat)


def test_random_lattices_against_the_oracle():
    from paper_1701_03038_gb300.fst import Fst
    rng = np.random.default_rng(41)
    seen = 0
    for _ in range(40):
        fa = synth.tiny_fst(rng, max_states=5, max_arcs=12)
        f, o = Fst.from_arrays(fa), oracle.Fst(fa)
        for _ in range(3):
            seen += _check_lattice(f, o, pins.random_dag(rng, fa.num_isyms, max_nodes=7, max_edges=12))
    assert seen > 20


def test_confusion_networks_on_a_larger_fst():
    # the shape of a recogniser's output: at every position the true symbol
    # (log 0.8) and two alternatives (log 0.1 each) between the same nodes
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=4, seed_offset=11)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    rng = np.random.default_rng(43)
    for b in range(strs.count):
        x = strs.get(b)[:12]
        frm, to, lab, w = [], [], [], []
        for t, a in enumerate(x):
            for alt, p in ((int(a), 0.8), (int(rng.integers(0, fa.num_isyms)), 0.1),
                           (int(rng.integers(0, fa.num_isyms)), 0.1)):
                frm.append(t)
                to.append(t + 1)
                lab.append(alt)
                w.append(math.log(p))
        lat = oracle.Lattice(len(x) + 1, frm, to, lab, np.array(w, np.float32))
        _check_lattice(f, o, lat)


def test_lattice_rejects_bad_edges():
    from paper_1701_03038_gb300._lib import FstError
    from paper_1701_03038_gb300.fst import Fst
    f = Fst.from_arrays(synth.fig1_fst())
    for frm, to, lab, w in (([1], [1], [0], [0.0]), ([0], [5], [0], [0.0]), ([0], [1], [9], [0.0]),
                            ([0], [1], [0], [np.nan])):
        with pytest.raises(FstError):
            f.lattice_viterbi(3, frm, to, lab, w)
        with pytest.raises(FstError):
            f.lattice_forward_backward(3, frm, to, lab, w)


def test_parallel_product_over_time():
    # dense HMMs (every state reaches every state on every symbol): log Z of
    # long strings by the pairwise product tree against the oracle's sweep;
    # the best score equals the oracle's Viterbi score up to the rounding of
    # float32 additions associated in tree order
    from paper_1701_03038_gb300._lib import UNSUPPORTED, FstError
    from paper_1701_03038_gb300.fst import Fst
    rng = np.random.default_rng(47)
    for K, V, n in ((4, 3, 1), (8, 5, 37), (32, 8, 200), (63, 6, 1000)):
        pi = rng.dirichlet(np.ones(K))
        trans = rng.dirichlet(np.ones(K), size=K)
        emit = rng.dirichlet(np.ones(V), size=K)
        fa = synth.hmm_fst(pi, trans, emit)
        f, o = Fst.from_arrays(fa), oracle.Fst(fa)
        for x in (rng.integers(0, V, size=n).astype(np.int32), np.zeros(0, np.int32)):
            lz, best, st = f.prefix_log_z(x)
            want = o.forward_backward(x)
            assert st == want["status"]
            assert_logz_close(lz, want["logz"])
            vb = float(o.viterbi(x)["best"])
            if math.isinf(vb):
                assert best == vb
            else:
                assert abs(float(best) - vb) <= 1e-5 * max(1.0, abs(vb)), (best, vb)
    big, _ = synth.make_config("c1", scale=1.0, strings=1)  # 1,000 states: beyond the dense product
    with pytest.raises(FstError) as ei:
        Fst.from_arrays(big).prefix_log_z(np.zeros(3, np.int32))
    assert ei.value.code == UNSUPPORTED
