"""Plain method (one string, one launch per position) against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal, ensure_built
import pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _fst(fa):
    from paper_1701_03038_gb300.fst import Fst
    return Fst.from_arrays(fa)


def check_string(f, o, x, fb=True):
    s, p, ol, rc = f.viterbi(x)
    assert_viterbi_equal(s, p, ol, rc, o.viterbi(x))
    if fb:
        lz, cnt, rc2 = f.forward_backward(x)
        ofb = o.forward_backward(x)
        assert rc2 == ofb["status"]
        assert_logz_close(lz, ofb["logz"])
        assert_counts_close(cnt, ofb["counts"])


def test_fig1_worked_example():
    fa, x, exp, exp_out, post = pins.fig1_case()
    f = _fst(fa)
    s, p, ol, rc = f.viterbi(x)
    assert rc == 0 and list(p) == exp["viterbi_arcs"] and list(ol) == exp_out
    assert s == np.float32(math.log(exp["viterbi_probability"]))
    lz, cnt, _ = f.forward_backward(x)
    assert abs(lz - math.log(exp["total_weight_Z"])) < 1e-6
    assert np.allclose(cnt, post, atol=1e-6)


def test_tiny_random_fsts():
    rng = np.random.default_rng(123)
    for _ in range(150):
        fa = synth.tiny_fst(rng)
        f, o = _fst(fa), oracle.Fst(fa)
        for _ in range(2):
            x = rng.integers(0, fa.num_isyms, size=int(rng.integers(0, 7))).astype(np.int32)
            check_string(f, o, x)


def test_c1_full_size():
    fa, strs = synth.make_config("c1", strings=6)
    f, o = _fst(fa), oracle.Fst(fa)
    for b in range(strs.count):
        check_string(f, o, strs.get(b))


def test_single_state_long_segments():
    # one state: every slice is one segment, far longer than a 128-arc window
    rng = np.random.default_rng(5)
    A, m = 5000, 3
    il = rng.integers(0, m, size=A).astype(np.int32)
    w = (rng.random(A) * 4).astype(np.float32)
    fa = synth.FstArrays(1, m, 4, np.zeros(A, np.int32), np.zeros(A, np.int32), il,
                         rng.integers(0, 4, size=A).astype(np.int32), w,
                         np.zeros(1, np.float32), np.zeros(1, np.float32))
    f, o = _fst(fa), oracle.Fst(fa)
    for n in (1, 2, 7, 30):
        check_string(f, o, rng.integers(0, m, size=n).astype(np.int32))


def test_hub_states_mix_long_and_short_segments():
    rng = np.random.default_rng(9)
    q, m, A = 300, 4, 20000
    src = rng.integers(0, q, size=A).astype(np.int32)
    dst = rng.integers(0, q, size=A).astype(np.int32)
    hub = rng.random(A) < 0.3
    dst[hub] = rng.integers(0, 3, size=int(hub.sum()))   # three hub destinations
    src[rng.random(A) < 0.2] = 7                          # a hub source (long backward segments)
    il = rng.integers(0, m, size=A).astype(np.int32)
    w = (rng.random(A) * 5).astype(np.float32)
    w[rng.random(A) < 0.05] = 1.0                         # exact ties
    start = np.full(q, np.inf, np.float32); start[:3] = [0.0, 0.5, 1.0]
    final = np.where(rng.random(q) < 0.2, 0.0, np.inf).astype(np.float32); final[0] = 0.25
    fa = synth.FstArrays(q, m, 5, src, dst, il, rng.integers(0, 5, size=A).astype(np.int32), w, start, final)
    f, o = _fst(fa), oracle.Fst(fa)
    strs = synth.make_strings(fa, 5, 5, 40, seed=3)
    for b in range(strs.count):
        check_string(f, o, strs.get(b))


def test_c2_scaled():
    fa, strs = synth.make_config("c2", scale=0.02, strings=25)
    f, o = _fst(fa), oracle.Fst(fa)
    for b in range(strs.count):
        check_string(f, o, strs.get(b))


def test_no_path_and_empty_string():
    fa, _ = synth.make_config("c1", scale=0.2, strings=1)
    f, o = _fst(fa), oracle.Fst(fa)
    iid = synth.make_strings(fa, 6, 20, 40, seed=77, kind="iid")
    seen_nopath = False
    for b in range(iid.count):
        x = iid.get(b)
        check_string(f, o, x)
        seen_nopath |= o.viterbi(x)["status"] == oracle.NO_PATH
    assert seen_nopath
    check_string(f, o, np.zeros(0, np.int32))


def test_symbol_without_arcs():
    fa = synth.fig1_fst()
    fa.num_isyms = 5  # symbols 3 and 4 have no arcs
    f, o = _fst(fa), oracle.Fst(fa)
    for x in ([0, 1, 2], [3], [0, 4, 2], []):
        check_string(f, o, np.array(x, np.int32))


def test_repeatable_bitwise():
    fa, strs = synth.make_config("c2", scale=0.01, strings=3)
    f = _fst(fa)
    x = strs.get(0)
    a = f.viterbi(x)
    b = f.viterbi(x)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    la, ca, _ = f.forward_backward(x)
    lb, cb, _ = f.forward_backward(x)
    assert la == lb and np.array_equal(ca, cb)


def test_posteriors_into_caller_buffer():
    # forward_backward(out=...) writes the counts into the caller's array
    # (here the numpy view of a pinned tensor, reused): the same values as a
    # fresh array, for the frontier kernels and the one-block kernels
    import torch
    from paper_1701_03038_gb300 import _lib
    fa, strs = synth.make_config("c2", scale=0.01, strings=3)
    f = _fst(fa)
    buf = torch.full((fa.num_arcs + 5,), 7.0, dtype=torch.float32).pin_memory().numpy()
    for method in (_lib.PLAIN_FRONTIER, _lib.PLAIN_BLOCK):
        f.set_plain_method(method)
        for b in range(strs.count):
            x = strs.get(b)
            la, ca, ra = f.forward_backward(x)
            lb, cb, rb = f.forward_backward(x, out=buf)
            assert la == lb and ra == rb and np.array_equal(ca, cb)
            assert np.shares_memory(cb, buf) and np.array_equal(buf[:fa.num_arcs], ca)
    for bad in (np.zeros(fa.num_arcs - 1, np.float32), np.zeros(fa.num_arcs, np.float64),
                np.zeros((2, fa.num_arcs), np.float32)[:, 0]):
        with pytest.raises(ValueError):
            f.forward_backward(strs.get(0), out=bad)


def test_invalid_inputs():
    from paper_1701_03038_gb300._lib import FstError
    from paper_1701_03038_gb300.fst import Fst
    fa = synth.fig1_fst()
    f = _fst(fa)
    with pytest.raises(FstError):
        f.viterbi(np.array([0, 9], np.int32))
    bad = synth.fig1_fst()
    bad.weight[1] = np.nan
    with pytest.raises(FstError):
        Fst.from_arrays(bad)
    bad = synth.fig1_fst()
    bad.dst[0] = 6
    with pytest.raises(FstError):
        Fst.from_arrays(bad)
    bad = synth.fig1_fst()
    bad.weight[0] = -np.inf  # cost -inf = theta +inf
    with pytest.raises(FstError):
        Fst.from_arrays(bad)


def test_store_info_and_symbol_stats():
    fa, _ = synth.make_config("c2", scale=0.01, strings=1)
    f = _fst(fa)
    info = f.info()
    arcs, dsts, srcs = f.symbol_stats()
    assert info["num_arcs"] == fa.num_arcs and arcs.sum() == fa.num_arcs
    want_arcs = np.bincount(fa.ilabel, minlength=fa.num_isyms)
    assert np.array_equal(arcs, want_arcs)
    pairs_d = np.unique(fa.ilabel.astype(np.int64) * fa.num_states + fa.dst)
    pairs_s = np.unique(fa.ilabel.astype(np.int64) * fa.num_states + fa.src)
    assert np.array_equal(dsts, np.bincount(pairs_d // fa.num_states, minlength=fa.num_isyms))
    assert np.array_equal(srcs, np.bincount(pairs_s // fa.num_states, minlength=fa.num_isyms))
    assert info["padded_arcs"] % 128 == 0 and info["padded_arcs"] >= fa.num_arcs


def test_shorter_strings_after_longer_on_one_handle():
    # frontier tags of one call must never be mistaken for those of the next
    fa, _ = synth.make_config("c2", scale=0.01, strings=1)
    f, o = _fst(fa), oracle.Fst(fa)
    for n in (60, 45, 30, 12, 5, 2, 1, 33):
        x = synth.make_strings(fa, 1, n, n, seed=100 + n).get(0)
        check_string(f, o, x)


def test_slice_relaxation_is_bit_identical():
    # the paper's relaxation (every arc of every slice, one thread per arc)
    # against the oracle and the frontier-driven plain path
    rng = np.random.default_rng(19)
    cases = [(synth.fig1_fst(), [np.array([0, 1, 2], np.int32), np.array([2], np.int32), np.zeros(0, np.int32)])]
    for _ in range(6):
        fa = synth.tiny_fst(rng)
        cases.append((fa, [rng.integers(0, fa.num_isyms, size=int(rng.integers(0, 7))).astype(np.int32)
                           for _ in range(4)]))
    fa, strs = synth.make_config("c2", scale=0.02, strings=6)
    cases.append((fa, [strs.get(b) for b in range(strs.count)]))
    for fa, xs in cases:
        f, o = _fst(fa), oracle.Fst(fa)
        for x in xs:
            ov = o.viterbi(x)
            s1, p1, st = f.viterbi_slice(x)
            assert st == ov["status"]
            assert s1 == ov["best"] or (np.isinf(ov["best"]) and s1 == ov["best"])
            if ov["status"] == 0:
                assert np.array_equal(p1, ov["path"])
                s2, p2, _, _ = f.viterbi(x)
                assert s1 == s2 and np.array_equal(p1, p2)



def test_slice_orders_and_paper_forward_backward():
    # the paper's design, both arc orders within a slice (by destination /
    # column-major, by source / row-major): Viterbi bit-identical to the
    # oracle; the float32 atomic log-add forward-backward (Eq. 3) within
    # 1e-5 of log Z, its posteriors within the looser bound that float32
    # values without rescaling can keep over these lengths
    from paper_1701_03038_gb300 import _lib
    rng = np.random.default_rng(23)
    cases = [(synth.fig1_fst(), [np.array([0, 1, 2], np.int32), np.zeros(0, np.int32)])]
    for _ in range(6):
        fa = synth.tiny_fst(rng)
        cases.append((fa, [rng.integers(0, fa.num_isyms, size=int(rng.integers(0, 7))).astype(np.int32)
                           for _ in range(4)]))
    fa, strs = synth.make_config("c1", scale=1.0, strings=2)
    cases.append((fa, [strs.get(b) for b in range(strs.count)]))
    fa, strs = synth.make_config("c2", scale=0.02, strings=4)
    cases.append((fa, [strs.get(b) for b in range(strs.count)]))
    worst = 0.0
    for fa, xs in cases:
        f, o = _fst(fa), oracle.Fst(fa)
        for order in (_lib.SLICE_BY_DESTINATION, _lib.SLICE_BY_SOURCE):
            f.set_slice_order(order)
            for x in xs:
                ov = o.viterbi(x)
                s1, p1, st = f.viterbi_slice(x)
                assert st == ov["status"]
                assert s1 == ov["best"] or (np.isinf(ov["best"]) and s1 == ov["best"])
                if st == 0:
                    assert np.array_equal(p1, ov["path"])
                ofb = o.forward_backward(x)
                lz, cnt, st2 = f.forward_backward_slice(x)
                assert st2 == ofb["status"]
                assert_logz_close(lz, ofb["logz"])
                err = float(np.abs(cnt.astype(np.float64) - ofb["counts"]).max()) if fa.num_arcs else 0.0
                worst = max(worst, err)
                assert err <= 5e-4, (order, err)
    print(f"paper forward-backward: largest posterior error {worst:.2e}")
    with pytest.raises(_lib.FstError):
        f.set_slice_order(2)


def test_plain_viterbi_methods_agree():
    # fst_viterbi through the frontier kernels, the slice-wide kernel, and the
    # calibrated automatic choice: the same score, path and output labels
    from paper_1701_03038_gb300 import _lib
    fa, strs = synth.make_config("c2", scale=0.02, strings=12)
    f, o = _fst(fa), oracle.Fst(fa)
    iid = synth.make_strings(fa, 4, 5, 20, seed=3, kind="iid")
    xs = [strs.get(b) for b in range(strs.count)] + [iid.get(b) for b in range(iid.count)] + [np.zeros(0, np.int32)]
    for method in (_lib.PLAIN_SLICE, _lib.PLAIN_FRONTIER):
        f.set_plain_method(method)
        for x in xs:
            s, p, ol, st = f.viterbi(x)
            assert_viterbi_equal(s, p, ol, st, o.viterbi(x))
    coef = f.autotune_plain(strs.ids, strs.offsets)
    assert coef.shape == (5,) and np.isfinite(coef).all()
    for x in xs:
        s, p, ol, st = f.viterbi(x)
        assert_viterbi_equal(s, p, ol, st, o.viterbi(x))
    with pytest.raises(_lib.FstError):
        f.set_plain_method(7)


@pytest.mark.parametrize("grid", [0, 1, 5])
def test_plain_forward_backward_persistent_driver(grid):
    # one cooperative launch per pass for a single string (grid 0 = one block
    # per SM): log Z and posteriors against the oracle, as the launch driver
    from paper_1701_03038_gb300 import _lib
    fa, strs = synth.make_config("c2", scale=0.02, strings=8)
    f, o = _fst(fa), oracle.Fst(fa)
    f.set_plain_driver(_lib.DRIVER_PERSISTENT, grid)
    f.set_plain_method(_lib.PLAIN_FRONTIER)
    iid = synth.make_strings(fa, 2, 5, 15, seed=9, kind="iid")
    for x in [strs.get(b) for b in range(strs.count)] + [iid.get(0), np.zeros(0, np.int32)]:
        s, p, ol, vst = f.viterbi(x)  # the frontier Viterbi under the same driver
        assert_viterbi_equal(s, p, ol, vst, o.viterbi(x))
        lz, cnt, st = f.forward_backward(x)
        ofb = o.forward_backward(x)
        assert st == ofb["status"]
        assert_logz_close(lz, ofb["logz"])
        assert_counts_close(cnt, ofb["counts"])
    f.set_plain_driver(_lib.DRIVER_LAUNCH)
    coef = f.autotune_plain(strs.ids, strs.offsets)  # also picks the driver
    for b in range(3):
        x = strs.get(b)
        lz, cnt, st = f.forward_backward(x)
        assert_logz_close(lz, o.forward_backward(x)["logz"])
    with pytest.raises(_lib.FstError):
        f.set_plain_driver(_lib.DRIVER_PERSISTENT, 10 ** 7)


def test_block_method_small_fsts():
    # the one-block kernels (position loop inside the kernel, per-state values
    # in shared memory): Viterbi bit-identical to the frontier kernels, log Z
    # and posteriors against the oracle, on the plain tests' small FSTs
    from paper_1701_03038_gb300 import _lib
    rng = np.random.default_rng(321)
    cases = []
    fa, x, _, _, _ = pins.fig1_case()
    cases.append((fa, [x, np.zeros(0, np.int32)]))
    for _ in range(40):
        fa = synth.tiny_fst(rng)
        cases.append((fa, [rng.integers(0, fa.num_isyms, size=int(rng.integers(0, 7))).astype(np.int32)
                           for _ in range(2)]))
    fa, strs = synth.make_config("c1", strings=4)
    cases.append((fa, [strs.get(b) for b in range(strs.count)]))
    fa, strs = synth.make_config("c2", scale=0.02, strings=10)  # 1,000 states, 100,000 arcs
    iid = synth.make_strings(fa, 3, 5, 20, seed=5, kind="iid")  # some without a path
    cases.append((fa, [strs.get(b) for b in range(strs.count)] + [iid.get(b) for b in range(iid.count)]))
    A, m = 5000, 3  # one state, slices far longer than the block
    il = rng.integers(0, m, size=A).astype(np.int32)
    fa = synth.FstArrays(1, m, 4, np.zeros(A, np.int32), np.zeros(A, np.int32), il,
                         rng.integers(0, 4, size=A).astype(np.int32), (rng.random(A) * 4).astype(np.float32),
                         np.zeros(1, np.float32), np.zeros(1, np.float32))
    cases.append((fa, [rng.integers(0, m, size=n).astype(np.int32) for n in (1, 7, 30)]))
    fa = synth.fig1_fst()
    fa.num_isyms = 5  # symbols without arcs
    cases.append((fa, [np.array(v, np.int32) for v in ([0, 1, 2], [3], [0, 4, 2])]))
    # 5,000 states: the Viterbi backtrace rows of a 6-position string fit in
    # shared memory, those of a 40-position one do not
    fa, _ = synth.make_config("c2", scale=0.1, strings=1)
    walks = synth.make_strings(fa, 2, 6, 6, seed=11, kind="walk")
    longw = synth.make_strings(fa, 2, 40, 40, seed=12, kind="walk")
    cases.append((fa, [walks.get(0), walks.get(1), longw.get(0), longw.get(1)]))
    for fa, xs in cases:
        f, o = _fst(fa), oracle.Fst(fa)
        f.set_plain_method(_lib.PLAIN_FRONTIER)
        ref = [f.viterbi(x) for x in xs]
        f.set_plain_method(_lib.PLAIN_BLOCK)
        for x, r in zip(xs, ref):
            s, p, ol, st = f.viterbi(x)
            assert s == r[0] and np.array_equal(p, r[1]) and np.array_equal(ol, r[2]) and st == r[3]
            check_string(f, o, x)
    # repeatable bit for bit, and the calibration picks it on c1
    fa, strs = synth.make_config("c1", strings=6)
    f = _fst(fa)
    f.set_plain_method(_lib.PLAIN_BLOCK)
    la, ca, _ = f.forward_backward(strs.get(0))
    lb, cb, _ = f.forward_backward(strs.get(0))
    assert la == lb and np.array_equal(ca, cb)
    f.set_plain_method(_lib.PLAIN_AUTO)
    assert f.plain_method()["method"] == _lib.PLAIN_FRONTIER  # not calibrated yet
    coef = f.autotune_plain(strs.ids, strs.offsets)
    # coefficients all zero exactly when the calibration took the block kernels
    assert (f.plain_method()["method"] == _lib.PLAIN_BLOCK) == (not np.any(coef))
    o = oracle.Fst(fa)
    for b in range(strs.count):
        check_string(f, o, strs.get(b))
    for m in (_lib.PLAIN_FRONTIER, _lib.PLAIN_SLICE, _lib.PLAIN_BLOCK):
        f.set_plain_method(m)
        assert f.plain_method()["method"] == m
    f.set_plain_driver(_lib.DRIVER_PERSISTENT, 4)
    assert f.plain_method() == {"method": _lib.PLAIN_BLOCK, "driver": _lib.DRIVER_PERSISTENT, "grid_blocks": 4}
    # beyond the shared-memory limit the method is refused
    big, _ = synth.make_config("c2", scale=0.2, strings=1)  # 10,000 states
    assert big.num_states > _lib.BLOCK_MAX_STATES
    with pytest.raises(_lib.FstError) as ei:
        _fst(big).set_plain_method(_lib.PLAIN_BLOCK)
    assert ei.value.code == _lib.UNSUPPORTED
