"""Parity at the benchmark's full size: the 20M-arc workload (200,000 states,
20,000 symbols, 4,096 strings of length 5..200) run the way bench.py runs
it (a Viterbi plan and a forward-backward plan on two streams), checked on
sampled strings against the oracle one by one, and through properties that
hold at any size for the batch sums."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_logz_close, assert_viterbi_equal, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_c3_full_size_sampled_parity():
    import torch
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c3")
    f = Fst.from_arrays(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    plan_v = f.plan(ids, off, mem_budget=48 << 30, flags=PLAN_NO_FB)
    plan_f = f.plan(ids, off, mem_budget=48 << 30, flags=PLAN_NO_VITERBI)
    assert plan_v.info()["waves"] == 1 and plan_f.info()["waves"] == 1
    s_v, s_f = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    plan_v.viterbi(stream=s_v)
    plan_f.forward_backward(stream=s_f)
    torch.cuda.synchronize()
    sc = plan_v.scores.cpu().numpy()
    pa = plan_v.paths.cpu().numpy()
    ol = plan_v.olabels.cpu().numpy()
    st = plan_v.status.cpu().numpy()
    lz = plan_f.logz.cpu().numpy()
    cnt = plan_f.counts.cpu().numpy().astype(np.float64)
    assert (st[:strs.count] == 0).all()  # random walks that end in a final state all have a path

    o = oracle.Fst(fa)
    lens = np.diff(strs.offsets)
    rng = np.random.default_rng(7)
    picks = sorted(set([int(np.argmax(lens)), int(np.argmin(lens))] + list(rng.choice(strs.count, 4, replace=False))))
    for b in picks:
        lo, hi = strs.offsets[b], strs.offsets[b + 1]
        x = strs.get(b)
        assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], o.viterbi(x))
        assert_logz_close(lz[b], o.forward_backward(x)["logz"])

    # batch sums: at every position of a string with a path the posteriors of
    # the slice's arcs sum to 1, so the counts sum to the number of tokens
    assert (cnt >= 0).all()
    total = float(cnt.sum())
    want = float(lens.sum())
    assert abs(total - want) <= 1e-5 * want, (total, want)
    # arcs whose symbol occurs in no string have no count
    used = np.zeros(fa.num_isyms, bool)
    used[strs.ids] = True
    assert (cnt[~used[fa.ilabel]] == 0).all()


def _sampled(strs, k, seed):
    lens = np.diff(strs.offsets)
    rng = np.random.default_rng(seed)
    return sorted(set([int(np.argmax(lens))] + list(rng.choice(strs.count, k, replace=False))))


def test_c2_full_size_plain_sampled():
    # 50,000 states, 10,000 symbols, 5,000,000 arcs; the plain method, one
    # string at a time (one launch per position)
    from paper_1701_03038_gb300.fst import Fst
    from gpu_util import assert_counts_close
    fa, strs = synth.make_config("c2")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    for b in _sampled(strs, 4, 21):
        x = strs.get(b)
        score, path, olab, st = f.viterbi(x)
        assert_viterbi_equal(score, path, olab, st, o.viterbi(x))
        lz, cnt, _ = f.forward_backward(x)
        ofb = o.forward_backward(x)
        assert_logz_close(lz, ofb["logz"])
        assert_counts_close(cnt, ofb["counts"])


def _batch_sampled_parity(cfg, picks_k, seed):
    import torch
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config(cfg)
    f = Fst.from_arrays(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    plan_v = f.plan(ids, off, flags=PLAN_NO_FB)
    plan_f = f.plan(ids, off, flags=PLAN_NO_VITERBI)
    plan_v.viterbi()
    plan_f.forward_backward()
    torch.cuda.synchronize()
    sc, pa, ol, st = (plan_v.scores.cpu().numpy(), plan_v.paths.cpu().numpy(), plan_v.olabels.cpu().numpy(),
                      plan_v.status.cpu().numpy())
    lz = plan_f.logz.cpu().numpy()
    cnt = plan_f.counts.cpu().numpy().astype(np.float64)
    o = oracle.Fst(fa)
    for b in _sampled(strs, picks_k, seed):
        lo, hi = strs.offsets[b], strs.offsets[b + 1]
        x = strs.get(b)
        assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], o.viterbi(x))
        assert_logz_close(lz[b], o.forward_backward(x)["logz"])
    lens = np.diff(strs.offsets)
    ok = np.isfinite(lz[:strs.count])
    want = float(lens[ok].sum())
    assert (cnt >= 0).all() and abs(float(cnt.sum()) - want) <= 1e-5 * want


def test_c4_full_size_batch_sampled():
    # the training workload: 100,000 states, 5,000 symbols, 2,000,000 arcs,
    # 1,024 strings of length 10..100
    _batch_sampled_parity("c4", 4, 23)


def test_c5_full_size_batch_sampled():
    # 1,000,000 states, 5,000 symbols, 100,000,000 arcs, 64 strings of 1,000
    _batch_sampled_parity("c5", 2, 25)
