"""Parity at the benchmark's full sizes, element by element.

The 20M-arc batching workload (200,000 states, 20,000 symbols, 4,096
strings of length 5..200) runs the way bench.py runs it (a Viterbi plan and
a forward-backward plan on two streams).  The strings checked against the
oracle are chosen where the kernels change regime: the strings with the
largest live frontiers (found on the host by set reachability, which
shares nothing with either side), the longest and shortest strings, and
random ones.  On that sub-batch every string's Viterbi result and log Z is
compared, and the batch's expected counts are compared arc by arc.  The
long-string workload (1,000,000 states, 64 strings of length 1,000) checks
per-string counts over 1,000 positions, and the training workload checks
the full-size gradient through autograd against the oracle's counts.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from frontiers import frontier_table
from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal, ensure_built

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _hard_subbatch(fa, strs, k_hard, k_rand, seed):
    """Indices: the k_hard strings with the largest live frontier, the
    longest and shortest strings, and k_rand random others."""
    mx, _ = frontier_table(fa, strs)
    lens = np.diff(strs.offsets)
    hard = [int(b) for b in np.argsort(-mx, kind="stable")[:k_hard]]
    rng = np.random.default_rng(seed)
    pick = set(hard) | {int(np.argmax(lens)), int(np.argmin(lens))}
    rest = [b for b in range(strs.count) if b not in pick]
    pick |= set(int(b) for b in rng.choice(rest, k_rand, replace=False))
    return sorted(pick), int(mx.max())


def _sub(strs, sel):
    parts = [strs.get(b) for b in sel]
    off = np.zeros(len(sel) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    return synth.Strings(np.concatenate(parts).astype(np.int32), off)


def _run_two_streams(f, strs, budget=0, flags=0, parts=(1, 1), pull=0):
    import torch
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    pv = f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_FB | flags, parts=parts[0])
    pf = f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_VITERBI | flags, parts=parts[1])
    pf.set_pull(pull)
    s_v, s_f = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    pv.viterbi(stream=s_v)
    pf.forward_backward(stream=s_f)
    torch.cuda.synchronize()
    B, N = strs.count, len(strs.ids)
    out = dict(scores=pv.scores[:B].cpu().numpy(), paths=pv.paths[:N].cpu().numpy(),
               olabels=pv.olabels[:N].cpu().numpy(), vstatus=pv.status[:B].cpu().numpy(),
               logz=pf.logz[:B].cpu().numpy(), fstatus=pf.status[:B].cpu().numpy(),
               counts=pf.counts.cpu().numpy().astype(np.float64))
    return out


def _check_strings(o, strs, sel, res, ov_cache=None):
    """Viterbi and log Z of strings ``sel`` of ``strs`` against the oracle."""
    ob = o.fb_batch(np.concatenate([strs.get(b) for b in sel]).astype(np.int32),
                    np.concatenate([[0], np.cumsum([len(strs.get(b)) for b in sel])]).astype(np.int64),
                    nthreads=THREADS, counts=False)
    for i, b in enumerate(sel):
        lo, hi = strs.offsets[b], strs.offsets[b + 1]
        ov = ov_cache[b] if ov_cache is not None and b in ov_cache else o.viterbi(strs.get(b))
        if ov_cache is not None:
            ov_cache[b] = ov
        assert_viterbi_equal(res["scores"][b], res["paths"][lo:hi], res["olabels"][lo:hi], res["vstatus"][b], ov)
        assert_logz_close(res["logz"][b], ob["logz"][i])


def test_c3_full_size_hard_strings_elementwise():
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c3")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    from paper_1701_03038_gb300._lib import PLAN_DENSE_ACC
    sel, biggest = _hard_subbatch(fa, strs, 24, 22, seed=7)
    assert biggest >= 100_000  # the sample reaches the hub regime
    # the whole batch, as the benchmark runs it (dense accumulators, 2 + 8
    # stream-parallel parts), with the forward pass's direction switch at
    # half the states: the hub tokens pull
    full = _run_two_streams(f, strs, budget=48 << 30, flags=PLAN_DENSE_ACC, parts=(2, 8), pull=-1)
    assert (full["vstatus"] == 0).all() and (full["fstatus"] == 0).all()
    # and with compact accumulators, every arc pushed: the same exact maxima
    # and fixed-point sums, so Viterbi and log Z agree bit for bit on all
    # 4,096 strings
    other = _run_two_streams(f, strs)
    for k in ("scores", "paths", "olabels", "vstatus", "logz", "fstatus"):
        assert np.array_equal(full[k], other[k]), k
    assert np.allclose(full["counts"], other["counts"], rtol=1e-9, atol=1e-9)
    del other
    cache = {}
    _check_strings(o, strs, sel, full, cache)
    # whole-batch properties: at every position of a string the posteriors of
    # the slice's arcs sum to 1, so the counts sum to the number of tokens;
    # arcs whose symbol occurs in no string have no count
    lens = np.diff(strs.offsets)
    cnt = full["counts"]
    assert (cnt >= 0).all()
    assert abs(float(cnt.sum()) - float(lens.sum())) <= 1e-5 * float(lens.sum())
    used = np.zeros(fa.num_isyms, bool)
    used[strs.ids] = True
    assert (cnt[~used[fa.ilabel]] == 0).all()
    # the sub-batch as a batch of its own: every string, and the counts arc by arc
    sub = _sub(strs, sel)
    res = _run_two_streams(f, sub)
    _check_strings(o, sub, list(range(sub.count)), res, {i: cache[b] for i, b in enumerate(sel)})
    ob = o.fb_batch(sub.ids, sub.offsets, nthreads=THREADS)
    assert_counts_close(res["counts"], ob["counts"], batch=True)


def test_c2_full_size_plain_sampled():
    # 50,000 states, 10,000 symbols, 5,000,000 arcs; the plain method, one
    # string at a time (one launch per position), on the strings with the
    # largest frontiers and random ones
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    sel, _ = _hard_subbatch(fa, strs, 4, 3, seed=21)
    for b in sel:
        x = strs.get(b)
        score, path, olab, st = f.viterbi(x)
        assert_viterbi_equal(score, path, olab, st, o.viterbi(x))
        lz, cnt, _ = f.forward_backward(x)
        ofb = o.forward_backward(x)
        assert_logz_close(lz, ofb["logz"])
        assert_counts_close(cnt, ofb["counts"])


def test_c4_full_size_gradient_elementwise():
    # the training workload (100,000 states, 5,000 symbols, 2,000,000 arcs,
    # strings of length 10..100): d sum_b log Z_b / d theta through autograd
    # on a 64-string sub-batch, arc by arc against the oracle's counts
    import torch
    from paper_1701_03038_gb300._lib import PLAN_SINGLE_WAVE
    from paper_1701_03038_gb300.autograd import LogZModule
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c4")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    sel, _ = _hard_subbatch(fa, strs, 32, 30, seed=23)
    sub = _sub(strs, sel)
    plan = f.plan(torch.from_numpy(sub.ids).cuda(), torch.from_numpy(sub.offsets).cuda(), flags=PLAN_SINGLE_WAVE)
    theta0 = -torch.from_numpy(fa.weight.astype(np.float32))
    mod = LogZModule(f, theta0)
    lz = mod(plan)
    lz.sum().backward()
    torch.cuda.synchronize()
    ob = o.fb_batch(sub.ids, sub.offsets, nthreads=THREADS)
    for i in range(sub.count):
        assert_logz_close(lz[i].item(), ob["logz"][i])
    assert_counts_close(mod.theta.grad.cpu().numpy(), ob["counts"], batch=True)
    # the same with unequal string weights g_b (the incoming gradient)
    mod.theta.grad = None
    g = torch.linspace(0.25, 2.0, sub.count, dtype=torch.float64, device="cuda")
    (mod(plan) * g).sum().backward()
    ow = o.fb_batch(sub.ids, sub.offsets, nthreads=THREADS, weights=g.cpu().numpy())
    assert_counts_close(mod.theta.grad.cpu().numpy(), ow["counts"], batch=True)


def test_c5_full_size_per_string_counts():
    # 1,000,000 states, 5,000 symbols, 100,000,000 arcs, strings of 1,000:
    # per-string counts summed over 1,000 positions (the compensated
    # accumulation of the single-string call) within 1e-5 absolute, and the
    # batch path's Viterbi and log Z on every string of a sub-batch
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c5")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    for b in (0, 17):
        x = strs.get(b)
        lz, cnt, st = f.forward_backward(x)
        ofb = o.forward_backward(x)
        assert st == ofb["status"] == 0
        assert_logz_close(lz, ofb["logz"])
        assert_counts_close(cnt, ofb["counts"])
        score, path, olab, vst = f.viterbi(x)
        assert_viterbi_equal(score, path, olab, vst, o.viterbi(x))
    # the oracle keeps (n+1) x Q float64 tables per string in flight (16 GB
    # here), so it runs two strings at a time
    sel = list(range(0, 64, 16))
    sub = _sub(strs, sel)
    res = _run_two_streams(f, sub)
    ob = o.fb_batch(sub.ids, sub.offsets, nthreads=2)
    for i in range(sub.count):
        lo, hi = sub.offsets[i], sub.offsets[i + 1]
        assert_viterbi_equal(res["scores"][i], res["paths"][lo:hi], res["olabels"][lo:hi], res["vstatus"][i],
                             o.viterbi(sub.get(i)))
        assert_logz_close(res["logz"][i], ob["logz"][i])
    assert_counts_close(res["counts"], ob["counts"], batch=True)
