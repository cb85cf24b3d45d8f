"""Batched method (plans: all strings advanced together) against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _dev(strs):
    import torch
    return torch.from_numpy(strs.ids).cuda(), torch.from_numpy(strs.offsets).cuda()


def check_batch_viterbi(o, strs, res):
    sc = res["scores"].cpu().numpy()
    pa = res["paths"].cpu().numpy()
    ol = res["olabels"].cpu().numpy()
    st = res["status"].cpu().numpy()
    ob = o.viterbi_batch(strs.ids, strs.offsets, nthreads=8)
    for b in range(strs.count):
        lo, hi = strs.offsets[b], strs.offsets[b + 1]
        ov = o.viterbi(strs.get(b))
        assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], ov)
        assert sc[b] == ob["best"][b] or (math.isinf(sc[b]) and sc[b] == ob["best"][b])


def check_batch_fb(o, strs, logz, counts, weights=None):
    ob = o.fb_batch(strs.ids, strs.offsets, nthreads=8, weights=weights)
    lz = logz.cpu().numpy()
    for b in range(strs.count):
        assert_logz_close(lz[b], ob["logz"][b])
    if counts is not None:
        assert_counts_close(counts.cpu().numpy(), ob["counts"], batch=True)


@pytest.fixture(scope="module")
def c2s():
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=60)
    return Fst.from_arrays(fa), oracle.Fst(fa), strs


def test_viterbi_batch(c2s):
    f, o, strs = c2s
    ids, off = _dev(strs)
    check_batch_viterbi(o, strs, f.viterbi_batch(ids, off))


def test_forward_backward_batch(c2s):
    f, o, strs = c2s
    ids, off = _dev(strs)
    r = f.forward_backward_batch(ids, off)
    check_batch_fb(o, strs, r["logz"], r["counts"])


@pytest.mark.parametrize("plan", [(0, 0, -1, -1), (2, 3, 0, 0), (2, 3, 1, 1), (1, 4, 1, 0), (3, 2, 0, 1)])
def test_repeated_batch_calls_reuse_storage(c2s, plan):
    # each batch call kind keeps its last plan's storage for the next call
    # (part by part for plans of several parts): a smaller batch reuses it, a
    # larger one replaces it, and results stay those of the oracle either way
    # (the accumulators stay empty between runs); the plans' parts and
    # accumulator layout as fst_set_batch_plan sets them
    import torch
    f, o, strs = c2s
    f.set_batch_plan(*plan)
    # on a side stream (a graph cannot record the legacy default stream)
    side = torch.cuda.Stream()
    subsets = [(0, 60), (10, 30), (0, 60), (25, 60), (0, 7)]
    for b0, b1 in subsets:
        sub = synth.Strings(strs.ids[strs.offsets[b0]:strs.offsets[b1]].copy(),
                            (strs.offsets[b0:b1 + 1] - strs.offsets[b0]).copy())
        ids, off = _dev(sub)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            v = f.viterbi_batch(ids, off, stream=side)
            r = f.forward_backward_batch(ids, off, stream=side)
        side.synchronize()
        check_batch_viterbi(o, sub, v)
        check_batch_fb(o, sub, r["logz"], r["counts"])
    f.set_batch_plan(0, 0, -1, -1)


def test_waves_match_single_wave(c2s):
    import torch
    f, o, strs = c2s
    ids, off = _dev(strs)
    p1 = f.plan(ids, off)
    p2 = f.plan(ids, off, mem_budget=1 << 20)  # forces many waves
    assert p1.info()["waves"] == 1 and p2.info()["waves"] > 2
    for p in (p1, p2):
        p.viterbi()
        p.forward_backward()
    torch.cuda.synchronize()
    # Viterbi is exact whatever the grouping; forward-backward sums in a
    # grouping-dependent order, so both splits are held to the oracle
    assert torch.equal(p1.scores, p2.scores) and torch.equal(p1.paths, p2.paths)
    check_batch_fb(o, strs, p1.logz[:strs.count], p1.counts[:o.A])
    check_batch_viterbi(o, strs, dict(scores=p2.scores[:strs.count], paths=p2.paths[:len(strs.ids)],
                                      olabels=p2.olabels[:len(strs.ids)], status=p2.status[:strs.count]))
    check_batch_fb(o, strs, p2.logz[:strs.count], p2.counts[:o.A])


def test_plain_equals_batched(c2s):
    f, o, strs = c2s
    ids, off = _dev(strs)
    r = f.viterbi_batch(ids, off)
    for b in range(0, strs.count, 7):
        s, p, _, _ = f.viterbi(strs.get(b))
        assert s == r["scores"][b].item()
        assert np.array_equal(p, r["paths"][strs.offsets[b]:strs.offsets[b + 1]].cpu().numpy())


def test_long_segments_batched():
    from paper_1701_03038_gb300.fst import Fst
    rng = np.random.default_rng(21)
    A, m = 4000, 2
    il = rng.integers(0, m, size=A).astype(np.int32)
    w = (rng.random(A) * 3).astype(np.float32)
    fa = synth.FstArrays(1, m, 3, np.zeros(A, np.int32), np.zeros(A, np.int32), il,
                         rng.integers(0, 3, size=A).astype(np.int32), w,
                         np.zeros(1, np.float32), np.zeros(1, np.float32))
    strs = synth.make_strings(fa, 40, 1, 25, seed=4)  # many tokens share a symbol: groups of GMAX
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    check_batch_viterbi(o, strs, f.viterbi_batch(ids, off))
    r = f.forward_backward_batch(ids, off)
    check_batch_fb(o, strs, r["logz"], r["counts"])


def test_split_forward_backward_weighted(c2s):
    import torch
    f, o, strs = c2s
    ids, off = _dev(strs)
    p = f.plan(ids, off, flags=1)  # single wave
    w = torch.linspace(-1.0, 2.0, strs.count, dtype=torch.float32, device="cuda")
    p.forward()
    p.backward(w)
    torch.cuda.synchronize()
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A], weights=w.double().cpu().numpy())


def test_graph_capture_and_replay_after_weight_change(c2s):
    import torch
    from paper_1701_03038_gb300.fst import Fst
    _, _, strs = c2s
    fa, _ = synth.make_config("c2", scale=0.02, strings=1)
    f = Fst.from_arrays(fa)
    ids, off = _dev(strs)
    p = f.plan(ids, off)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p.viterbi(stream=s)
        p.forward_backward(stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.viterbi(stream=s)
        p.forward_backward(stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    o = oracle.Fst(fa)
    check_batch_viterbi(o, strs, dict(scores=p.scores[:strs.count], paths=p.paths[:len(strs.ids)],
                                      olabels=p.olabels[:len(strs.ids)], status=p.status[:strs.count]))
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])
    # new weights, same graph: every run leaves its accumulators zero, so replays stay exact
    rng = np.random.default_rng(8)
    fa.weight = (fa.weight * rng.uniform(0.5, 1.5, size=fa.num_arcs)).astype(np.float32)
    f.set_weights(fa.weight)
    g.replay()
    torch.cuda.synchronize()
    o = oracle.Fst(fa)
    check_batch_viterbi(o, strs, dict(scores=p.scores[:strs.count], paths=p.paths[:len(strs.ids)],
                                      olabels=p.olabels[:len(strs.ids)], status=p.status[:strs.count]))
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])


def test_empty_and_zero_length_strings():
    import torch
    from paper_1701_03038_gb300.fst import Fst
    fa = synth.fig1_fst()
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    strs = synth.Strings(np.array([0, 1, 2, 0, 1, 2], np.int32), np.array([0, 0, 3, 3, 6, 6], np.int64))
    ids, off = _dev(strs)
    check_batch_viterbi(o, strs, f.viterbi_batch(ids, off))
    r = f.forward_backward_batch(ids, off)
    check_batch_fb(o, strs, r["logz"], r["counts"])
    empty = f.viterbi_batch(torch.zeros(0, dtype=torch.int32, device="cuda"),
                            torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert empty["scores"].numel() == 0


def test_iid_strings_no_path_status():
    from paper_1701_03038_gb300.fst import Fst
    fa, _ = synth.make_config("c1", scale=0.2, strings=1)
    strs = synth.make_strings(fa, 30, 10, 30, seed=5, kind="iid")
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    r = f.viterbi_batch(ids, off)
    check_batch_viterbi(o, strs, r)
    assert (r["status"].cpu().numpy() == 2).any()
    rf = f.forward_backward_batch(ids, off)
    check_batch_fb(o, strs, rf["logz"], rf["counts"])


def test_large_groups():
    # few symbols and many strings: most positions have groups of 32 tokens
    # with the same symbol (one window load serves up to 32 strings)
    from paper_1701_03038_gb300.fst import Fst
    fa = synth.random_fst(400, 3, 6, 30000, label_law="zipf", src_law="lognormal", mean_degree=75.0,
                          dirichlet=0.5, seed=31)
    strs = synth.make_strings(fa, 300, 5, 40, seed=32)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    check_batch_viterbi(o, strs, f.viterbi_batch(ids, off))
    r = f.forward_backward_batch(ids, off)
    check_batch_fb(o, strs, r["logz"], r["counts"])


@pytest.mark.parametrize("grid", [0, 1, 7, -1])
def test_persistent_driver_matches_launch_driver(c2s, grid):
    # one cooperative launch per pass with grid barriers between positions:
    # Viterbi bit-identical to the per-position launches, forward-backward
    # held to the oracle; grid 0 = the plan's estimate, -1 = every block that
    # can be co-resident; also over several waves and the split
    # forward / backward calls
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    ref = f.plan(ids, off)
    ref.viterbi()
    torch.cuda.synchronize()
    for budget, flags in ((0, 0), (1 << 20, 0), (0, _lib.PLAN_SINGLE_WAVE)):
        p = f.plan(ids, off, mem_budget=budget, flags=flags)
        g = grid
        if g < 0:
            p.set_driver(_lib.DRIVER_PERSISTENT, 1)
            g = 1
            while True:  # the largest co-resident grid
                try:
                    p.set_driver(_lib.DRIVER_PERSISTENT, g * 2)
                    g *= 2
                except _lib.FstError:
                    break
        p.set_driver(_lib.DRIVER_PERSISTENT, g)
        assert p.driver()[0] == _lib.DRIVER_PERSISTENT
        p.viterbi()
        if flags & _lib.PLAN_SINGLE_WAVE:
            p.forward()
            p.backward()
        else:
            p.forward_backward()
        torch.cuda.synchronize()
        assert torch.equal(p.scores, ref.scores) and torch.equal(p.paths, ref.paths)
        assert torch.equal(p.olabels, ref.olabels) and torch.equal(p.status, ref.status)
        check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])
        info = p.info()
        assert info["viterbi_launches"] == 4 * info["waves"]


def test_autotune_keeps_results_and_caches(c2s, tmp_path, monkeypatch):
    # the autotuner times the plan under every driver configuration and
    # keeps the fastest; results are those of the oracle whatever it picks,
    # and a second plan of the same shapes takes the cached choice
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    p = f.plan(ids, off)
    choice = p.autotune(refresh=True)
    assert choice["driver"] in ("launch", "persistent") and choice["ms"] > 0
    assert (p.driver()[0] == _lib.DRIVER_PERSISTENT) == (choice["driver"] == "persistent")
    p.viterbi()
    p.forward_backward()
    torch.cuda.synchronize()
    check_batch_viterbi(o, strs, dict(scores=p.scores[:strs.count], paths=p.paths[:len(strs.ids)],
                                      olabels=p.olabels[:len(strs.ids)], status=p.status[:strs.count]))
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])
    q = f.plan(ids, off)
    again = q.autotune()
    assert again == choice  # cached: same configuration, same recorded time


@pytest.mark.parametrize("parts", [2, 3, 7])
def test_stream_parallel_parts(c2s, parts):
    # a plan cut into stream-parallel parts: Viterbi bit-identical to the
    # one-part plan, forward-backward held to the oracle, the split forward /
    # backward calls and graph capture work the same, the parts' live work
    # adds up to the whole
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    ref = f.plan(ids, off)
    ref.viterbi()
    ref.forward_backward()
    torch.cuda.synchronize()
    p = f.plan(ids, off, parts=parts)
    info = p.info()
    assert info["strings"] == strs.count and info["relaxations"] == ref.info()["relaxations"]
    p.viterbi()
    p.forward_backward()
    torch.cuda.synchronize()
    assert torch.equal(p.scores, ref.scores) and torch.equal(p.paths, ref.paths)
    assert torch.equal(p.olabels, ref.olabels) and torch.equal(p.status, ref.status)
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])
    assert p.live_work() == ref.live_work()
    # weighted split forward / backward (single-wave parts)
    q = f.plan(ids, off, flags=_lib.PLAN_SINGLE_WAVE, parts=parts)
    w = torch.linspace(-1.0, 2.0, strs.count, dtype=torch.float32, device="cuda")
    q.forward()
    q.backward(w)
    torch.cuda.synchronize()
    check_batch_fb(o, strs, q.logz[:strs.count], q.counts[:o.A], weights=w.double().cpu().numpy())
    # captured and replayed
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.viterbi(stream=s)
        p.forward_backward(stream=s)
    p.scores.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(p.scores, ref.scores)
    check_batch_fb(o, strs, p.logz[:strs.count], p.counts[:o.A])
    # profiles add up over the parts
    p.profile(True)
    p.viterbi()
    torch.cuda.synchronize()
    prof = p.profile_read()
    p.profile(False)
    assert prof["vit_step"][1] > 0
    with pytest.raises(_lib.FstError):
        p.set_driver(_lib.DRIVER_PERSISTENT)


@pytest.mark.parametrize("driver", ["launch", "persistent"])
def test_dense_and_compact_accumulators_agree(c2s, driver):
    # the hash-table accumulators (default) and the dense per-string arrays
    # (FST_PLAN_DENSE_ACC) compute the same quantities: Viterbi bit for bit,
    # log Z bit for bit (exact maxima and fixed-point sums do not depend on
    # the order of the atomics), counts within float64 rounding
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    pc = f.plan(ids, off)
    pd = f.plan(ids, off, flags=_lib.PLAN_DENSE_ACC)
    assert pc.table_slots() >= 1024 and pd.table_slots() == 0
    if driver == "persistent":
        for p in (pc, pd):
            p.set_driver(_lib.DRIVER_PERSISTENT, 0)
    for p in (pc, pd):
        p.viterbi()
        p.forward_backward(states=True)
    torch.cuda.synchronize()
    for k in ("scores", "paths", "olabels", "status", "logz"):
        assert torch.equal(getattr(pc, k), getattr(pd, k)), k
    assert np.allclose(pc.counts.cpu().numpy(), pd.counts.cpu().numpy(), rtol=1e-9, atol=1e-12)
    B, N = strs.count, len(strs.ids)
    check_batch_viterbi(o, strs, dict(scores=pc.scores[:B], paths=pc.paths[:N], olabels=pc.olabels[:N],
                                      status=pc.status[:B]))
    check_batch_fb(o, strs, pc.logz[:B], pc.counts[:o.A])


def test_compact_tables_near_full(c2s):
    # shrinking the tables drives the probe sequences through collisions:
    # each run is exact or, once a position's live states no longer fit,
    # reports FST_ERR_OOM for every string; the exact runs include tables at
    # more than half load
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    B, N = strs.count, len(strs.ids)
    pv = f.plan(ids, off, flags=_lib.PLAN_NO_FB)
    pf = f.plan(ids, off, flags=_lib.PLAN_NO_VITERBI)
    pv.viterbi()
    pf.forward_backward()
    torch.cuda.synchronize()
    ref = {k: getattr(pv, k).clone() for k in ("scores", "paths", "olabels")}
    ref_lz, ref_cnt = pf.logz.clone(), pf.counts.clone()
    cap = pv.table_slots()
    exact, full = [], []
    slots = cap
    while slots >= 2:
        pv.limit_table(slots)
        pf.limit_table(slots)
        pv.viterbi()
        pf.forward_backward()
        torch.cuda.synchronize()
        sv, sf = pv.status[:B].cpu().numpy(), pf.status[:B].cpu().numpy()
        if (sv == _lib.OOM).all():
            assert (sf == _lib.OOM).all() and np.isneginf(pf.logz[:B].cpu().numpy()).all()
            assert (pv.paths[:N].cpu().numpy() == -1).all()
            full.append(slots)
        else:
            for k, v in ref.items():
                assert torch.equal(getattr(pv, k), v), (k, slots)
            assert torch.equal(pf.logz, ref_lz)
            assert np.allclose(pf.counts.cpu().numpy(), ref_cnt.cpu().numpy(), rtol=1e-9, atol=1e-12)
            exact.append(slots)
        slots //= 2
    assert exact and full
    # the smallest exact table is within a factor 2 of overflowing: its
    # busiest position filled more than half of it
    assert min(exact) == 2 * max(full)
    pv.limit_table(0)
    pf.limit_table(0)


@pytest.mark.parametrize("parts", [1, 3])
def test_forward_pull_matches_push(c2s, parts):
    # the direction switch of the forward pass (dense accumulators): with a
    # threshold of 1 every token of a position that has a slot (16) pulls
    # over the destination-ordered slice and the rest push; log Z bit for
    # bit as with every arc pushed, counts and state posteriors within
    # float64 rounding; run twice (the dense vectors must come back to
    # -inf), and in several waves
    import torch
    from paper_1701_03038_gb300 import _lib
    f, o, strs = c2s
    ids, off = _dev(strs)
    B = strs.count
    res = {}
    for name, pull, budget in (("push", 0, 0), ("pull", 1, 0), ("pull_waves", 1, 1 << 21)):
        p = f.plan(ids, off, mem_budget=budget, flags=_lib.PLAN_NO_VITERBI | _lib.PLAN_DENSE_ACC, parts=parts)
        p.set_pull(pull)
        for _ in range(2):
            p.forward_backward(states=True)
            torch.cuda.synchronize()
            res.setdefault(name, []).append((p.logz[:B].clone(), p.counts.clone(), p.start_counts.clone(),
                                             p.final_counts.clone(), p.status[:B].clone()))
        if name == "pull_waves" and parts == 1:
            assert p.info()["waves"] > 1
    ref = res["push"][0]
    for name, runs in res.items():
        for lz, cnt, st, fi, status in runs:
            if name != "pull_waves":
                assert torch.equal(lz, ref[0]), name
            else:
                assert np.allclose(lz.cpu().numpy(), ref[0].cpu().numpy(), rtol=1e-12, atol=1e-9)
            assert torch.equal(status, ref[4])
            for a, b in ((cnt, ref[1]), (st, ref[2]), (fi, ref[3])):
                assert np.allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-9, atol=1e-12), name
    check_batch_fb(o, strs, res["pull"][1][0], res["pull"][1][1][:o.A])
