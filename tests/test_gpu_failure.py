"""Failure paths of the batched method, made on the host (no GPU fault).

A run whose live pool overflows must report FST_ERR_OOM for every string of
its wave, write the no-result markers, and leave the plan usable: the next
run on the same plan clears what the overflowing one left behind and is
exact again.  The overflow is forced by capping the pool
(fst_plan_limit_pool), which allocates nothing and touches no memory out of
bounds.
"""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_pool_overflow_reports_oom_then_recovers():
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=24)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    pv = f.plan(ids, off, flags=PLAN_NO_FB)
    pf = f.plan(ids, off, flags=PLAN_NO_VITERBI | _lib.PLAN_DENSE_ACC)
    pf.set_pull(1)  # the forward pass's dense vectors must survive an overflowed run
    B, N = strs.count, len(strs.ids)
    ov = [o.viterbi(strs.get(b)) for b in range(B)]
    ofb = o.fb_batch(strs.ids, strs.offsets, nthreads=8)

    def check_exact():
        pv.viterbi()
        pf.forward_backward()
        torch.cuda.synchronize()
        sc, pa, ol, st = (pv.scores.cpu().numpy(), pv.paths.cpu().numpy(), pv.olabels.cpu().numpy(),
                          pv.status.cpu().numpy())
        for b in range(B):
            lo, hi = strs.offsets[b], strs.offsets[b + 1]
            assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], ov[b])
            assert_logz_close(pf.logz[b].item(), ofb["logz"][b])
        assert (pf.status[:B].cpu().numpy() == 0).all()
        assert_counts_close(pf.counts.cpu().numpy(), ofb["counts"], batch=True)

    check_exact()
    # every string has at least one live state per position, so 8 entries
    # cannot hold the run's live states
    for limit in (8, 1):
        pv.limit_pool(limit)
        pf.limit_pool(limit)
        pv.viterbi()
        pf.forward_backward()
        torch.cuda.synchronize()
        assert (pv.status[:B].cpu().numpy() == _lib.OOM).all()
        assert (pf.status[:B].cpu().numpy() == _lib.OOM).all()
        assert np.isneginf(pv.scores[:B].cpu().numpy()).all()
        assert (pv.paths[:N].cpu().numpy() == -1).all()
        assert np.isneginf(pf.logz[:B].cpu().numpy()).all()
        assert (pf.counts.cpu().numpy() == 0).all()
        # the cap lifted, the same plans are exact again
        pv.limit_pool(0)
        pf.limit_pool(0)
        check_exact()


def test_table_overflow_reports_oom_then_recovers():
    # the compact accumulator tables capped at 8 slots cannot hold one
    # position's live states (24 strings, each with at least one): the run
    # reports FST_ERR_OOM everywhere, and with the cap lifted the same plans
    # are exact again (the overflowing run's leftovers are cleared)
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=24)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    pv = f.plan(ids, off, flags=PLAN_NO_FB)
    pf = f.plan(ids, off, flags=PLAN_NO_VITERBI)
    B, N = strs.count, len(strs.ids)
    ofb = o.fb_batch(strs.ids, strs.offsets, nthreads=8)
    for rnd in range(2):
        pv.limit_table(8)
        pf.limit_table(8)
        pv.viterbi()
        pf.forward_backward()
        torch.cuda.synchronize()
        assert (pv.status[:B].cpu().numpy() == _lib.OOM).all()
        assert (pf.status[:B].cpu().numpy() == _lib.OOM).all()
        assert (pv.paths[:N].cpu().numpy() == -1).all()
        assert (pf.counts.cpu().numpy() == 0).all()
        pv.limit_table(0)
        pf.limit_table(0)
        pv.viterbi()
        pf.forward_backward()
        torch.cuda.synchronize()
        sc, pa, ol, st = (pv.scores.cpu().numpy(), pv.paths.cpu().numpy(), pv.olabels.cpu().numpy(),
                          pv.status.cpu().numpy())
        for b in range(B):
            lo, hi = strs.offsets[b], strs.offsets[b + 1]
            assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], o.viterbi(strs.get(b)))
            assert_logz_close(pf.logz[b].item(), ofb["logz"][b])
        assert_counts_close(pf.counts.cpu().numpy(), ofb["counts"], batch=True)
    with pytest.raises(_lib.FstError):
        pv.limit_table(-1)


def test_pool_limit_rejects_negative():
    import torch
    from paper_1701_03038_gb300._lib import FstError
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c1", scale=0.2, strings=2)
    f = Fst.from_arrays(fa)
    p = f.plan(torch.from_numpy(strs.ids).cuda(), torch.from_numpy(strs.offsets).cuda())
    with pytest.raises(FstError):
        p.limit_pool(-1)


def test_persistent_barrier_timeout_reports_and_recovers():
    # the persistent passes' grid barriers are told to wait for one block
    # that does not exist: every wait runs out after its limit (0.2 s here),
    # the run ends early with FST_ERR_TIMEOUT for every string, the GPU keeps
    # answering, and the next run on the same plans is exact
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c2", scale=0.02, strings=16)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    pv = f.plan(ids, off, flags=PLAN_NO_FB)
    pf = f.plan(ids, off, flags=PLAN_NO_VITERBI)
    for p in (pv, pf):
        p.set_driver(_lib.DRIVER_PERSISTENT, 0, 200_000)
    B = strs.count
    ov = [o.viterbi(strs.get(b)) for b in range(B)]
    ofb = o.fb_batch(strs.ids, strs.offsets, nthreads=8)
    for p in (pv, pf):
        p.fault_inject(_lib.FAULT_BARRIER_STALL, 1)
    t0 = time.perf_counter()
    pv.viterbi()
    torch.cuda.synchronize()
    pf.forward_backward()
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert waited < 30.0
    assert (pv.status[:B].cpu().numpy() == _lib.TIMEOUT).all()
    assert (pf.status[:B].cpu().numpy() == _lib.TIMEOUT).all()
    assert np.isneginf(pv.scores[:B].cpu().numpy()).all()
    assert np.isneginf(pf.logz[:B].cpu().numpy()).all()
    assert (pf.counts.cpu().numpy() == 0).all()
    # the context is still usable: the same plans, injection off, are exact
    for p in (pv, pf):
        p.fault_inject(_lib.FAULT_NONE)
    pv.viterbi()
    pf.forward_backward()
    torch.cuda.synchronize()
    sc, pa, ol, st = pv.scores.cpu().numpy(), pv.paths.cpu().numpy(), pv.olabels.cpu().numpy(), pv.status.cpu().numpy()
    for b in range(B):
        lo, hi = strs.offsets[b], strs.offsets[b + 1]
        assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], ov[b])
        assert_logz_close(pf.logz[b].item(), ofb["logz"][b])
    assert_counts_close(pf.counts.cpu().numpy(), ofb["counts"], batch=True)


def test_fault_inject_rejects_bad_arguments():
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import FstError
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c1", scale=0.2, strings=2)
    f = Fst.from_arrays(fa)
    p = f.plan(torch.from_numpy(strs.ids).cuda(), torch.from_numpy(strs.offsets).cuda())
    for kind, value in ((7, 0), (_lib.FAULT_BARRIER_STALL, -1), (_lib.FAULT_BARRIER_STALL, 5000)):
        with pytest.raises(FstError):
            p.fault_inject(kind, value)
    with pytest.raises(FstError):
        p.set_driver(5)
    with pytest.raises(FstError):
        p.set_driver(_lib.DRIVER_PERSISTENT, 10 ** 7)  # far more blocks than can be co-resident
