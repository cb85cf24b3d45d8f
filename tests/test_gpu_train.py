"""Training on the device: the EM M-step (fst_em_update) and the conditional
(CRF-style) likelihood through the output-clamped FST (fst_create_clamped),
against the oracle's EM update and clamped forward-backward."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_counts_close, assert_logz_close, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _case(strings=40, seed=0):
    fa, strs = synth.make_config("c2", scale=0.02, strings=strings, seed_offset=seed)
    return fa, strs


def test_em_update_matches_oracle():
    import torch
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = _case()
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    counts = o.fb_batch(strs.ids, strs.offsets, nthreads=8)["counts"]  # the oracle's counts feed both sides
    c32 = counts.astype(np.float32)
    for alpha in (0.0, 0.5):
        want = o.em_update(c32.astype(np.float64), alpha=alpha)
        got_h = f.em_update(c32, alpha)  # host arrays
        got_d = f.em_update(torch.from_numpy(c32).cuda(), alpha).cpu().numpy()  # device arrays
        for got in (got_h, got_d):
            # float64 arithmetic rounded once to float32
            assert np.allclose(got, want, rtol=2 ** -22, atol=1e-12), np.abs(got - want).max()
        # every used state's arcs form a distribution again
        used = np.bincount(fa.src, weights=c32 + alpha, minlength=fa.num_states) > 0
        tot = np.bincount(fa.src, weights=np.exp(got_h.astype(np.float64)), minlength=fa.num_states)
        assert np.allclose(tot[used], 1.0, atol=1e-5)


def test_em_apply_and_training_raises_likelihood():
    # EM iterations on the device (counts from the batched backward pass,
    # then the M-step installed with FST_EM_APPLY) beside the same
    # iterations in the oracle from the same start: the likelihoods
    # sum_b log Z_b agree at every iteration and never fall
    import torch
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = _case(strings=30, seed=3)
    f = Fst.from_arrays(fa)
    ids = torch.from_numpy(strs.ids).cuda()
    off = torch.from_numpy(strs.offsets).cuda()
    p = f.plan(ids, off)
    theta_o = oracle.theta_of_cost(fa.weight).astype(np.float64)
    prev = -math.inf
    for it in range(4):
        fo = synth.FstArrays(fa.num_states, fa.num_isyms, fa.num_osyms, fa.src, fa.dst, fa.ilabel, fa.olabel,
                             (-theta_o).astype(np.float32), fa.start_weight, fa.final_weight)
        o = oracle.Fst(fo)
        ob = o.fb_batch(strs.ids, strs.offsets, nthreads=8)
        p.forward_backward()
        torch.cuda.synchronize()
        for b in range(strs.count):
            assert_logz_close(p.logz[b].item(), ob["logz"][b])
        L = float(ob["logz"].sum())
        assert L >= prev - 1e-6 * max(1.0, abs(prev)), (it, L, prev)
        prev = L
        f.em_update(p.counts[:fa.num_arcs].clone(), 0.0, apply=True)
        theta_o = o.em_update(ob["counts"])


def test_clamped_log_z_and_posteriors_match_oracle():
    # log Z(x, y) and the posteriors given x and y: y the output of the
    # oracle's best path (a pair with paths), or random outputs (mostly none)
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = _case(strings=12, seed=5)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    cf = f.clamped()
    assert cf.num_pairs == len(set(zip(fa.ilabel.tolist(), fa.olabel.tolist())))
    rng = np.random.default_rng(4)
    seen = 0
    for b in range(strs.count):
        x = strs.get(b)
        for y in (o.viterbi(x)["olabels"], rng.integers(0, fa.num_osyms, size=len(x)).astype(np.int32)):
            want = o.forward_backward_clamped(x, y)
            lz, cnt, st = cf.forward_backward(cf.clamp(x, y))
            assert_logz_close(lz, want["logz"])
            assert_counts_close(cnt, want["counts"])
            seen += want["logz"] > -math.inf
            # the clamped weight never exceeds the unclamped one
            assert lz <= o.forward_backward(x)["logz"] + 1e-6
    assert seen >= strs.count


def test_crf_loss_gradient_and_training():
    # batched -log p(y|x) through autograd: its gradient is counts(x) -
    # counts(x, y); a few SGD steps lower it
    import torch
    from paper_1701_03038_gb300._lib import PLAN_SINGLE_WAVE
    from paper_1701_03038_gb300.autograd import CrfModule
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = _case(strings=24, seed=7)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ys = [o.viterbi(strs.get(b))["olabels"] for b in range(strs.count)]
    mod = CrfModule(f, -torch.from_numpy(fa.weight.astype(np.float32)))
    pair_ids = np.concatenate([mod.clamped.clamp(strs.get(b), ys[b]) for b in range(strs.count)]).astype(np.int32)
    off = torch.from_numpy(strs.offsets).cuda()
    plan_x = f.plan(torch.from_numpy(strs.ids).cuda(), off, flags=PLAN_SINGLE_WAVE)
    plan_xy = mod.clamped.plan(torch.from_numpy(pair_ids).cuda(), off, flags=PLAN_SINGLE_WAVE)
    nll = mod(plan_x, plan_xy)
    loss = nll.sum()
    loss.backward()
    torch.cuda.synchronize()
    ox = o.fb_batch(strs.ids, strs.offsets, nthreads=8)
    cxy = np.zeros(fa.num_arcs)
    for b in range(strs.count):
        r = o.forward_backward_clamped(strs.get(b), ys[b])
        assert_logz_close(ox["logz"][b] - nll[b].item(), r["logz"])
        cxy += r["counts"]
    want = ox["counts"] - cxy
    got = mod.theta.grad.cpu().numpy().astype(np.float64)
    tol = 1e-5 * np.maximum(1.0, ox["counts"] + cxy)
    assert (np.abs(got - want) <= tol).all(), np.abs(got - want).max()
    # training: the conditional likelihood of the pairs rises
    opt = torch.optim.SGD(mod.parameters(), lr=0.05)
    first = float(loss.item())
    for _ in range(5):
        opt.zero_grad()
        loss = mod(plan_x, plan_xy).sum()
        loss.backward()
        opt.step()
    final = float(mod(plan_x, plan_xy).sum().item())
    assert final < first - 1e-3, (first, final)
