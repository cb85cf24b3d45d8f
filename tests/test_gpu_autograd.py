"""Differentiation: d log Z / d theta = expected arc counts (Alg. 2), checked
against float64 finite differences on the GPU and against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_counts_close, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def sub_fst(seed=41):
    # the training workload's laws (Zipf labels, lognormal out-degree, mean
    # degree 20, Dirichlet(0.5)) on a 100-state, 2,000-arc sub-FST
    return synth.random_fst(100, 50, 50, 2000, label_law="zipf", src_law="lognormal", mean_degree=20.0,
                            dirichlet=0.5, seed=seed)


def _dev(strs):
    import torch
    return torch.from_numpy(strs.ids).cuda(), torch.from_numpy(strs.offsets).cuda()


def test_float64_log_z_matches_oracle():
    from paper_1701_03038_gb300.fst import Fst
    for fa, strs in [(sub_fst(), None), synth.make_config("c2", scale=0.01, strings=4)]:
        if strs is None:
            strs = synth.make_strings(fa, 4, 10, 60, seed=7)
        f, o = Fst.from_arrays(fa), oracle.Fst(fa)
        th = o.theta.astype(np.float64)
        for b in range(strs.count):
            x = strs.get(b)
            got = f.log_z_f64(x, th if b == 0 else None)
            want = o.forward_backward(x)["logz"]
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (got, want)


def test_float64_log_z_long_segments():
    from paper_1701_03038_gb300.fst import Fst
    rng = np.random.default_rng(3)
    A = 900
    fa = synth.FstArrays(1, 2, 2, np.zeros(A, np.int32), np.zeros(A, np.int32),
                         rng.integers(0, 2, size=A).astype(np.int32), np.zeros(A, np.int32),
                         (rng.random(A) * 3).astype(np.float32), np.zeros(1, np.float32), np.zeros(1, np.float32))
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    x = rng.integers(0, 2, size=9).astype(np.int32)
    got = f.log_z_f64(x, o.theta.astype(np.float64))
    want = o.forward_backward(x)["logz"]
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_gradient_equals_counts_and_finite_differences():
    import torch
    from paper_1701_03038_gb300.autograd import log_z
    from paper_1701_03038_gb300.fst import Fst
    fa = sub_fst()
    strs = synth.make_strings(fa, 4, 10, 40, seed=11)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    plan = f.plan(ids, off, flags=1 | 2)  # single wave, no Viterbi storage
    theta = torch.tensor(o.theta, device="cuda", requires_grad=True)
    lz = log_z(theta, f, plan)
    lz.sum().backward()
    g = theta.grad.double().cpu().numpy()
    ob = o.fb_batch(strs.ids, strs.offsets, nthreads=4)
    assert np.allclose(lz.detach().cpu().numpy(), ob["logz"], rtol=1e-5, atol=0)
    assert_counts_close(g, ob["counts"], batch=True)
    # float64 central differences on the GPU, h = 1e-6, on the arcs with the
    # largest counts and a random sample of the rest
    th = o.theta.astype(np.float64)
    rng = np.random.default_rng(5)
    ks = list(np.argsort(-ob["counts"])[:40]) + list(rng.choice(fa.num_arcs, size=40, replace=False))
    h = 1e-6

    def total(t):
        return math.fsum(f.log_z_f64(strs.get(b), t if b == 0 else None) for b in range(strs.count))

    for k in ks:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (total(tp) - total(tm)) / (2 * h)
        assert abs(fd - ob["counts"][k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, ob["counts"][k])
        assert abs(g[k] - fd) <= 1e-4 * max(abs(fd), 1e-2), (k, g[k], fd)


def test_weighted_gradient_and_training_loop():
    import torch
    from paper_1701_03038_gb300.autograd import LogZModule
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = synth.make_config("c4", scale=0.01, strings=24)
    f = Fst.from_arrays(fa)
    ids, off = _dev(strs)
    plan = f.plan(ids, off, flags=1 | 2)
    o = oracle.Fst(fa)
    model = LogZModule(f, torch.tensor(o.theta, device="cuda"))
    opt = torch.optim.SGD(model.parameters(), lr=0.05)
    w = torch.linspace(0.5, 1.5, strs.count, device="cuda", dtype=torch.float64)
    for step in range(3):
        opt.zero_grad()
        lz = model(plan)
        loss = -(w * lz).sum()
        loss.backward()
        # gradient = -sum_b w_b count_b at the current weights
        cur = fa.weight.copy()
        th = model.theta.detach().cpu().numpy()
        cur = (-th).astype(np.float32)
        fa_cur = synth.FstArrays(fa.num_states, fa.num_isyms, fa.num_osyms, fa.src, fa.dst, fa.ilabel, fa.olabel,
                                 cur, fa.start_weight, fa.final_weight)
        ob = oracle.Fst(fa_cur).fb_batch(strs.ids, strs.offsets, nthreads=4, weights=w.cpu().numpy())
        assert_counts_close(-model.theta.grad.double().cpu().numpy(), ob["counts"], batch=True)
        assert np.allclose(lz.detach().cpu().numpy(), ob["logz"], rtol=1e-5, atol=0)
        opt.step()


def _multi_start_fst(seed=43):
    # several start states and final states with unequal weights, so that
    # the start and final posteriors are spread out
    fa = sub_fst(seed)
    rng = np.random.default_rng(seed)
    sw = np.full(fa.num_states, np.inf, np.float32)
    starts = rng.choice(fa.num_states, 6, replace=False)
    sw[starts] = rng.uniform(0.0, 3.0, 6).astype(np.float32)
    sw[0] = 0.0
    fw = np.full(fa.num_states, np.inf, np.float32)
    finals = rng.choice(fa.num_states, 25, replace=False)
    fw[finals] = rng.uniform(0.0, 3.0, 25).astype(np.float32)
    fa.start_weight, fa.final_weight = sw, fw
    return fa


def test_state_posteriors_match_oracle():
    import torch
    from paper_1701_03038_gb300.fst import Fst
    fa = _multi_start_fst()
    strs = synth.make_strings(fa, 12, 1, 30, seed=12)
    # append an empty string: its path starts and ends in the same state
    strs = synth.Strings(strs.ids, np.concatenate([strs.offsets, strs.offsets[-1:]]))
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    w = np.linspace(0.5, 2.0, strs.count).astype(np.float32)
    plan = f.plan(ids, off, flags=1 | 2)
    plan.forward_backward(torch.from_numpy(w).cuda(), states=True)
    torch.cuda.synchronize()
    want = o.state_posteriors_batch(strs.ids, strs.offsets, weights=w)
    assert_counts_close(plan.start_counts[:fa.num_states].cpu().numpy(), want["start"], batch=True)
    assert_counts_close(plan.final_counts[:fa.num_states].cpu().numpy(), want["final"], batch=True)
    assert want["start"].sum() == pytest.approx(float(w.sum()), rel=1e-9)
    # forward then backward with states gives the same
    plan.forward()
    plan.backward(torch.from_numpy(w).cuda(), states=True)
    torch.cuda.synchronize()
    assert_counts_close(plan.final_counts[:fa.num_states].cpu().numpy(), want["final"], batch=True)


def test_gradients_of_start_and_final_weights():
    import torch
    from paper_1701_03038_gb300.autograd import log_z
    from paper_1701_03038_gb300.fst import Fst
    fa = _multi_start_fst(47)
    strs = synth.make_strings(fa, 8, 5, 25, seed=13)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids, off = _dev(strs)
    plan = f.plan(ids, off, flags=1 | 2)
    theta = torch.tensor(o.theta, device="cuda", requires_grad=True)
    ts = torch.tensor(oracle.theta_of_cost(fa.start_weight), device="cuda", dtype=torch.float32, requires_grad=True)
    tf = torch.tensor(oracle.theta_of_cost(fa.final_weight), device="cuda", dtype=torch.float32, requires_grad=True)
    lz = log_z(theta, f, plan, ts, tf)
    lz.sum().backward()
    want = o.state_posteriors_batch(strs.ids, strs.offsets)
    assert_counts_close(ts.grad.double().cpu().numpy(), want["start"], batch=True)
    assert_counts_close(tf.grad.double().cpu().numpy(), want["final"], batch=True)
    ob = o.fb_batch(strs.ids, strs.offsets, nthreads=4)
    assert_counts_close(theta.grad.double().cpu().numpy(), ob["counts"], batch=True)
    # a changed final weight reaches log Z: one gradient step on theta_f
    # raises sum log Z by about |grad|^2 * lr
    with torch.no_grad():
        tf2 = torch.where(torch.isfinite(tf), tf + 0.01 * tf.grad, tf)
    lz2 = log_z(theta.detach(), f, plan, ts.detach(), tf2)
    gain = float((lz2.sum() - lz.sum()).item())
    g2 = float((tf.grad[torch.isfinite(tf)] ** 2).sum().item())
    assert gain == pytest.approx(0.01 * g2, rel=0.05)

