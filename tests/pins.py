"""Independent checks that pin the CPU oracle to the paper and to mathematics.

Each ``pin_*`` function takes an oracle library handle (so that the mutant
test can run the same checks against a deliberately broken build) and
raises AssertionError on a mismatch.  None of them re-types the oracle's
recurrences: they use the worked example of Figs. 1-2, exhaustive path
enumeration, a textbook dense HMM, closed forms and invariants.
"""
from __future__ import annotations

import fractions
import itertools
import json
import math
import os

import numpy as np

import oracle
from paper_1701_03038_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _f32(x):
    return np.float32(x)


def _lse(v):
    v = np.asarray(v, np.float64)
    if v.size == 0:
        return -math.inf
    m = np.max(v)
    if m == -math.inf:
        return -math.inf
    return float(m + math.log(math.fsum(np.exp(v - m))))


# --------------------------------------------------------------------------
# Fig. 1 / Fig. 2 worked example
# --------------------------------------------------------------------------
def fig1_case():
    with open(os.path.join(GOLDEN, "fig1.json")) as fh:
        g = json.load(fh)
    isym = {s: i for i, s in enumerate(g["input_symbols"])}
    osym = {s: i for i, s in enumerate(g["output_symbols"])}
    R = g["R"]
    il = np.zeros(len(g["S"]), np.int32)
    for a in range(len(R) - 1):
        il[R[a]:R[a + 1]] = a
    q = g["num_states"]
    fst = synth.FstArrays(
        q, len(isym), len(osym), np.array(g["S"], np.int32), np.array(g["T"], np.int32), il,
        np.array([osym[o] for o in g["O"]], np.int32),
        (-np.log(np.array(g["P"], np.float64))).astype(np.float32),
        np.where(np.arange(q) == g["start_state"], 0.0, np.inf).astype(np.float32),
        np.array([(-math.log(g["final_states"][str(s)]) if str(s) in g["final_states"] else np.inf)
                  for s in range(q)], np.float32))
    x = np.array([isym[s] for s in g["input"]], np.int32)
    exp = g["expected"]
    exp_out = [osym[o] for o in exp["viterbi_output"]]
    post = [float(fractions.Fraction(p)) for p in exp["arc_posteriors"]]
    return fst, x, exp, exp_out, post


def pin_fig1(lib):
    fst, x, exp, exp_out, post = fig1_case()
    o = oracle.Fst(fst, lib)
    v = o.viterbi(x)
    assert v["status"] == oracle.OK
    assert list(v["path"]) == exp["viterbi_arcs"]
    assert list(v["olabels"]) == exp_out
    # one path with log-weight log(0.48) + 0 + 0 (+ final weight log 1 = 0)
    assert v["best"] == _f32(math.log(exp["viterbi_probability"]))
    fb = o.forward_backward(x)
    assert fb["status"] == oracle.OK
    assert abs(fb["logz"] - math.log(exp["total_weight_Z"])) < 1e-6  # P are float32
    assert np.allclose(fb["counts"], post, atol=1e-6, rtol=0)


# --------------------------------------------------------------------------
# Exhaustive path enumeration on tiny FSTs
# --------------------------------------------------------------------------
def enumerate_paths(fst, x):
    """All accepting arc sequences for string x, with their float32
    left-to-right weight and float64 weight."""
    th = oracle.theta_of_cost(fst.weight)
    ts = oracle.theta_of_cost(fst.start_weight)
    tf = oracle.theta_of_cost(fst.final_weight)
    by_label = {}
    for k in range(fst.num_arcs):
        by_label.setdefault(int(fst.ilabel[k]), []).append(k)
    n = len(x)
    out = []
    if n == 0:
        for q in range(fst.num_states):
            if ts[q] > -np.inf and tf[q] > -np.inf:
                out.append(((), _f32(ts[q]) + _f32(tf[q]), float(ts[q]) + float(tf[q]), q))
        return out
    cand = [by_label.get(int(a), []) for a in x]
    for seq in itertools.product(*cand):
        if ts[fst.src[seq[0]]] == -np.inf:
            continue
        ok = all(fst.dst[seq[i]] == fst.src[seq[i + 1]] for i in range(n - 1))
        qn = int(fst.dst[seq[-1]])
        if not ok or tf[qn] == -np.inf:
            continue
        w32 = _f32(ts[fst.src[seq[0]]])
        w64 = float(ts[fst.src[seq[0]]])
        for k in seq:
            w32 = _f32(w32 + th[k])
            w64 += float(th[k])
        w32 = _f32(w32 + tf[qn])
        w64 += float(tf[qn])
        out.append((seq, w32, w64, qn))
    return out


def _path_weight32(fst, seq, q0=None):
    th = oracle.theta_of_cost(fst.weight)
    ts = oracle.theta_of_cost(fst.start_weight)
    tf = oracle.theta_of_cost(fst.final_weight)
    w = _f32(ts[fst.src[seq[0]]])
    for k in seq:
        w = _f32(w + th[k])
    return _f32(w + tf[fst.dst[seq[-1]]])


def pin_bruteforce(lib, cases=150, seed=7):
    rng = np.random.default_rng(seed)
    checked_paths = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng)
        n = int(rng.integers(0, 6))
        x = rng.integers(0, fst.num_isyms, size=n).astype(np.int32)
        paths = enumerate_paths(fst, x)
        o = oracle.Fst(fst, lib)
        v = o.viterbi(x)
        fb = o.forward_backward(x)
        if not paths:
            assert v["status"] == oracle.NO_PATH and v["best"] == -np.inf
            assert fb["status"] == oracle.NO_PATH and fb["logz"] == -math.inf
            assert np.all(fb["counts"] == 0)
            continue
        checked_paths += len(paths)
        best = max(p[1] for p in paths)
        assert v["status"] == oracle.OK
        assert v["best"] == best, (v["best"], best)
        if n > 0:
            seq = tuple(int(k) for k in v["path"])
            assert seq in {p[0] for p in paths}
            assert _path_weight32(fst, seq) == best
        logz = _lse([p[2] for p in paths])
        assert abs(fb["logz"] - logz) <= 1e-12 * max(1.0, abs(logz))
        cnt = np.zeros(fst.num_arcs)
        for seq, _, w64, _ in paths:
            for k in seq:
                cnt[k] += math.exp(w64 - logz)
        assert np.allclose(fb["counts"], cnt, atol=1e-12, rtol=1e-12)
    assert checked_paths > 50


def pin_ties(lib, cases=60, seed=11):
    """All weights zero: every accepting path ties.  The tie rule (lowest arc
    id into each state at each step, then lowest final state) then fixes the
    path; derive it from the reachable sets of the enumerated paths."""
    rng = np.random.default_rng(seed)
    seen = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng, multi_start=True)
        fst.weight[:] = 0.0
        fst.start_weight[np.isfinite(fst.start_weight)] = 0.0
        fst.final_weight[np.isfinite(fst.final_weight)] = 0.0
        n = int(rng.integers(1, 5))
        x = rng.integers(0, fst.num_isyms, size=n).astype(np.int32)
        paths = enumerate_paths(fst, x)
        if not paths:
            continue
        seen += 1
        # states reachable after t symbols (from any start, ignoring finals)
        reach = [set(int(q) for q in np.flatnonzero(np.isfinite(fst.start_weight)))]
        for t in range(n):
            nxt = set()
            for k in range(fst.num_arcs):
                if fst.ilabel[k] == x[t] and int(fst.src[k]) in reach[t]:
                    nxt.add(int(fst.dst[k]))
            reach.append(nxt)
        qf = min(p[3] for p in paths)
        expect = [0] * n
        q = qf
        for t in range(n, 0, -1):
            ks = [k for k in range(fst.num_arcs)
                  if fst.ilabel[k] == x[t - 1] and fst.dst[k] == q and int(fst.src[k]) in reach[t - 1]]
            expect[t - 1] = min(ks)
            q = int(fst.src[min(ks)])
        v = oracle.Fst(fst, lib).viterbi(x)
        assert v["best"] == 0.0
        assert v["final_state"] == qf
        assert list(v["path"]) == expect, (list(v["path"]), expect)
    assert seen > 10


# --------------------------------------------------------------------------
# Dense HMM (textbook forward-backward and Viterbi)
# --------------------------------------------------------------------------
def pin_hmm(lib, cases=20, seed=3):
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        K, V = int(rng.integers(2, 5)), int(rng.integers(2, 5))
        n = int(rng.integers(1, 8))
        pi = rng.dirichlet(np.ones(K))
        A = rng.dirichlet(np.ones(K), size=K)
        Bm = rng.dirichlet(np.ones(V), size=K)
        obs = rng.integers(0, V, size=n)
        fst = synth.hmm_fst(pi, A, Bm)
        # the FST stores float32 costs: use exactly those probabilities
        p_start = np.exp(-fst.weight[:K * V].astype(np.float64)).reshape(K, V)
        p_tr = np.exp(-fst.weight[K * V:].astype(np.float64)).reshape(K, K, V)
        # textbook scaled-free forward / backward in the probability domain
        al = np.zeros((n, K))
        al[0] = p_start[:, obs[0]]
        for t in range(1, n):
            al[t] = al[t - 1] @ p_tr[:, :, obs[t]]
        be = np.ones((n, K))
        for t in range(n - 2, -1, -1):
            be[t] = p_tr[:, :, obs[t + 1]] @ be[t + 1]
        Z = al[-1].sum()
        cnt = np.zeros(fst.num_arcs)
        for j in range(K):
            cnt[j * V + obs[0]] += p_start[j, obs[0]] * be[0, j] / Z
        for t in range(1, n):
            xi = al[t - 1][:, None] * p_tr[:, :, obs[t]] * be[t][None, :] / Z
            for i in range(K):
                for j in range(K):
                    cnt[K * V + (i * K + j) * V + obs[t]] += xi[i, j]
        o = oracle.Fst(fst, lib)
        fb = o.forward_backward(obs.astype(np.int32))
        assert abs(fb["logz"] - math.log(Z)) < 1e-10
        assert np.allclose(fb["counts"], cnt, atol=1e-10)
        # textbook Viterbi (dense delta table) in float32 log weights
        th = oracle.theta_of_cost(fst.weight)
        th_s = th[:K * V].reshape(K, V)
        th_t = th[K * V:].reshape(K, K, V)
        delta = np.array([_f32(th_s[j, obs[0]]) for j in range(K)], np.float32)
        psi = np.zeros((n, K), np.int64)
        for t in range(1, n):
            nd = np.empty(K, np.float32)
            for j in range(K):
                c = np.array([_f32(delta[i] + th_t[i, j, obs[t]]) for i in range(K)], np.float32)
                psi[t, j] = int(np.argmax(c))
                nd[j] = c[psi[t, j]]
            delta = nd
        jb = int(np.argmax(delta))
        states = [jb]
        for t in range(n - 1, 0, -1):
            states.append(int(psi[t, states[-1]]))
        states = states[::-1]
        v = o.viterbi(obs.astype(np.int32))
        assert v["best"] == delta[jb]
        # the arcs' destinations are the hidden states (+1)
        assert [int(fst.dst[k]) - 1 for k in v["path"]] == states


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------
def pin_single_state(lib, cases=20, seed=5):
    """One state, all arcs self-loops: log Z = sum_t LSE of the slice,
    Viterbi = float32 running sum of the slice maxima, gamma_t = softmax."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        m = int(rng.integers(1, 6))
        A = int(rng.integers(m, 40))
        il = np.concatenate([np.arange(m), rng.integers(0, m, size=A - m)]).astype(np.int32)
        w = (rng.random(A) * 4.0).astype(np.float32)
        w[rng.random(A) < 0.1] = w[0]  # some exact ties
        fst = synth.FstArrays(1, m, 2, np.zeros(A, np.int32), np.zeros(A, np.int32), il,
                              np.zeros(A, np.int32), w, np.zeros(1, np.float32),
                              np.zeros(1, np.float32))
        n = int(rng.integers(0, 30))
        x = rng.integers(0, m, size=n).astype(np.int32)
        th = oracle.theta_of_cost(w)
        logz = math.fsum(_lse(th[il == a].astype(np.float64)) for a in x)
        cnt = np.zeros(A)
        best = _f32(0.0)
        path = []
        for a in x:
            idx = np.flatnonzero(il == a)
            v = th[idx].astype(np.float64)
            cnt[idx] += np.exp(v - _lse(v))
            j = idx[int(np.argmax(th[idx]))]  # first maximum = lowest arc id
            path.append(int(j))
            best = _f32(best + th[j])
        o = oracle.Fst(fst, lib)
        fb = o.forward_backward(x)
        assert abs(fb["logz"] - logz) <= 1e-11 * max(1.0, abs(logz))
        assert np.allclose(fb["counts"], cnt, atol=1e-11)
        v = o.viterbi(x)
        assert v["best"] == best
        assert list(v["path"]) == path


def pin_unweighted_count(lib, cases=15, seed=9):
    """All weights zero (p = 1): Z is the number of accepting paths, counted
    here exactly with Python integers; the expected count of an arc is the
    number of (path, position) uses divided by Z."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        q, m, A = int(rng.integers(2, 12)), int(rng.integers(1, 4)), int(rng.integers(4, 60))
        fst = synth.random_fst(q, m, 2, A, seed=int(rng.integers(1 << 30)))
        fst.weight[:] = 0.0
        fst.final_weight[np.isfinite(fst.final_weight)] = 0.0
        fst.final_weight[int(rng.integers(0, q))] = 0.0
        n = int(rng.integers(1, 12))
        x = rng.integers(0, m, size=n).astype(np.int32)
        fwd = [[0] * q for _ in range(n + 1)]
        fwd[0][0] = 1
        for t in range(1, n + 1):
            for k in range(A):
                if fst.ilabel[k] == x[t - 1]:
                    fwd[t][fst.dst[k]] += fwd[t - 1][fst.src[k]]
        fin = [int(np.isfinite(fst.final_weight[s])) for s in range(q)]
        bwd = [[0] * q for _ in range(n + 1)]
        bwd[n] = fin[:]
        for t in range(n, 0, -1):
            for k in range(A):
                if fst.ilabel[k] == x[t - 1]:
                    bwd[t - 1][fst.src[k]] += bwd[t][fst.dst[k]]
        total = sum(fwd[n][s] * fin[s] for s in range(q))
        assert total == bwd[0][0]
        fb = oracle.Fst(fst, lib).forward_backward(x)
        if total == 0:
            assert fb["logz"] == -math.inf
            continue
        assert abs(fb["logz"] - math.log(total)) <= 1e-12 * max(1.0, math.log(total))
        uses = np.zeros(A)
        for t in range(1, n + 1):
            for k in range(A):
                if fst.ilabel[k] == x[t - 1]:
                    uses[k] += fwd[t - 1][fst.src[k]] * bwd[t][fst.dst[k]]
        assert np.allclose(fb["counts"], uses / total, atol=1e-12, rtol=1e-10)


# --------------------------------------------------------------------------
# Invariants on a c1-shaped FST
# --------------------------------------------------------------------------
def pin_invariants(lib, seed=1):
    fst, strs = synth.make_config("c1", scale=0.2, strings=3)
    o = oracle.Fst(fst, lib)
    th = o.theta
    for b in range(strs.count):
        x = strs.get(b)
        n = len(x)
        fb = o.forward_backward(x, tables=True)
        assert fb["status"] == oracle.OK
        logz, al, be = fb["logz"], fb["alpha"], fb["beta"]
        for t in range(n + 1):
            assert abs(_lse(al[t] + be[t]) - logz) < 1e-9 * max(1, abs(logz))
        assert abs(_lse(o.theta_s.astype(np.float64) + be[0]) - logz) < 1e-9 * max(1, abs(logz))
        # per-step posteriors sum to one, total count = n
        for t in range(1, n + 1):
            idx = np.flatnonzero(fst.ilabel == x[t - 1])
            g = np.exp(al[t - 1][fst.src[idx]] + th[idx] + be[t][fst.dst[idx]] - logz)
            assert abs(g.sum() - 1.0) < 1e-9
        assert abs(fb["counts"].sum() - n) < 1e-8 * n
        v = o.viterbi(x)
        assert v["best"] <= logz + 1e-4
        assert v["status"] == oracle.OK


def pin_deterministic(lib, cases=10, seed=13):
    """A deterministic FST (one arc per (state, symbol)) has a single path per
    string, so Viterbi = log Z and the counts are 0/1 along that path."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        q, m = int(rng.integers(2, 30)), int(rng.integers(1, 5))
        src = np.repeat(np.arange(q), m).astype(np.int32)
        il = np.tile(np.arange(m), q).astype(np.int32)
        dst = rng.integers(0, q, size=q * m).astype(np.int32)
        w = (rng.random(q * m) * 3).astype(np.float32)
        perm = rng.permutation(q * m)
        fst = synth.FstArrays(q, m, 2, src[perm], dst[perm], il[perm], np.zeros(q * m, np.int32),
                              w[perm], np.where(np.arange(q) == 0, 0, np.inf).astype(np.float32),
                              np.zeros(q, np.float32))
        x = rng.integers(0, m, size=int(rng.integers(1, 40))).astype(np.int32)
        o = oracle.Fst(fst, lib)
        v, fb = o.viterbi(x), o.forward_backward(x)
        assert abs(float(v["best"]) - fb["logz"]) <= 1e-5 * max(1, abs(fb["logz"]))
        c = np.zeros(fst.num_arcs)
        np.add.at(c, v["path"], 1.0)
        assert np.allclose(fb["counts"], c, atol=1e-12)


def pin_state_posteriors(lib, cases=120, seed=17):
    """Start and final state posteriors against exhaustive path enumeration:
    P(start in q) and P(end in q) summed over the accepting paths, and the
    worked example of Figs. 1-2 (one start state, one final state)."""
    fst, x, _, _, _ = fig1_case()
    r = oracle.Fst(fst, lib).state_posteriors(x)
    one0 = np.zeros(fst.num_states)
    one0[0] = 1.0
    assert np.allclose(r["start"], one0, atol=1e-12)
    assert abs(r["final"].sum() - 1.0) < 1e-12 and r["final"].argmax() == 5
    rng = np.random.default_rng(seed)
    seen = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng)
        ts = oracle.theta_of_cost(fst.start_weight)
        n = int(rng.integers(0, 5))
        x = rng.integers(0, fst.num_isyms, size=n).astype(np.int32)
        paths = enumerate_paths(fst, x)
        r = oracle.Fst(fst, lib).state_posteriors(x)
        ws, wf = np.zeros(fst.num_states), np.zeros(fst.num_states)
        if paths:
            seen += 1
            logz = _lse([p[2] for p in paths])
            for seq, _, w64, qn in paths:
                q0 = qn if not seq else int(fst.src[seq[0]])
                ws[q0] += math.exp(w64 - logz)
                wf[qn] += math.exp(w64 - logz)
            assert abs(ws.sum() - 1.0) < 1e-9 and abs(wf.sum() - 1.0) < 1e-9
            assert np.all(ws[ts == -np.inf] == 0)
        assert np.allclose(r["start"], ws, atol=1e-12, rtol=1e-12), (r["start"], ws)
        assert np.allclose(r["final"], wf, atol=1e-12, rtol=1e-12), (r["final"], wf)
    assert seen > 20


# --------------------------------------------------------------------------
# Output-clamped log Z (the numerator of a conditional / CRF likelihood)
# --------------------------------------------------------------------------
def pin_clamped_bruteforce(lib, cases=150, seed=19):
    """log Z(x, y) and the arc posteriors given x and y against the accepting
    paths of x whose output labels spell y, enumerated; y is the output of
    a random accepting path half of the time, else random."""
    rng = np.random.default_rng(seed)
    seen = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng)
        n = int(rng.integers(0, 5))
        x = rng.integers(0, fst.num_isyms, size=n).astype(np.int32)
        paths = enumerate_paths(fst, x)
        if paths and rng.random() < 0.5:
            seq = paths[int(rng.integers(0, len(paths)))][0]
            y = np.array([fst.olabel[k] for k in seq], np.int32)
        else:
            y = rng.integers(0, 4, size=n).astype(np.int32)
        keep = [p for p in paths if tuple(int(fst.olabel[k]) for k in p[0]) == tuple(int(v) for v in y)]
        r = oracle.Fst(fst, lib).forward_backward_clamped(x, y)
        if not keep:
            assert r["logz"] == -math.inf and np.all(r["counts"] == 0)
            continue
        seen += 1
        logz = _lse([p[2] for p in keep])
        assert abs(r["logz"] - logz) <= 1e-12 * max(1.0, abs(logz))
        cnt = np.zeros(fst.num_arcs)
        for seq, _, w64, _ in keep:
            for k in seq:
                cnt[k] += math.exp(w64 - logz)
        assert np.allclose(r["counts"], cnt, atol=1e-12, rtol=1e-12)
    assert seen > 30


def pin_clamped_marginal(lib, cases=40, seed=23):
    """Summing Z(x, y) over every output string y of length n gives Z(x):
    each path writes exactly one y."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        fst = synth.tiny_fst(rng)
        n = int(rng.integers(0, 4))
        x = rng.integers(0, fst.num_isyms, size=n).astype(np.int32)
        o = oracle.Fst(fst, lib)
        want = o.forward_backward(x)["logz"]
        got = _lse([o.forward_backward_clamped(x, np.array(y, np.int32))["logz"]
                    for y in itertools.product(range(4), repeat=n)])
        if want == -math.inf:
            assert got == -math.inf
        else:
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


# --------------------------------------------------------------------------
# EM re-estimation from expected counts (Sec. 4: the counts serve EM)
# --------------------------------------------------------------------------
def pin_em_fig1(lib):
    """Worked example: the counts of "le chat </s>" are 6/7, 1/7 on the two
    arcs out of state 0 and the same on the single arcs of states 1-4, so
    the M-step gives log 6/7, log 1/7 and log 1 = 0 elsewhere; with a
    pseudo-count of 1, state 0 gets (6/7 + 1) / 3 = 13/21 and 8/21."""
    fst, x, _, _, post = fig1_case()
    o = oracle.Fst(fst, lib)
    c = o.forward_backward(x)["counts"]
    assert np.allclose(c, post, atol=1e-6)
    exact = np.array(post, np.float64)
    th = o.em_update(exact)
    want = np.log([6 / 7, 1 / 7, 1.0, 1.0, 1.0, 1.0])
    assert np.allclose(th, want, atol=1e-14, rtol=0)
    th1 = o.em_update(exact, alpha=1.0)
    want1 = np.log([13 / 21, 8 / 21, 1.0, 1.0, 1.0, 1.0])
    assert np.allclose(th1, want1, atol=1e-14, rtol=0)


def pin_em_invariants(lib, cases=60, seed=29):
    """On random FSTs: each used state's new arc probabilities sum to one,
    unused states keep their weights, the pseudo-count closed form holds,
    and an EM step from normalised weights never lowers the likelihood
    sum_b log Z(x_b) (the M-step maximises the expected complete
    log-likelihood over per-state distributions)."""
    rng = np.random.default_rng(seed)
    rises = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng, max_states=5, max_arcs=12)
        o = oracle.Fst(fst, lib)
        # normalised starting weights: each state's arcs as a distribution
        p0 = np.exp(o.theta.astype(np.float64))
        tot = np.bincount(fst.src, weights=p0, minlength=fst.num_states)
        th0 = np.log(p0 / tot[fst.src])
        fa = synth.FstArrays(fst.num_states, fst.num_isyms, fst.num_osyms, fst.src, fst.dst, fst.ilabel,
                             fst.olabel, (-th0).astype(np.float32), fst.start_weight, fst.final_weight)
        o = oracle.Fst(fa, lib)
        xs = [rng.integers(0, fst.num_isyms, size=int(rng.integers(1, 5))).astype(np.int32) for _ in range(4)]
        fbs = [o.forward_backward(x) for x in xs]
        if all(r["logz"] == -math.inf for r in fbs):
            continue
        L0 = sum(r["logz"] for r in fbs if r["logz"] > -math.inf)
        counts = sum(r["counts"] for r in fbs)
        th1 = o.em_update(counts)
        used = np.bincount(fst.src, weights=counts, minlength=fst.num_states) > 0
        for q in range(fst.num_states):
            arcs = np.flatnonzero(fst.src == q)
            if arcs.size and used[q]:
                assert abs(np.exp(th1[arcs]).sum() - 1.0) < 1e-12
            elif arcs.size:
                assert np.array_equal(th1[arcs], o.theta[arcs].astype(np.float64))
        a = 0.5
        th2 = o.em_update(counts, alpha=a)
        den = np.bincount(fst.src, weights=counts + a, minlength=fst.num_states)
        assert np.allclose(th2, np.log((counts + a) / den[fst.src]), atol=1e-12, rtol=0)
        # the likelihood in float64 weights (float32 storage would blur a tiny rise)
        L1 = sum(_lse([p[2] for p in _enum64(fa, th1, x)]) for x, r in zip(xs, fbs) if r["logz"] > -math.inf)
        L0e = sum(_lse([p[2] for p in _enum64(fa, th0, x)]) for x, r in zip(xs, fbs) if r["logz"] > -math.inf)
        assert abs(L0e - L0) < 1e-5 * max(1.0, abs(L0))
        assert L1 >= L0e - 1e-9, (L1, L0e)
        rises += L1 > L0e + 1e-9
    assert rises > 10


def _enum64(fst, theta64, x):
    """Accepting paths of x with float64 arc log-weights theta64."""
    ts = oracle.theta_of_cost(fst.start_weight).astype(np.float64)
    tf = oracle.theta_of_cost(fst.final_weight).astype(np.float64)
    cand = [np.flatnonzero(fst.ilabel == a) for a in x]
    out = []
    for seq in itertools.product(*cand):
        if ts[fst.src[seq[0]]] == -np.inf or tf[fst.dst[seq[-1]]] == -np.inf:
            continue
        if not all(fst.dst[seq[i]] == fst.src[seq[i + 1]] for i in range(len(seq) - 1)):
            continue
        out.append((seq, None, ts[fst.src[seq[0]]] + sum(theta64[k] for k in seq) + tf[fst.dst[seq[-1]]]))
    return out


# --------------------------------------------------------------------------
# Acyclic input lattices (Sec. 6.1: an FST composed with an input lattice)
# --------------------------------------------------------------------------
def random_dag(rng, num_isyms, max_nodes=5, max_edges=7):
    n = int(rng.integers(1, max_nodes + 1))
    frm, to = [], []
    if n > 1:
        for _ in range(int(rng.integers(1, max_edges + 1))):
            u = int(rng.integers(0, n - 1))
            frm.append(u)
            to.append(int(rng.integers(u + 1, n)))
    e = len(frm)
    return oracle.Lattice(n, frm, to, rng.integers(0, num_isyms, size=e),
                          (-rng.random(e) * 2.0).astype(np.float32))


def lattice_paths(lat, v=0):
    """Edge sequences from node v to the end node."""
    if v == lat.N - 1:
        return [()]
    out = []
    for e in range(lat.E):
        if lat.frm[e] == v:
            out += [(e,) + rest for rest in lattice_paths(lat, int(lat.to[e]))]
    return out


def pin_lattice_chain(lib, cases=60, seed=31):
    """A string written as a linear lattice (edge weights 0) decodes exactly
    as the string: the same Viterbi score and arcs, log Z and counts."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        fst = synth.tiny_fst(rng)
        x = rng.integers(0, fst.num_isyms, size=int(rng.integers(0, 6))).astype(np.int32)
        o = oracle.Fst(fst, lib)
        lat = oracle.Lattice.from_string(x)
        v, lv = o.viterbi(x), oracle.lattice_viterbi(o, lat)
        assert lv["status"] == v["status"] and lv["best"] == v["best"]
        if v["status"] == oracle.OK:
            assert np.array_equal(lv["arcs"], v["path"]) and np.array_equal(lv["edges"], np.arange(len(x)))
        fb, lfb = o.forward_backward(x), oracle.lattice_forward_backward(o, lat)
        assert lfb["status"] == fb["status"]
        if fb["logz"] == -math.inf:
            assert lfb["logz"] == -math.inf
        else:
            assert abs(lfb["logz"] - fb["logz"]) <= 1e-12 * max(1.0, abs(fb["logz"]))
            assert np.allclose(lfb["counts"], fb["counts"], atol=1e-12, rtol=1e-12)
            assert np.allclose(lfb["edge_post"], 1.0, atol=1e-12)


def pin_lattice_bruteforce(lib, cases=150, seed=37):
    """Random small DAGs against every (lattice path, FST path) pair: the
    best float32 joint score (each step fl(fl(V + theta) + w)) and a path
    reaching it; log Z, arc and edge posteriors from the float64 weights."""
    rng = np.random.default_rng(seed)
    seen = 0
    for _ in range(cases):
        fst = synth.tiny_fst(rng, max_states=4, max_arcs=10)
        lat = random_dag(rng, fst.num_isyms)
        o = oracle.Fst(fst, lib)
        th = o.theta
        ts, tf = o.theta_s, o.theta_f
        joint = []
        for ep in lattice_paths(lat):
            x = np.array([lat.label[e] for e in ep], np.int32)
            for seq, _, w64, qn in enumerate_paths(fst, x):
                if seq:
                    v = _f32(ts[fst.src[seq[0]]])
                    for e, k in zip(ep, seq):
                        v = _f32(_f32(v + th[k]) + lat.weight[e])
                    v = _f32(v + tf[qn])
                else:
                    v = _f32(ts[qn] + tf[qn])
                joint.append((ep, seq, v, w64 + sum(float(lat.weight[e]) for e in ep)))
        lv = oracle.lattice_viterbi(o, lat)
        lfb = oracle.lattice_forward_backward(o, lat)
        if not joint:
            assert lv["status"] == oracle.NO_PATH and lfb["logz"] == -math.inf
            assert np.all(lfb["counts"] == 0) and np.all(lfb["edge_post"] == 0)
            continue
        seen += 1
        best = max(j[2] for j in joint)
        assert lv["best"] == best, (lv["best"], best)
        got = (tuple(int(e) for e in lv["edges"]), tuple(int(k) for k in lv["arcs"]))
        assert any(j[0] == got[0] and tuple(j[1]) == got[1] and j[2] == best for j in joint), got
        logz = _lse([j[3] for j in joint])
        assert abs(lfb["logz"] - logz) <= 1e-12 * max(1.0, abs(logz))
        cnt, ep_ = np.zeros(fst.num_arcs), np.zeros(lat.E)
        for ep, seq, _, w in joint:
            g = math.exp(w - logz)
            for k in seq:
                cnt[k] += g
            for e in ep:
                ep_[e] += g
        assert np.allclose(lfb["counts"], cnt, atol=1e-12, rtol=1e-12)
        assert np.allclose(lfb["edge_post"], ep_, atol=1e-12, rtol=1e-12)
    assert seen > 30


ALL_PINS = [pin_fig1, pin_bruteforce, pin_ties, pin_hmm, pin_single_state,
            pin_unweighted_count, pin_invariants, pin_deterministic, pin_state_posteriors,
            pin_clamped_bruteforce, pin_clamped_marginal, pin_em_fig1, pin_em_invariants,
            pin_lattice_chain, pin_lattice_bruteforce]
