"""Seeded synthetic FSTs and input strings.

This module only draws random inputs; it holds none of the decoding
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper's FSTs (a Europarl bigram LM composed with a GIZA++ translation
table, Sec. 7 and Table 4) are not available, so seeded generators with the
shapes of the five workloads stand in for them:

    c1  1,000 states, 50 input / 20 output symbols, 20,000 arcs, uniform
        sources, destinations and labels, Dirichlet(1) weights, one string
        of length 50.
    c2  50,000 states, 10,000 symbols, 5,000,000 arcs, Zipf(1) arcs per
        symbol, lognormal out-degree (mean 100), Dirichlet(0.5) weights,
        1,000 strings of length U[10, 60].
    c3  200,000 states, 20,000 symbols, 20,000,000 arcs, the laws of c2,
        4,096 strings of length U[5, 200].
    c4  100,000 states, 5,000 symbols, 2,000,000 arcs, the laws of c2 with
        mean out-degree 20, 1,024 strings of length U[10, 100].
    c5  1,000,000 states, 5,000 symbols, 100,000,000 arcs, uniform laws,
        Dirichlet(1) weights, 64 strings of length 1,000.

Weights are costs w = -log p (p drawn per source state from a Dirichlet over
its outgoing arcs, computed in float64, clamped at p >= 1e-300, stored as
float32).  The start state is 0; floor(0.1 Q) states, chosen without
replacement, are final with cost 0.  Symbol id r-1 has Zipf rank r, both in
the arc labels and in the strings.

Strings are seeded random walks from state 0 (one uniform out-arc per step,
the exact sampled length, rejected until the end state is final), so every
string has at least one accepting path.  ``kind="iid"`` draws i.i.d. symbols
from the label law instead; those strings are mostly rejected by the FST.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["FstArrays", "Strings", "CONFIGS", "random_fst", "make_strings",
           "make_config", "fig1_fst", "hmm_fst", "tiny_fst"]


@dataclasses.dataclass
class FstArrays:
    """An epsilon-free weighted FST in coordinate form (caller arc order).

    Weights are costs (w = -log p): ``weight[k]`` for arc k, and per state
    ``start_weight`` / ``final_weight`` with +inf meaning "not a start" /
    "not final".
    """
    num_states: int
    num_isyms: int
    num_osyms: int
    src: np.ndarray      # int32 [A]
    dst: np.ndarray      # int32 [A]
    ilabel: np.ndarray   # int32 [A]
    olabel: np.ndarray   # int32 [A]
    weight: np.ndarray   # float32 [A], cost domain
    start_weight: np.ndarray  # float32 [Q]
    final_weight: np.ndarray  # float32 [Q]

    @property
    def num_arcs(self) -> int:
        return int(self.src.shape[0])


@dataclasses.dataclass
class Strings:
    """A batch of input strings, concatenated: string b is ids[off[b]:off[b+1]]."""
    ids: np.ndarray      # int32 [N]
    offsets: np.ndarray  # int64 [B+1]

    @property
    def count(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def get(self, b: int) -> np.ndarray:
        return self.ids[self.offsets[b]:self.offsets[b + 1]]


CONFIGS = {
    "c1": dict(num_states=1_000, num_isyms=50, num_osyms=20, num_arcs=20_000,
               label_law="uniform", src_law="uniform", mean_degree=None,
               dirichlet=1.0, strings=1, len_lo=50, len_hi=50),
    "c2": dict(num_states=50_000, num_isyms=10_000, num_osyms=10_000, num_arcs=5_000_000,
               label_law="zipf", src_law="lognormal", mean_degree=100.0,
               dirichlet=0.5, strings=1_000, len_lo=10, len_hi=60),
    "c3": dict(num_states=200_000, num_isyms=20_000, num_osyms=20_000, num_arcs=20_000_000,
               label_law="zipf", src_law="lognormal", mean_degree=100.0,
               dirichlet=0.5, strings=4_096, len_lo=5, len_hi=200),
    "c4": dict(num_states=100_000, num_isyms=5_000, num_osyms=5_000, num_arcs=2_000_000,
               label_law="zipf", src_law="lognormal", mean_degree=20.0,
               dirichlet=0.5, strings=1_024, len_lo=10, len_hi=100),
    "c5": dict(num_states=1_000_000, num_isyms=5_000, num_osyms=5_000, num_arcs=100_000_000,
               label_law="uniform", src_law="uniform", mean_degree=None,
               dirichlet=1.0, strings=64, len_lo=1_000, len_hi=1_000),
}

FST_SEED_BASE = 1000
STRING_SEED_BASE = 2000


def _zipf_labels(rng: np.random.Generator, m: int, size: int, s: float = 1.0) -> np.ndarray:
    """i.i.d. draws from the finite Zipf law over ranks 1..m; returns rank-1."""
    w = 1.0 / np.arange(1, m + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(size)
    out = np.searchsorted(cdf, u, side="right")
    return np.minimum(out, m - 1).astype(np.int32)


def _lognormal_degrees(rng: np.random.Generator, q: int, total: int, mean: float,
                       sigma: float = 1.0) -> np.ndarray:
    """Out-degrees from a lognormal law (mean ``mean``), rounded by largest
    remainder so they sum to ``total``, each at least 1."""
    mu = math.log(mean) - sigma * sigma / 2.0
    x = rng.lognormal(mu, sigma, size=q)
    y = x * (total / x.sum())
    d = np.floor(y).astype(np.int64)
    rem = total - int(d.sum())
    if rem > 0:
        order = np.argsort(-(y - d), kind="stable")
        d[order[:rem]] += 1
    # every state keeps at least one outgoing arc
    zeros = np.flatnonzero(d == 0)
    if zeros.size:
        d[zeros] = 1
        excess = zeros.size
        order = np.argsort(-d, kind="stable")
        i = 0
        while excess > 0:
            j = order[i % q]
            if d[j] > 1:
                d[j] -= 1
                excess -= 1
            i += 1
    assert int(d.sum()) == total and int(d.min()) >= 1
    return d


def _dirichlet_costs(rng: np.random.Generator, src: np.ndarray, q: int, alpha: float) -> np.ndarray:
    """Per source state, p ~ Dirichlet(alpha) over its outgoing arcs; returns
    float32 costs -log(max(p, 1e-300)) computed in float64."""
    g = rng.gamma(alpha, 1.0, size=src.shape[0])
    sums = np.bincount(src, weights=g, minlength=q)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = g / sums[src]
    p = np.where(np.isfinite(p), p, 1.0)
    return (-np.log(np.maximum(p, 1e-300))).astype(np.float32)


def random_fst(num_states: int, num_isyms: int, num_osyms: int, num_arcs: int,
               label_law: str = "uniform", src_law: str = "uniform",
               mean_degree: float | None = None, dirichlet: float = 1.0,
               final_frac: float = 0.1, seed: int = 0, shuffle: bool = True) -> FstArrays:
    """Random epsilon-free FST with the given laws (see module docstring)."""
    rng = np.random.default_rng(seed)
    q, a = int(num_states), int(num_arcs)
    if src_law == "uniform":
        src = rng.integers(0, q, size=a, dtype=np.int64).astype(np.int32)
    elif src_law == "lognormal":
        deg = _lognormal_degrees(rng, q, a, mean_degree if mean_degree else a / q)
        src = np.repeat(np.arange(q, dtype=np.int32), deg)
    else:
        raise ValueError(src_law)
    dst = rng.integers(0, q, size=a, dtype=np.int64).astype(np.int32)
    if label_law == "uniform":
        il = rng.integers(0, num_isyms, size=a, dtype=np.int64).astype(np.int32)
    elif label_law == "zipf":
        il = _zipf_labels(rng, num_isyms, a)
    else:
        raise ValueError(label_law)
    ol = rng.integers(0, num_osyms, size=a, dtype=np.int64).astype(np.int32)
    if shuffle:
        perm = rng.permutation(a)
        src, dst, il, ol = src[perm], dst[perm], il[perm], ol[perm]
    w = _dirichlet_costs(rng, src, q, dirichlet)
    start = np.full(q, np.inf, dtype=np.float32)
    start[0] = 0.0
    final = np.full(q, np.inf, dtype=np.float32)
    nf = max(1, int(math.floor(final_frac * q)))
    final[rng.choice(q, size=nf, replace=False)] = 0.0
    return FstArrays(q, int(num_isyms), int(num_osyms), src, dst, il, ol, w, start, final)


def _out_arc_index(fst: FstArrays):
    order = np.argsort(fst.src, kind="stable")
    cnt = np.bincount(fst.src, minlength=fst.num_states)
    off = np.zeros(fst.num_states + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    return order, off


def make_strings(fst: FstArrays, count: int, len_lo: int, len_hi: int, seed: int,
                 kind: str = "walk", max_rounds: int = 10_000,
                 label_law: str | None = None) -> Strings:
    """``count`` strings with lengths uniform in [len_lo, len_hi].

    kind="walk": random walks from the start states that end in a final
    state (every string is accepted).  kind="iid": i.i.d. symbols drawn
    from ``label_law`` ("uniform" or "zipf")."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(len_lo, len_hi + 1, size=count, dtype=np.int64)
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    n_tot = int(offsets[-1])
    ids = np.empty(n_tot, dtype=np.int32)
    if kind == "iid":
        law = label_law or "uniform"
        if law == "zipf":
            ids[:] = _zipf_labels(rng, fst.num_isyms, n_tot)
        else:
            ids[:] = rng.integers(0, fst.num_isyms, size=n_tot, dtype=np.int64)
        return Strings(ids, offsets)
    if kind != "walk":
        raise ValueError(kind)
    order, off = _out_arc_index(fst)
    deg = off[1:] - off[:-1]
    starts = np.flatnonzero(np.isfinite(fst.start_weight))
    final = np.isfinite(fst.final_weight)
    pending = np.arange(count)
    for _ in range(max_rounds):
        if pending.size == 0:
            break
        m = pending.size
        state = starts[rng.integers(0, starts.size, size=m)]
        alive = np.ones(m, dtype=bool)
        plen = lens[pending]
        out = np.zeros((m, int(plen.max())), dtype=np.int32)
        for t in range(int(plen.max())):
            active = alive & (t < plen)
            d = deg[state]
            alive &= ~(active & (d == 0))
            active &= alive
            idx = np.flatnonzero(active)
            if idx.size == 0:
                continue
            dd = d[idx]
            pick = (rng.random(idx.size) * dd).astype(np.int64)
            pick = np.minimum(pick, dd - 1)
            arc = order[off[state[idx]] + pick]
            out[idx, t] = fst.ilabel[arc]
            state[idx] = fst.dst[arc]
        ok = alive & final[state]
        for i in np.flatnonzero(ok):
            b = pending[i]
            ids[offsets[b]:offsets[b + 1]] = out[i, :lens[b]]
        pending = pending[~ok]
    if pending.size:
        raise RuntimeError(f"{pending.size} random walks never ended in a final state")
    return Strings(ids, offsets)


def make_config(name: str, scale: float = 1.0, strings: int | None = None,
                kind: str = "walk", seed_offset: int = 0):
    """Build workload ``name`` (c1..c5).  ``scale`` < 1 shrinks states, symbols
    and arcs by the same factor (for CPU-sized cases); ``strings`` overrides
    the batch size.  Returns (FstArrays, Strings)."""
    cfg = CONFIGS[name]
    i = int(name[1:])
    q = max(8, int(round(cfg["num_states"] * scale)))
    s = max(4, int(round(cfg["num_isyms"] * scale)))
    o = max(4, int(round(cfg["num_osyms"] * scale)))
    a = max(16, int(round(cfg["num_arcs"] * scale)))
    md = cfg["mean_degree"]
    fst = random_fst(q, s, o, a, label_law=cfg["label_law"], src_law=cfg["src_law"],
                     mean_degree=md, dirichlet=cfg["dirichlet"],
                     seed=FST_SEED_BASE + i + seed_offset)
    nb = cfg["strings"] if strings is None else strings
    strs = make_strings(fst, nb, cfg["len_lo"], cfg["len_hi"],
                        seed=STRING_SEED_BASE + i + seed_offset, kind=kind,
                        label_law=cfg["label_law"])
    return fst, strs


def fig1_fst() -> FstArrays:
    """The FST of Fig. 1 with the arc arrays of Fig. 2 (S, T, O, P; R = [0,2,4,6]).

    Input symbols: le=0, chat=1, </s>=2.  Output symbols: the=0, a=1, cat=2,
    </s>=3.  State 0 is the start; state 5 is final with weight 1 (the figure
    marks no accepting state; this is the reading that makes "le chat </s>"
    accepted)."""
    src = np.array([0, 0, 1, 2, 3, 4], np.int32)
    dst = np.array([1, 2, 3, 4, 5, 5], np.int32)
    il = np.array([0, 0, 1, 1, 2, 2], np.int32)
    ol = np.array([0, 1, 2, 2, 3, 3], np.int32)
    p = np.array([0.48, 0.08, 1, 1, 1, 1], np.float64)
    w = (-np.log(p)).astype(np.float32)
    start = np.full(6, np.inf, np.float32)
    start[0] = 0.0
    final = np.full(6, np.inf, np.float32)
    final[5] = 0.0
    return FstArrays(6, 3, 4, src, dst, il, ol, w, start, final)


def hmm_fst(pi: np.ndarray, trans: np.ndarray, emit: np.ndarray) -> FstArrays:
    """Encode a K-state HMM (initial pi[K], transitions trans[K,K], emissions
    emit[K,V]) as an FST: state 0 is a fresh start state, state j+1 is hidden
    state j; arc (i -> j+1, label v) carries p = trans[i,j] * emit[j,v] (or
    pi[j] * emit[j,v] out of the start state).  Every hidden state is final
    with weight 1.  Arc order: start arcs first, then by (i, j, v)."""
    k, v = emit.shape
    src, dst, il, p = [], [], [], []
    for j in range(k):
        for o in range(v):
            src.append(0); dst.append(j + 1); il.append(o); p.append(pi[j] * emit[j, o])
    for i in range(k):
        for j in range(k):
            for o in range(v):
                src.append(i + 1); dst.append(j + 1); il.append(o)
                p.append(trans[i, j] * emit[j, o])
    p = np.asarray(p, np.float64)
    w = (-np.log(p)).astype(np.float32)
    q = k + 1
    start = np.full(q, np.inf, np.float32)
    start[0] = 0.0
    final = np.zeros(q, np.float32)
    final[0] = np.inf
    a = len(src)
    return FstArrays(q, v, v, np.asarray(src, np.int32), np.asarray(dst, np.int32),
                     np.asarray(il, np.int32), np.asarray(il, np.int32), w, start, final)


def tiny_fst(rng: np.random.Generator, max_states: int = 6, max_syms: int = 3,
             max_arcs: int = 14, multi_start: bool = True) -> FstArrays:
    """A tiny random FST for exhaustive checks: parallel arcs, self loops,
    several start states and random finals (costs in [0, 3))."""
    q = int(rng.integers(1, max_states + 1))
    s = int(rng.integers(1, max_syms + 1))
    a = int(rng.integers(1, max_arcs + 1))
    src = rng.integers(0, q, size=a).astype(np.int32)
    dst = rng.integers(0, q, size=a).astype(np.int32)
    il = rng.integers(0, s, size=a).astype(np.int32)
    ol = rng.integers(0, 4, size=a).astype(np.int32)
    w = (rng.random(a) * 3.0).astype(np.float32)
    start = np.full(q, np.inf, np.float32)
    start[0] = 0.0
    if multi_start and q > 1:
        extra = rng.random(q) < 0.3
        start[extra] = (rng.random(int(extra.sum())) * 2.0).astype(np.float32)
    final = np.where(rng.random(q) < 0.5, (rng.random(q) * 2.0), np.inf).astype(np.float32)
    if not np.isfinite(final).any():
        final[int(rng.integers(0, q))] = 0.0
    return FstArrays(q, s, 4, src, dst, il, ol, w, start, final)
