"""Frontier sizes on the host, by plain set reachability (no weights).

The live states of a string at position t are the states some path from a
start state reaches by reading w_1..w_t.  Which strings have the largest
frontiers decides which strings the full-size parity tests pick: the
kernels change regime (flattened walks, aggregated atomics, large staging
ranges) exactly there.  This is test infrastructure: it uses numpy only and
shares nothing with the CUDA path or the oracle's arithmetic.
"""
from __future__ import annotations

import numpy as np


class Reach:
    """Arcs sorted by (input symbol, source) for range lookups."""

    def __init__(self, fa):
        self.Q = int(fa.num_states)
        key = fa.ilabel.astype(np.int64) * self.Q + fa.src.astype(np.int64)
        order = np.argsort(key, kind="stable")
        self.key = key[order]
        self.dst = fa.dst[order].astype(np.int64)
        self.starts = np.flatnonzero(np.isfinite(fa.start_weight)).astype(np.int64)

    def live_counts(self, x) -> tuple[np.ndarray, np.ndarray]:
        """Per position t = 1..n: live states after reading w_t, and the arcs
        out of the live states of t-1 on w_t (the pushes of position t)."""
        live = self.starts
        n = len(x)
        lc = np.zeros(n, np.int64)
        ac = np.zeros(n, np.int64)
        for t in range(n):
            k = int(x[t]) * self.Q + live
            lo = np.searchsorted(self.key, k, "left")
            hi = np.searchsorted(self.key, k, "right")
            cnt = hi - lo
            tot = int(cnt.sum())
            ac[t] = tot
            if tot == 0:
                live = live[:0]
                continue
            rep = np.repeat(lo - np.cumsum(cnt) + cnt, cnt) + np.arange(tot)
            live = np.unique(self.dst[rep])
            lc[t] = live.size
        return lc, ac


def frontier_table(fa, strs, limit=None):
    """Largest live count and total pushes of each string (first ``limit``)."""
    r = Reach(fa)
    B = strs.count if limit is None else min(limit, strs.count)
    mx = np.zeros(B, np.int64)
    pushes = np.zeros(B, np.int64)
    for b in range(B):
        lc, ac = r.live_counts(strs.get(b))
        mx[b] = lc.max() if lc.size else 0
        pushes[b] = ac.sum()
    return mx, pushes
