"""CPU oracle for FST Viterbi and forward-backward (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The arithmetic lives in ``oracle.c`` (plain C, compiled on first use into
``oracle/_build/liboracle.so``); this module only marshals numpy arrays,
except for ``Fst.clamped``, which writes down the output-clamped problem of
a pair (x, y) by its definition (the arcs read the pair of their input and
output labels) so that ``forward_backward_clamped`` is the pinned
forward-backward of that problem.  Pins: brute-force enumeration of the paths
of x that write y, and sum_y Z(x, y) = Z(x).  ``lattice_viterbi`` and
``lattice_forward_backward`` (an acyclic input lattice composed with the
FST, Sec. 6.1) are plain loops over the edges in node order, pinned by the
linear lattice of a string (which must decode exactly as the string) and by
brute force over every (lattice path, FST path) pair.
Inputs are FSTs in the cost domain (w = -log p), as produced by
``paper_1701_03038_gb300.synth``; they are turned into natural-log weights
theta = -w here, with -0.0 stored as +0.0 and +inf costs as -inf.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, NO_PATH, OOM = 0, 1, 2, 3

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread"]


def build(force: bool = False, lib_path: str = _LIB_PATH, extra=()) -> str:
    """Compile oracle.c with gcc (no FMA contraction) into ``lib_path``."""
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    if (not force and os.path.exists(lib_path)
            and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC) and not extra):
        return lib_path
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *extra, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


def _declare(lib):
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
    vp = C.c_void_p
    fst = [C.c_int32, C.c_int64, i32p, i32p, i32p, f32p, f32p, f32p, C.c_int32]
    lib.oracle_viterbi.argtypes = fst + [i32p, C.c_int32, f32p, i32p, i32p, vp, vp]
    lib.oracle_forward_backward.argtypes = fst + [i32p, C.c_int32, f64p, vp, vp, vp]
    lib.oracle_viterbi_batch.argtypes = fst + [i32p, i64p, C.c_int32, C.c_int32, f32p, i32p, i32p]
    lib.oracle_fb_batch.argtypes = fst + [i32p, i64p, C.c_int32, C.c_int32, vp, f64p, vp, i32p]
    lib.oracle_em_update.argtypes = [C.c_int32, C.c_int64, i32p, f64p, f32p, C.c_double, f64p]
    for f in (lib.oracle_viterbi, lib.oracle_forward_backward, lib.oracle_viterbi_batch,
              lib.oracle_fb_batch, lib.oracle_em_update):
        f.restype = C.c_int
    return lib


def load(lib_path: str | None = None):
    """Load (building if needed) the oracle library."""
    global _lib
    if lib_path is not None:
        return _declare(C.CDLL(lib_path))
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def theta_of_cost(w) -> np.ndarray:
    """theta = -w in float32, +inf cost -> -inf, and -0.0 -> +0.0 (reading R1)."""
    t = -np.asarray(w, dtype=np.float32)
    t = t + np.float32(0.0)  # -0.0 + 0.0 == +0.0 under round-to-nearest
    return np.ascontiguousarray(t, dtype=np.float32)


class Fst:
    """An FST view for the oracle (theta domain)."""

    def __init__(self, fst, lib=None):
        self.Q = int(fst.num_states)
        self.A = int(fst.num_arcs)
        self.m = int(fst.num_isyms)
        self.src = np.ascontiguousarray(fst.src, np.int32)
        self.dst = np.ascontiguousarray(fst.dst, np.int32)
        self.ilabel = np.ascontiguousarray(fst.ilabel, np.int32)
        self.olabel = np.ascontiguousarray(fst.olabel, np.int32)
        self.theta = theta_of_cost(fst.weight)
        self.theta_s = theta_of_cost(fst.start_weight)
        self.theta_f = theta_of_cost(fst.final_weight)
        self.lib = lib if lib is not None else load()

    def _args(self):
        return (self.Q, self.A, self.src, self.dst, self.ilabel, self.theta, self.theta_s,
                self.theta_f, self.m)

    def viterbi(self, x, tables: bool = False):
        """Alg. 1 (Sec. 5.1) on one string.  Returns dict(status, best
        (float32), final_state, path[n] arc ids, olabels[n]) and, with
        tables=True, V[(n+1),Q] and bp[n,Q]."""
        x = np.ascontiguousarray(x, np.int32)
        n = int(x.shape[0])
        best = np.zeros(1, np.float32)
        qf = np.zeros(1, np.int32)
        path = np.zeros(max(n, 1), np.int32)
        V = np.zeros((n + 1, self.Q), np.float32) if tables else None
        bp = np.zeros((max(n, 1), self.Q), np.int32) if tables else None
        rc = self.lib.oracle_viterbi(*self._args(), x, n, best, qf, path, _ptr(V), _ptr(bp))
        if rc in (INVALID, OOM):
            raise RuntimeError(f"oracle_viterbi failed: {rc}")
        path = path[:n]
        out = dict(status=rc, best=best[0], final_state=int(qf[0]), path=path,
                   olabels=np.where(path >= 0, self.olabel[np.maximum(path, 0)], -1).astype(np.int32))
        if tables:
            out["V"] = V
            out["bp"] = bp[:n]
        return out

    def forward_backward(self, x, tables: bool = False):
        """Alg. 2 (Sec. 5.2) on one string.  Returns dict(status, logz (float64), counts[A] float64) and, with
        tables=True, alpha and beta [(n+1), Q] float64."""
        x = np.ascontiguousarray(x, np.int32)
        n = int(x.shape[0])
        logz = np.zeros(1, np.float64)
        counts = np.zeros(max(self.A, 1), np.float64)
        al = np.zeros((n + 1, self.Q), np.float64) if tables else None
        be = np.zeros((n + 1, self.Q), np.float64) if tables else None
        rc = self.lib.oracle_forward_backward(*self._args(), x, n, logz, _ptr(counts), _ptr(al), _ptr(be))
        if rc in (INVALID, OOM):
            raise RuntimeError(f"oracle_forward_backward failed: {rc}")
        out = dict(status=rc, logz=float(logz[0]), counts=counts[:self.A])
        if tables:
            out["alpha"] = al
            out["beta"] = be
        return out

    def state_posteriors(self, x):
        """Expected start and final state of string x, the two ends of
        Alg. 2: P(the path starts in q | x) = exp(alpha_0[q] + beta_0[q] -
        log Z) and P(it ends in q | x) = exp(alpha_n[q] + beta_n[q] - log Z),
        which are also d log Z / d (start log-weight of q) and d log Z /
        d (final log-weight of q).  All zero when x has no path."""
        x = np.ascontiguousarray(x, np.int32)
        n = int(x.shape[0])
        fb = self.forward_backward(x, tables=True)
        lz = fb["logz"]
        if lz == -np.inf:
            z = np.zeros(self.Q, np.float64)
            return dict(status=fb["status"], logz=lz, start=z, final=z.copy())
        al, be = fb["alpha"], fb["beta"]
        with np.errstate(invalid="ignore"):
            start = np.exp(al[0] + be[0] - lz)
            final = np.exp(al[n] + be[n] - lz)
        return dict(status=fb["status"], logz=lz, start=np.nan_to_num(start), final=np.nan_to_num(final))

    def state_posteriors_batch(self, ids, offsets, weights=None):
        """Weighted sums over a batch of state_posteriors (reading R14; weight 1 by
        default): the gradients of sum_b g_b log Z_b."""
        off = np.asarray(offsets, np.int64)
        start = np.zeros(self.Q, np.float64)
        final = np.zeros(self.Q, np.float64)
        for b in range(int(off.shape[0] - 1)):
            r = self.state_posteriors(np.asarray(ids)[off[b]:off[b + 1]])
            g = 1.0 if weights is None else float(weights[b])
            start += g * r["start"]
            final += g * r["final"]
        return dict(start=start, final=final)

    def viterbi_batch(self, ids, offsets, nthreads: int = 1):
        """Alg. 1 on every string of a batch (threads over strings)."""
        ids = np.ascontiguousarray(ids, np.int32)
        off = np.ascontiguousarray(offsets, np.int64)
        B = int(off.shape[0] - 1)
        best = np.zeros(max(B, 1), np.float32)
        paths = np.zeros(max(int(off[-1]), 1), np.int32)
        status = np.zeros(max(B, 1), np.int32)
        rc = self.lib.oracle_viterbi_batch(*self._args(), ids, off, B, int(nthreads), best, paths, status)
        if rc:
            raise RuntimeError(f"oracle_viterbi_batch failed: {rc}")
        return dict(best=best[:B], paths=paths[:int(off[-1])], status=status[:B])

    def fb_batch(self, ids, offsets, nthreads: int = 1, weights=None, counts: bool = True):
        """Alg. 2 on every string of a batch (threads over strings): log Z per
        string and sum_b weights[b] count_b (reading R10)."""
        ids = np.ascontiguousarray(ids, np.int32)
        off = np.ascontiguousarray(offsets, np.int64)
        B = int(off.shape[0] - 1)
        logz = np.zeros(max(B, 1), np.float64)
        cs = np.zeros(max(self.A, 1), np.float64) if counts else None
        status = np.zeros(max(B, 1), np.int32)
        w = None if weights is None else np.ascontiguousarray(weights, np.float64)
        rc = self.lib.oracle_fb_batch(*self._args(), ids, off, B, int(nthreads), _ptr(w), logz,
                                      _ptr(cs), status)
        if rc:
            raise RuntimeError(f"oracle_fb_batch failed: {rc}")
        return dict(logz=logz[:B], counts=None if cs is None else cs[:self.A], status=status[:B])

    # ------------------------------------------------------------ training
    def em_update(self, counts, alpha: float = 0.0) -> np.ndarray:
        """EM re-estimation (Sec. 4; oracle_em_update in oracle.c): float64 log-weights
        theta'_k = log((count_k + alpha) / sum over the arcs of src_k of
        (count + alpha)); states with a zero total keep their old weights."""
        c = np.ascontiguousarray(counts, np.float64)
        out = np.zeros(max(self.A, 1), np.float64)
        rc = self.lib.oracle_em_update(self.Q, self.A, self.src, c, self.theta, float(alpha), out)
        if rc:
            raise RuntimeError(f"oracle_em_update failed: {rc}")
        return out[:self.A]

    def clamped(self, x, y):
        """The output-clamped problem of (x, y) (reading R18): the paths that read x and
        write y are the paths of the FST whose arc k reads the pair
        (ilabel_k, olabel_k), run on the string of pairs (x_t, y_t).  Returns
        (an Fst view of that FST, the pair string); a pair no arc carries maps
        to a symbol without arcs.  Arc ids, weights and states are unchanged,
        so counts stay per original arc."""
        x = np.asarray(x, np.int64)
        y = np.asarray(y, np.int64)
        if x.shape != y.shape:
            raise ValueError("x and y differ in length")
        pairs = {}
        lab = np.zeros(self.A, np.int32)
        for k in range(self.A):
            key = (int(self.ilabel[k]), int(self.olabel[k]))
            lab[k] = pairs.setdefault(key, len(pairs))
        absent = len(pairs)
        xs = np.array([pairs.get((int(a), int(b)), absent) for a, b in zip(x, y)], np.int32)
        v = Fst.__new__(Fst)
        v.Q, v.A, v.m = self.Q, self.A, absent + 1
        v.src, v.dst, v.ilabel, v.olabel = self.src, self.dst, lab, self.olabel
        v.theta, v.theta_s, v.theta_f, v.lib = self.theta, self.theta_s, self.theta_f, self.lib
        return v, xs

    def forward_backward_clamped(self, x, y):
        """log Z(x, y) (the total weight of the paths reading x and writing
        y) and the arc posteriors given both: forward-backward of the
        output-clamped problem."""
        v, xs = self.clamped(x, y)
        return v.forward_backward(xs)


# ---------------------------------------------------------------- lattices
class Lattice:
    """An acyclic input lattice: nodes 0..num_nodes-1, node 0 the start and
    node num_nodes-1 the end; edge e goes from frm[e] to to[e] > frm[e],
    reads symbol label[e] and carries log-weight weight[e] (float32)."""

    def __init__(self, num_nodes, frm, to, label, weight):
        self.N = int(num_nodes)
        self.frm = np.asarray(frm, np.int64)
        self.to = np.asarray(to, np.int64)
        self.label = np.asarray(label, np.int64)
        self.weight = np.asarray(weight, np.float32)
        self.E = int(self.frm.shape[0])
        if self.N < 1 or np.any(self.frm >= self.to) or np.any(self.frm < 0) or np.any(self.to >= self.N):
            raise ValueError("edges must go from a lower to a higher node id within [0, num_nodes)")

    @classmethod
    def from_string(cls, x):
        """The linear lattice of a string: edge t reads x_t, weight 0."""
        n = len(x)
        return cls(n + 1, np.arange(n), np.arange(1, n + 1), np.asarray(x), np.zeros(n, np.float32))


def lattice_viterbi(o: Fst, lat: Lattice):
    """Viterbi (Alg. 1) over an input lattice (Sec. 6.1) composed with the
    FST, node by node in id order (a topological order), float32 as the
    string case: a candidate
    through edge e = (u -> v) and arc k is fl(fl(V[u][src_k] + theta_k) +
    w_e); the best wins, ties to the lowest arc id, then the lowest edge id.
    At the end node the best state adds its final weight (lowest state on
    ties).  Returns dict(status, best, edges[L], arcs[L]) along the best
    path (L = its number of edges)."""
    Q, N = o.Q, lat.N
    NEG = np.float32(-np.inf)
    V = np.full((N, Q), NEG, np.float32)
    V[0] = o.theta_s
    bk = np.full((N, Q), -1, np.int64)  # best arc
    be = np.full((N, Q), -1, np.int64)  # its edge
    by_label = {}
    for k in range(o.A):
        by_label.setdefault(int(o.ilabel[k]), []).append(k)
    order = np.lexsort((np.arange(lat.E), lat.to))  # by destination node, then edge id
    for e in order:
        u, v, w = int(lat.frm[e]), int(lat.to[e]), np.float32(lat.weight[e])
        for k in by_label.get(int(lat.label[e]), []):
            s, d = int(o.src[k]), int(o.dst[k])
            if V[u][s] == NEG:
                continue
            c = np.float32(np.float32(V[u][s] + o.theta[k]) + w)
            if c == NEG:
                continue
            if c > V[v][d] or (c == V[v][d] and k < bk[v][d]):
                V[v][d], bk[v][d], be[v][d] = c, k, e
    best, qb = NEG, -1
    for q in range(Q):
        c = np.float32(V[N - 1][q] + o.theta_f[q])
        if c > best:
            best, qb = c, q
    if qb < 0:
        return dict(status=NO_PATH, best=NEG, edges=np.zeros(0, np.int32), arcs=np.zeros(0, np.int32))
    edges, arcs = [], []
    v, q = N - 1, qb
    while v != 0 or bk[v][q] >= 0:
        k, e = int(bk[v][q]), int(be[v][q])
        if k < 0:
            break
        edges.append(e)
        arcs.append(k)
        v, q = int(lat.frm[e]), int(o.src[k])
    return dict(status=OK, best=best, edges=np.array(edges[::-1], np.int32), arcs=np.array(arcs[::-1], np.int32))


def _lse(v):
    v = np.asarray(v, np.float64)
    if v.size == 0:
        return -np.inf
    m = v.max()
    if m == -np.inf:
        return -np.inf
    return float(m + np.log(np.exp(v - m).sum()))


def lattice_forward_backward(o: Fst, lat: Lattice):
    """Forward-backward over an input lattice composed with the FST, float64:
    alpha[v][q'] = LSE over edges e = (u -> v) and arcs k = (q -> q') on the
    edge's symbol of alpha[u][q] + w_e + theta_k (alpha[0] = theta_s);
    beta[u][q] likewise towards the end node (beta[N-1] = theta_f); log Z =
    LSE_q(alpha[N-1][q] + theta_f[q]); the posterior of arc k is the sum over
    the edges reading its symbol of exp(alpha[u][src_k] + w_e + theta_k +
    beta[v][dst_k] - log Z), and that of edge e the sum over its arcs.
    Returns dict(status, logz, counts[A], edge_post[E])."""
    Q, N = o.Q, lat.N
    th = o.theta.astype(np.float64)
    al = np.full((N, Q), -np.inf)
    al[0] = o.theta_s.astype(np.float64)
    be = np.full((N, Q), -np.inf)
    be[N - 1] = o.theta_f.astype(np.float64)
    arcs_of = {a: np.flatnonzero(o.ilabel == a) for a in set(lat.label.tolist())}
    into = [[e for e in range(lat.E) if lat.to[e] == v] for v in range(N)]
    outof = [[e for e in range(lat.E) if lat.frm[e] == v] for v in range(N)]
    for v in range(1, N):
        terms = [[] for _ in range(Q)]
        for e in into[v]:
            u, w = int(lat.frm[e]), float(lat.weight[e])
            for k in arcs_of[int(lat.label[e])]:
                terms[int(o.dst[k])].append(al[u][o.src[k]] + w + th[k])
        al[v] = [_lse(t) for t in terms]
    for v in range(N - 2, -1, -1):
        terms = [[] for _ in range(Q)]
        for e in outof[v]:
            t, w = int(lat.to[e]), float(lat.weight[e])
            for k in arcs_of[int(lat.label[e])]:
                terms[int(o.src[k])].append(w + th[k] + be[t][o.dst[k]])
        be[v] = [_lse(x) for x in terms]
    logz = _lse(al[N - 1] + o.theta_f.astype(np.float64))
    counts = np.zeros(o.A)
    epost = np.zeros(lat.E)
    if logz > -np.inf:
        for e in range(lat.E):
            u, v, w = int(lat.frm[e]), int(lat.to[e]), float(lat.weight[e])
            for k in arcs_of[int(lat.label[e])]:
                g = np.exp(al[u][o.src[k]] + w + th[k] + be[v][o.dst[k]] - logz)
                counts[k] += g
                epost[e] += g
    return dict(status=OK if logz > -np.inf else NO_PATH, logz=logz, counts=counts, edge_post=epost)
