"""CPU oracle for FST Viterbi and forward-backward (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The arithmetic lives in ``oracle.c`` (plain C, compiled on first use into
``oracle/_build/liboracle.so``); this module only marshals numpy arrays,
except for ``Fst.clamped``, which writes down the output-clamped problem of
a pair (x, y) by its definition (the arcs read the pair of their input and
output labels) so that ``forward_backward_clamped`` is the pinned
forward-backward of that problem.  Pins: brute-force enumeration of the paths
of x that write y, and sum_y Z(x, y) = Z(x).
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
    """theta = -w in float32, +inf cost -> -inf, and -0.0 -> +0.0."""
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
        """Returns dict(status, best (float32), final_state, path[n] arc ids,
        olabels[n]) and, with tables=True, V[(n+1),Q] and bp[n,Q]."""
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
        """Returns dict(status, logz (float64), counts[A] float64) and, with
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
        """Weighted sums over a batch of state_posteriors (weight 1 by
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
        """EM re-estimation (see oracle_em_update in oracle.c): float64 log-weights
        theta'_k = log((count_k + alpha) / sum over the arcs of src_k of
        (count + alpha)); states with a zero total keep their old weights."""
        c = np.ascontiguousarray(counts, np.float64)
        out = np.zeros(max(self.A, 1), np.float64)
        rc = self.lib.oracle_em_update(self.Q, self.A, self.src, c, self.theta, float(alpha), out)
        if rc:
            raise RuntimeError(f"oracle_em_update failed: {rc}")
        return out[:self.A]

    def clamped(self, x, y):
        """The output-clamped problem of (x, y): the paths that read x and
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
