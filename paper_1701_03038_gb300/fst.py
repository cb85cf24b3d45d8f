"""Python front end of libfstgpu: FST handles, single-string calls and batch
plans.  Argument marshalling only -- every step runs in the CUDA library;
PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check

__all__ = ["Fst", "Plan"]


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Fst:
    """An epsilon-free weighted FST resident on one GPU.

    Arrays are given in the caller's arc order; weights are costs
    (``weight_kind="cost"``, w = -log p) or log-weights (``"log"``).  Host
    numpy arrays or CUDA tensors are accepted (all of one kind).
    """

    def __init__(self, num_states, src, dst, ilabel, olabel, weight, start_weight, final_weight,
                 num_isyms, weight_kind: str = "cost", device=None):
        self._lib = _lib.load()
        self._h = None
        kind = {"cost": _lib.WEIGHT_COST, "log": _lib.WEIGHT_LOG}[weight_kind]
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        on_device = isinstance(src, torch.Tensor)
        h = C.c_void_p()
        with torch.cuda.device(dev):
            if on_device:
                arrs = [src, dst, ilabel, olabel, weight, start_weight, final_weight]
                dts = [torch.int32] * 4 + [torch.float32] * 3
                arrs = [a.to(device=dev, dtype=d).contiguous() for a, d in zip(arrs, dts)]
                keep = arrs
                ptrs = [_dptr(a) for a in arrs]
                flags = _lib.FLAG_DEVICE_PTRS
                na = int(arrs[0].numel())
            else:
                arrs = [_host(src, np.int32), _host(dst, np.int32), _host(ilabel, np.int32),
                        _host(olabel, np.int32), _host(weight, np.float32),
                        _host(start_weight, np.float32), _host(final_weight, np.float32)]
                keep = arrs
                ptrs = [_hptr(a) for a in arrs]
                flags = 0
                na = int(arrs[0].shape[0])
            rc = self._lib.fst_create(int(num_states), na, ptrs[0], ptrs[1], ptrs[2], ptrs[3], ptrs[4],
                                      kind, ptrs[5], ptrs[6], int(num_isyms), flags, C.byref(h))
            del keep
            check(rc, "fst_create")
        self._h = h
        self.num_states = int(num_states)
        self.num_arcs = na
        self.num_isyms = int(num_isyms)

    @classmethod
    def _wrap(cls, handle, num_states: int, num_arcs: int, num_isyms: int, device) -> "Fst":
        """An Fst object around a handle the library made (e.g. fst_create_clamped)."""
        f = cls.__new__(cls)
        f._lib = _lib.load()
        f._h = handle
        f.device = device
        f.num_states, f.num_arcs, f.num_isyms = int(num_states), int(num_arcs), int(num_isyms)
        return f

    @classmethod
    def from_arrays(cls, fa, device=None) -> "Fst":
        """Build from a ``synth.FstArrays`` (cost-domain weights)."""
        return cls(fa.num_states, fa.src, fa.dst, fa.ilabel, fa.olabel, fa.weight, fa.start_weight,
                   fa.final_weight, fa.num_isyms, weight_kind="cost", device=device)

    @classmethod
    def from_att(cls, source, isyms=None, osyms=None, device=None, **kw) -> "Fst":
        """Build from OpenFst / AT&T text (a path, text or file object; see
        ``att.read_att`` for the symbol tables and options)."""
        from . import att
        return cls.from_arrays(att.read_att(source, isyms, osyms, **kw), device=device)

    def close(self):
        if self._h is not None and self._h.value:
            self._lib.fst_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------ queries
    def info(self) -> dict:
        q, m = C.c_int32(), C.c_int32()
        a, p, w, ds, ss = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        check(self._lib.fst_info(self._h, C.byref(q), C.byref(a), C.byref(m), C.byref(p), C.byref(w),
                                 C.byref(ds), C.byref(ss)), "fst_info")
        return dict(num_states=q.value, num_arcs=a.value, num_isyms=m.value, padded_arcs=p.value,
                    windows=w.value, dst_segments=ds.value, src_segments=ss.value)

    def symbol_stats(self):
        """(|delta[a]|, D_a distinct destinations, U_a distinct sources) per symbol."""
        arcs = np.zeros(self.num_isyms, np.int64)
        dsts = np.zeros(self.num_isyms, np.int64)
        srcs = np.zeros(self.num_isyms, np.int64)
        check(self._lib.fst_symbol_stats(self._h, _hptr(arcs), _hptr(dsts), _hptr(srcs)), "fst_symbol_stats")
        return arcs, dsts, srcs

    def set_weights(self, weight, weight_kind: str = "cost"):
        kind = {"cost": _lib.WEIGHT_COST, "log": _lib.WEIGHT_LOG}[weight_kind]
        if isinstance(weight, torch.Tensor):
            w = weight.detach().to(device=self.device, dtype=torch.float32).contiguous()
            with torch.cuda.device(self.device):
                torch.cuda.current_stream().synchronize()
                check(self._lib.fst_set_weights(self._h, _dptr(w), kind, _lib.FLAG_DEVICE_PTRS),
                      "fst_set_weights")
        else:
            w = _host(weight, np.float32)
            with torch.cuda.device(self.device):
                check(self._lib.fst_set_weights(self._h, _hptr(w), kind, 0), "fst_set_weights")

    def set_state_weights(self, start=None, final=None, weight_kind: str = "cost"):
        """Replace the start and/or final weight of every state ([num_states]
        each; None keeps the old ones)."""
        kind = {"cost": _lib.WEIGHT_COST, "log": _lib.WEIGHT_LOG}[weight_kind]
        if any(isinstance(v, torch.Tensor) for v in (start, final)):
            vs = [None if v is None else torch.as_tensor(v).detach().to(device=self.device, dtype=torch.float32)
                  .contiguous() for v in (start, final)]
            with torch.cuda.device(self.device):
                torch.cuda.current_stream().synchronize()
                check(self._lib.fst_set_state_weights(self._h, _dptr(vs[0]), _dptr(vs[1]), kind,
                                                      _lib.FLAG_DEVICE_PTRS), "fst_set_state_weights")
        else:
            vs = [None if v is None else _host(v, np.float32) for v in (start, final)]
            with torch.cuda.device(self.device):
                check(self._lib.fst_set_state_weights(self._h, *[None if v is None else _hptr(v) for v in vs], kind, 0),
                      "fst_set_state_weights")

    # ------------------------------------------------- plain method (one string)
    def viterbi(self, ids):
        """Alg. 1 (Sec. 5.1): best path of one string: (score float32, arc ids int32[n], output
        labels int32[n], status).  Status NO_PATH means no accepting path."""
        x = _host(ids, np.int32)
        n = int(x.shape[0])
        best = np.zeros(1, np.float32)
        path = np.zeros(max(n, 1), np.int32)
        olab = np.zeros(max(n, 1), np.int32)
        with torch.cuda.device(self.device):
            rc = self._lib.fst_viterbi(self._h, _hptr(x), n, _hptr(best), _hptr(path), _hptr(olab))
        check(rc, "fst_viterbi", allow=(_lib.OK, _lib.NO_PATH))
        return best[0], path[:n], olab[:n], rc

    def viterbi_slice(self, ids):
        """The paper's relaxation of Sec. 5.1 (every arc of every slice, one thread per
        arc), for comparison: (score float32, arc ids int32[n], status),
        bit-identical to viterbi()."""
        x = _host(ids, np.int32)
        n = int(x.shape[0])
        best = np.zeros(1, np.float32)
        path = np.zeros(max(n, 1), np.int32)
        with torch.cuda.device(self.device):
            rc = self._lib.fst_viterbi_slice(self._h, _hptr(x), n, _hptr(best), _hptr(path))
        check(rc, "fst_viterbi_slice", allow=(_lib.OK, _lib.NO_PATH))
        return best[0], path[:n], rc

    def forward_backward_slice(self, ids, posteriors: bool = True):
        """The paper's forward-backward of Sec. 5.2 (every arc of every slice, atomic
        log-add-exp in float32), for comparison: (log Z, counts, status)."""
        x = _host(ids, np.int32)
        n = int(x.shape[0])
        lz = np.zeros(1, np.float64)
        cnt = np.zeros(max(self.num_arcs, 1), np.float32) if posteriors else None
        with torch.cuda.device(self.device):
            rc = self._lib.fst_forward_backward_slice(self._h, _hptr(x), n, _hptr(lz),
                                                      _hptr(cnt) if posteriors else None)
        check(rc, "fst_forward_backward_slice", allow=(_lib.OK, _lib.NO_PATH))
        return float(lz[0]), (cnt[:self.num_arcs] if posteriors else None), rc

    def set_plain_method(self, method: int):
        """Kernels of the single-string calls: _lib.PLAIN_FRONTIER, PLAIN_SLICE,
        PLAIN_AUTO or PLAIN_BLOCK (see fst_set_plain_method)."""
        check(self._lib.fst_set_plain_method(self._h, int(method)), "fst_set_plain_method")

    def set_plain_driver(self, driver: int, grid_blocks: int = 0):
        """Driver of the single-string forward-backward: _lib.DRIVER_LAUNCH or
        _lib.DRIVER_PERSISTENT (see fst_set_plain_driver)."""
        with torch.cuda.device(self.device):
            check(self._lib.fst_set_plain_driver(self._h, int(driver), int(grid_blocks)), "fst_set_plain_driver")

    def plain_method(self) -> dict:
        """What the single-string calls take now (fst_get_plain_method):
        {"method", "driver", "grid_blocks"}."""
        m, d, g = C.c_int32(), C.c_int32(), C.c_int32()
        check(self._lib.fst_get_plain_method(self._h, C.byref(m), C.byref(d), C.byref(g)), "fst_get_plain_method")
        return {"method": m.value, "driver": d.value, "grid_blocks": g.value}

    def autotune_plain(self, ids, offsets) -> np.ndarray:
        """Calibrate the automatic choice of the single-string Viterbi kernels on
        sample strings (see fst_autotune_plain); returns the fitted
        coefficients (d0, d1, c0, c1, c2) in microseconds."""
        x = _host(ids, np.int32)
        off = _host(offsets, np.int64)
        coef = np.zeros(5, np.float64)
        with torch.cuda.device(self.device):
            check(self._lib.fst_autotune_plain(self._h, _hptr(x), _hptr(off), int(off.shape[0] - 1), _hptr(coef)),
                  "fst_autotune_plain")
        return coef

    def set_slice_order(self, order: int):
        """Arc order within a slice for the paper-design calls:
        _lib.SLICE_BY_DESTINATION (column-major) or _lib.SLICE_BY_SOURCE (row-major)."""
        check(self._lib.fst_set_slice_order(self._h, int(order)), "fst_set_slice_order")

    def forward_backward(self, ids, posteriors: bool = True, out: np.ndarray | None = None):
        """Alg. 2 (Sec. 5.2) on one string: (log Z float64, expected arc counts float32[A] or None, status).
        ``out``, a C-contiguous float32 host array of at least A elements
        (for instance the numpy view of a pinned torch tensor, reused from
        call to call), receives the counts instead of a new array; the
        counts returned are its first A elements.  Passing ``out`` asks for
        the counts whatever ``posteriors`` says."""
        x = _host(ids, np.int32)
        n = int(x.shape[0])
        lz = np.zeros(1, np.float64)
        if out is not None:
            if (not isinstance(out, np.ndarray) or out.dtype != np.float32 or not out.flags.c_contiguous
                    or out.ndim != 1 or out.shape[0] < max(self.num_arcs, 1)):
                raise ValueError(f"out must be a contiguous float32 array of at least {max(self.num_arcs, 1)} elements")
            posteriors = True
        cnt = (out if out is not None else np.zeros(max(self.num_arcs, 1), np.float32)) if posteriors else None
        with torch.cuda.device(self.device):
            rc = self._lib.fst_forward_backward(self._h, _hptr(x), n, _hptr(lz),
                                                _hptr(cnt) if posteriors else None)
        check(rc, "fst_forward_backward", allow=(_lib.OK, _lib.NO_PATH))
        return float(lz[0]), (cnt[:self.num_arcs] if posteriors else None), rc

    def log_z_f64(self, ids, theta=None) -> float:
        """log Z of one string in float64 (finite-difference checks).
        ``theta``: float64 log-weights [A] in caller order, or None to reuse
        the previous call's."""
        x = _host(ids, np.int32)
        lz = np.zeros(1, np.float64)
        th = None if theta is None else _host(theta, np.float64)
        with torch.cuda.device(self.device):
            check(self._lib.fst_log_z_f64(self._h, None if th is None else _hptr(th), _hptr(x), int(x.shape[0]),
                                          _hptr(lz)), "fst_log_z_f64")
        return float(lz[0])

    # ------------------------------------------------------------ lattices
    @staticmethod
    def _lattice_args(num_nodes, frm, to, label, weight):
        arrs = [_host(frm, np.int32), _host(to, np.int32), _host(label, np.int32), _host(weight, np.float32)]
        e = int(arrs[0].shape[0])
        if any(int(a.shape[0]) != e for a in arrs):
            raise ValueError("lattice arrays differ in length")
        return int(num_nodes), e, arrs

    def lattice_viterbi(self, num_nodes, frm, to, label, weight):
        """Best (lattice path, FST path) of an acyclic input lattice (Sec. 6.1; see
        fst_lattice_viterbi): (score float32, edges int32[L], arcs int32[L], status)."""
        n, e, (a, b, c, d) = self._lattice_args(num_nodes, frm, to, label, weight)
        best = np.zeros(1, np.float32)
        ep = np.zeros(max(n - 1, 1), np.int32)
        ap = np.zeros(max(n - 1, 1), np.int32)
        ln = np.zeros(1, np.int32)
        with torch.cuda.device(self.device):
            rc = self._lib.fst_lattice_viterbi(self._h, n, e, _hptr(a), _hptr(b), _hptr(c), _hptr(d), _hptr(best),
                                               _hptr(ep), _hptr(ap), _hptr(ln))
        check(rc, "fst_lattice_viterbi", allow=(_lib.OK, _lib.NO_PATH))
        L = int(ln[0])
        return best[0], ep[:L], ap[:L], rc

    def lattice_forward_backward(self, num_nodes, frm, to, label, weight):
        """Alg. 2 over an input lattice (Sec. 6.1): (log Z, arc counts float32[A], edge posteriors float32[E], status)
        of an acyclic input lattice (see fst_lattice_forward_backward)."""
        n, e, (a, b, c, d) = self._lattice_args(num_nodes, frm, to, label, weight)
        lz = np.zeros(1, np.float64)
        cnt = np.zeros(max(self.num_arcs, 1), np.float32)
        ep = np.zeros(max(e, 1), np.float32)
        with torch.cuda.device(self.device):
            rc = self._lib.fst_lattice_forward_backward(self._h, n, e, _hptr(a), _hptr(b), _hptr(c), _hptr(d),
                                                        _hptr(lz), _hptr(cnt), _hptr(ep))
        check(rc, "fst_lattice_forward_backward", allow=(_lib.OK, _lib.NO_PATH))
        return float(lz[0]), cnt[:self.num_arcs], ep[:e], rc

    def prefix_log_z(self, ids):
        """(log Z, best score, status) of one string by the parallel product (Sec. 6.1) of
        its dense slice matrices (small dense FSTs; see fst_prefix_log_z)."""
        x = _host(ids, np.int32)
        lz = np.zeros(1, np.float64)
        best = np.zeros(1, np.float32)
        with torch.cuda.device(self.device):
            rc = self._lib.fst_prefix_log_z(self._h, _hptr(x), int(x.shape[0]), _hptr(lz), _hptr(best))
        check(rc, "fst_prefix_log_z", allow=(_lib.OK, _lib.NO_PATH))
        return float(lz[0]), best[0], rc

    # ------------------------------------------------------------ training
    def em_update(self, counts, pseudo_count: float = 0.0, apply: bool = False):
        """EM M-step (Sec. 4; fst_em_update): new log-weights, each state's outgoing
        arcs renormalised from their expected counts.  ``counts``: a CUDA
        float32 tensor (returns a CUDA tensor) or a host array (returns
        numpy).  ``apply`` also installs them as the FST's weights."""
        flags = _lib.EM_APPLY if apply else 0
        if isinstance(counts, torch.Tensor):
            c = counts.detach().to(device=self.device, dtype=torch.float32).contiguous()
            out = torch.empty(max(self.num_arcs, 1), dtype=torch.float32, device=self.device)
            with torch.cuda.device(self.device):
                torch.cuda.current_stream().synchronize()
                check(self._lib.fst_em_update(self._h, _dptr(c), float(pseudo_count), _dptr(out),
                                              flags | _lib.FLAG_DEVICE_PTRS), "fst_em_update")
            return out[:self.num_arcs]
        c = _host(counts, np.float32)
        out = np.zeros(max(self.num_arcs, 1), np.float32)
        with torch.cuda.device(self.device):
            check(self._lib.fst_em_update(self._h, _hptr(c), float(pseudo_count), _hptr(out), flags),
                  "fst_em_update")
        return out[:self.num_arcs]

    def clamped(self) -> "Fst":
        """The output-clamped FST (fst_create_clamped): same arcs and ids, input
        symbols = (input, output) label pairs; log Z(x, y) is its log Z on
        the pair string clamp(x, y)."""
        h = C.c_void_p()
        npairs = C.c_int32()
        with torch.cuda.device(self.device):
            check(self._lib.fst_create_clamped(self._h, C.byref(h), C.byref(npairs)), "fst_create_clamped")
        f = Fst._wrap(h, self.num_states, self.num_arcs, npairs.value + 1, self.device)
        f.num_pairs = npairs.value
        return f

    def clamp(self, ids, olabels) -> np.ndarray:
        """Pair string of an input string and an output string of the same
        length (for a clamped FST; see fst_clamp_labels)."""
        x = _host(ids, np.int32)
        y = _host(olabels, np.int32)
        if x.shape != y.shape:
            raise ValueError("ids and olabels differ in length")
        out = np.zeros(max(x.shape[0], 1), np.int32)
        check(self._lib.fst_clamp_labels(self._h, _hptr(x), _hptr(y), int(x.shape[0]), _hptr(out)),
              "fst_clamp_labels")
        return out[:x.shape[0]]

    # ------------------------------------------------------- measurement
    def profile(self, enable: bool = True):
        """Bracket every kernel of the following single-string calls with CUDA events."""
        check(self._lib.fst_profile(self._h, 1 if enable else 0), "fst_profile")

    def profile_read(self) -> dict:
        """{kind: (milliseconds, launches)} of the single-string calls since the last read."""
        ms = np.zeros(len(_lib.PROF_KINDS), np.float64)
        n = np.zeros(len(_lib.PROF_KINDS), np.int64)
        with torch.cuda.device(self.device):
            check(self._lib.fst_profile_read(self._h, _hptr(ms), _hptr(n)), "fst_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(_lib.PROF_KINDS)}

    def live_work(self) -> dict:
        """Live states and pushed arcs of the last single-string call (see fst_live_work)."""
        e, a = C.c_int64(), C.c_int64()
        with torch.cuda.device(self.device):
            check(self._lib.fst_live_work(self._h, C.byref(e), C.byref(a)), "fst_live_work")
        return dict(entries=e.value, arcs=a.value)

    # ------------------------------------------------------ batched method
    def set_batch_budget(self, nbytes: int):
        """Storage budget of the plans built by viterbi_batch and
        forward_backward_batch (0 = the library default)."""
        check(self._lib.fst_set_batch_budget(self._h, int(nbytes)), "fst_set_batch_budget")

    def set_batch_plan(self, parts_viterbi: int = 0, parts_fb: int = 0, layout: int = -1, graph: int = -1):
        """Plans of viterbi_batch and forward_backward_batch: stream-parallel
        parts (0 = by batch size), accumulators (-1 = dense when they fit
        the budget, 0 = compact, 1 = dense) and CUDA-graph launch (-1 = above
        256 launches, 0 = never, 1 = always); see fst_set_batch_plan."""
        check(self._lib.fst_set_batch_plan(self._h, int(parts_viterbi), int(parts_fb), int(layout), int(graph)),
              "fst_set_batch_plan")

    def plan(self, ids: torch.Tensor, offsets: torch.Tensor, mem_budget: int = 0, flags: int = 0,
             stream=None, parts: int = 1) -> "Plan":
        """A batch plan (see fst_plan_create); ``parts`` > 1 runs the batch as
        that many stream-parallel parts (FST_PLAN_PARTS)."""
        if parts > 1:
            flags |= (int(parts) & 0xFF) << 8
        return Plan(self, ids, offsets, mem_budget=mem_budget, flags=flags, stream=stream)

    def viterbi_batch(self, ids: torch.Tensor, offsets: torch.Tensor, stream=None):
        """Alg. 1 for every string of a batch (fst_viterbi_batch): dict of
        scores [B], paths [N], olabels [N], status [B] on the device."""
        _require_cuda(ids, torch.int32, "ids")
        _require_cuda(offsets, torch.int64, "offsets")
        B = int(offsets.numel()) - 1
        scores = torch.empty(max(B, 1), dtype=torch.float32, device=ids.device)
        paths = torch.empty(max(int(ids.numel()), 1), dtype=torch.int32, device=ids.device)
        olab = torch.empty_like(paths)
        status = torch.empty(max(B, 1), dtype=torch.int32, device=ids.device)
        with torch.cuda.device(self.device):
            check(self._lib.fst_viterbi_batch(self._h, _dptr(ids), _dptr(offsets), B, _dptr(scores),
                                              _dptr(paths), _dptr(olab), _dptr(status), _stream(stream)),
                  "fst_viterbi_batch")
        n = int(ids.numel())
        return dict(scores=scores[:B], paths=paths[:n], olabels=olab[:n], status=status[:B])

    def forward_backward_batch(self, ids: torch.Tensor, offsets: torch.Tensor, weights=None,
                               counts: bool = True, stream=None):
        """Alg. 2 for every string of a batch (fst_forward_backward_batch):
        dict of logz [B], counts [A] (sum_b weights[b] count_b, or None) and
        status [B] on the device."""
        _require_cuda(ids, torch.int32, "ids")
        _require_cuda(offsets, torch.int64, "offsets")
        B = int(offsets.numel()) - 1
        logz = torch.empty(max(B, 1), dtype=torch.float64, device=ids.device)
        status = torch.empty(max(B, 1), dtype=torch.int32, device=ids.device)
        cnt = torch.empty(max(self.num_arcs, 1), dtype=torch.float32, device=ids.device) if counts else None
        if weights is not None:
            _require_cuda(weights, torch.float32, "weights")
        with torch.cuda.device(self.device):
            check(self._lib.fst_forward_backward_batch(self._h, _dptr(ids), _dptr(offsets), B, _dptr(weights),
                                                       _dptr(logz), _dptr(cnt), _dptr(status), _stream(stream)),
                  "fst_forward_backward_batch")
        return dict(logz=logz[:B], counts=None if cnt is None else cnt[:self.num_arcs], status=status[:B])


class Plan:
    """Device work lists and storage for one batch (see fst_plan_create): the
    per-position loops of Alg. 1 and Alg. 2 (Sec. 5) for every string.
    Run calls allocate nothing and are safe to capture in a CUDA graph."""

    def __init__(self, fst: Fst, ids: torch.Tensor, offsets: torch.Tensor, mem_budget: int = 0,
                 flags: int = 0, stream=None):
        _require_cuda(ids, torch.int32, "ids")
        _require_cuda(offsets, torch.int64, "offsets")
        self.fst = fst
        self._lib = fst._lib
        self._h = None
        h = C.c_void_p()
        self.B = int(offsets.numel()) - 1
        self.N = int(ids.numel())
        with torch.cuda.device(fst.device):
            check(self._lib.fst_plan_create(fst.handle, _dptr(ids), _dptr(offsets), self.B, int(mem_budget),
                                            int(flags), _stream(stream), C.byref(h)), "fst_plan_create")
        self._h = h
        dev = fst.device
        self.scores = torch.empty(max(self.B, 1), dtype=torch.float32, device=dev)
        self.paths = torch.empty(max(self.N, 1), dtype=torch.int32, device=dev)
        self.olabels = torch.empty(max(self.N, 1), dtype=torch.int32, device=dev)
        self.status = torch.empty(max(self.B, 1), dtype=torch.int32, device=dev)
        self.logz = torch.empty(max(self.B, 1), dtype=torch.float64, device=dev)
        self.counts = torch.empty(max(fst.num_arcs, 1), dtype=torch.float32, device=dev)
        # expected start and final states (forward_backward / backward with states=True)
        self.start_counts = torch.empty(max(fst.num_states, 1), dtype=torch.float32, device=dev)
        self.final_counts = torch.empty(max(fst.num_states, 1), dtype=torch.float32, device=dev)

    def close(self):
        if self._h is not None and self._h.value:
            self._lib.fst_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        b, w, ml = C.c_int32(), C.c_int32(), C.c_int32()
        n, r, vl, fl, by = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        check(self._lib.fst_plan_info(self._h, C.byref(b), C.byref(n), C.byref(w), C.byref(ml), C.byref(r),
                                      C.byref(vl), C.byref(fl), C.byref(by)), "fst_plan_info")
        return dict(strings=b.value, tokens=n.value, waves=w.value, max_len=ml.value, relaxations=r.value,
                    viterbi_launches=vl.value, fb_launches=fl.value, device_bytes=by.value)

    def live_work(self, stream=None) -> dict:
        """Live states and pushed arcs of the last pass (see fst_plan_live_work)."""
        e, a = C.c_int64(), C.c_int64()
        check(self._lib.fst_plan_live_work(self._h, C.byref(e), C.byref(a), _stream(stream)), "fst_plan_live_work")
        return dict(entries=e.value, arcs=a.value)

    def set_driver(self, driver: int, grid_blocks: int = 0, barrier_timeout_us: int = 0):
        """Driver of the following runs: _lib.DRIVER_LAUNCH (one launch per
        position) or _lib.DRIVER_PERSISTENT (one cooperative launch per pass)."""
        with torch.cuda.device(self.fst.device):
            check(self._lib.fst_plan_set_driver(self._h, int(driver), int(grid_blocks), int(barrier_timeout_us)),
                  "fst_plan_set_driver")

    def autotune(self, refresh: bool = False, stream=None) -> dict:
        """Time the plan's pass under each driver configuration and keep the
        fastest (see fst_plan_autotune); returns the choice."""
        d, g, ms = C.c_int32(), C.c_int32(), C.c_double()
        with torch.cuda.device(self.fst.device):
            check(self._lib.fst_plan_autotune(self._h, _stream(stream), _lib.TUNE_REFRESH if refresh else 0,
                                              C.byref(d), C.byref(g), C.byref(ms)), "fst_plan_autotune")
        return dict(driver="persistent" if d.value == _lib.DRIVER_PERSISTENT else "launch", grid=g.value,
                    ms=ms.value)

    def driver(self) -> tuple[int, int]:
        d, g = C.c_int32(), C.c_int32()
        check(self._lib.fst_plan_get_driver(self._h, C.byref(d), C.byref(g)), "fst_plan_get_driver")
        return d.value, g.value

    def fault_inject(self, kind: int, value: int = 0):
        """Testing hook: _lib.FAULT_BARRIER_STALL makes the persistent passes'
        barriers wait for `value` blocks that do not exist (their waits time out)."""
        check(self._lib.fst_plan_fault_inject(self._h, int(kind), int(value)), "fst_plan_fault_inject")

    def limit_pool(self, entries: int = 0):
        """Cap the live pool of the following runs (0 = the full capacity)."""
        check(self._lib.fst_plan_limit_pool(self._h, int(entries)), "fst_plan_limit_pool")

    def set_pull(self, min_live: int = -1):
        """Direction switch of the forward pass (dense accumulators, launch
        driver): tokens with at least min_live live states pull (0 = off,
        the default; -1 = half the states); see fst_plan_set_pull."""
        check(self._lib.fst_plan_set_pull(self._h, int(min_live)), "fst_plan_set_pull")

    def limit_table(self, slots: int = 0):
        """Cap the compact accumulator tables of the following runs (0 = the full capacity)."""
        check(self._lib.fst_plan_limit_table(self._h, int(slots)), "fst_plan_limit_table")

    def table_slots(self) -> int:
        """Slots of each compact accumulator table (0: dense accumulators)."""
        n = C.c_int64()
        check(self._lib.fst_plan_table_slots(self._h, C.byref(n)), "fst_plan_table_slots")
        return n.value

    def profile(self, enable: bool = True):
        """Bracket every kernel of the following runs with CUDA events."""
        check(self._lib.fst_plan_profile(self._h, 1 if enable else 0), "fst_plan_profile")

    def profile_read(self) -> dict:
        """{kind: (milliseconds, launches)} accumulated since the last read."""
        ms = np.zeros(len(_lib.PROF_KINDS), np.float64)
        n = np.zeros(len(_lib.PROF_KINDS), np.int64)
        check(self._lib.fst_plan_profile_read(self._h, _hptr(ms), _hptr(n)), "fst_plan_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(_lib.PROF_KINDS)}

    def viterbi(self, stream=None):
        """Queue Viterbi (Alg. 1) for every string; results land in self.scores /
        self.paths / self.olabels / self.status."""
        check(self._lib.fst_plan_viterbi(self._h, _dptr(self.scores), _dptr(self.paths), _dptr(self.olabels),
                                         _dptr(self.status), _stream(stream)), "fst_plan_viterbi")

    def forward(self, stream=None):
        """Forward pass only (Alg. 2's forward loop): log Z into self.logz;
        the forward values stay in the plan for backward()."""
        check(self._lib.fst_plan_forward(self._h, _dptr(self.logz), _dptr(self.status), _stream(stream)),
              "fst_plan_forward")

    def backward(self, weights: torch.Tensor | None = None, stream=None, states: bool = False):
        """Backward pass (Alg. 2's backward and count loops) after forward(): arc counts into self.counts and,
        with states=True, expected start and final states into
        self.start_counts / self.final_counts."""
        if weights is not None:
            _require_cuda(weights, torch.float32, "weights")
        if states:
            check(self._lib.fst_plan_backward_ex(self._h, _dptr(weights), _dptr(self.counts),
                                                 _dptr(self.start_counts), _dptr(self.final_counts),
                                                 _stream(stream)), "fst_plan_backward_ex")
        else:
            check(self._lib.fst_plan_backward(self._h, _dptr(weights), _dptr(self.counts), _stream(stream)),
                  "fst_plan_backward")

    def forward_backward(self, weights: torch.Tensor | None = None, counts: bool = True, stream=None,
                         states: bool = False):
        if weights is not None:
            _require_cuda(weights, torch.float32, "weights")
        if states:
            check(self._lib.fst_plan_forward_backward_ex(
                self._h, _dptr(weights), _dptr(self.logz), _dptr(self.counts) if counts else None,
                _dptr(self.start_counts), _dptr(self.final_counts), _dptr(self.status), _stream(stream)),
                "fst_plan_forward_backward_ex")
        else:
            check(self._lib.fst_plan_forward_backward(self._h, _dptr(weights), _dptr(self.logz),
                                                      _dptr(self.counts) if counts else None, _dptr(self.status),
                                                      _stream(stream)), "fst_plan_forward_backward")


def debug_checks() -> dict:
    """The bounds-checked build's violation record (fst_debug_checks), read
    and cleared: {"violations", "code", "index", "bound"}.  Raises FstError
    (UNSUPPORTED) on a normal build."""
    lib = _lib.load()
    v, c, i, b = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()
    check(lib.fst_debug_checks(C.byref(v), C.byref(c), C.byref(i), C.byref(b)), "fst_debug_checks")
    return {"violations": v.value, "code": c.value, "index": i.value, "bound": b.value}
