"""FSTs in the OpenFst / AT&T text format.

The paper's implementations read this format for compatibility with the
toolkits they are compared with (Sec. 6).  A file lists one item per line:

* an arc: ``src dst ilabel olabel [weight]`` (``src dst label [weight]`` for
  an acceptor, whose output labels equal its input labels);
* a final state: ``state [weight]``.

The source state of the first line is the start state.  Weights are costs,
``w = -log p`` (the tropical and log semirings), ``0`` when omitted.  Labels
are integers, or names resolved through symbol tables (OpenFst's text form:
one ``symbol id`` per line).  The method needs epsilon-free FSTs (Sec. 3):
an arc labelled epsilon (the name ``<eps>`` in a symbol table, or the
integer given as ``epsilon``) is rejected.  Arc ids are the arcs' line order.
This module is host-side input and output; it does no decoding.
"""
from __future__ import annotations

import io
import math
import os

import numpy as np

from .synth import FstArrays

__all__ = ["read_symbols", "read_att", "write_att", "encode"]

EPSILON_NAMES = ("<eps>", "<epsilon>")


def _lines(source):
    if hasattr(source, "read"):
        return source.read().splitlines()
    if isinstance(source, (list, tuple)):
        return list(source)
    if isinstance(source, str) and ("\n" in source or not os.path.exists(source)):
        return source.splitlines()
    with open(source) as fh:
        return fh.read().splitlines()


def read_symbols(source) -> dict:
    """A symbol table: ``{name: id}`` from lines ``name id``."""
    table = {}
    for n, line in enumerate(_lines(source), 1):
        f = line.split()
        if not f:
            continue
        if len(f) != 2:
            raise ValueError(f"symbol table line {n}: expected 'symbol id', got {line!r}")
        name, sid = f[0], int(f[1])
        if sid < 0:
            raise ValueError(f"symbol table line {n}: negative id {sid}")
        table[name] = sid
    return table


def _cost(tok: str, n: int) -> float:
    try:
        w = float(tok)
    except ValueError:
        raise ValueError(f"line {n}: bad weight {tok!r}") from None
    if math.isnan(w) or w == -math.inf:
        raise ValueError(f"line {n}: weight {tok!r} is not a cost (NaN or -inf)")
    return w


def read_att(source, isyms: dict | None = None, osyms: dict | None = None, acceptor: bool = False,
             epsilon: int | None = None, num_isyms: int | None = None, num_states: int | None = None) -> FstArrays:
    """Parse an FST (path, text or file object) into caller-order arc arrays.

    ``isyms`` / ``osyms``: symbol tables for named labels (else integers).
    ``epsilon``: the integer label that means epsilon when there is no input
    table (OpenFst files use 0); ``None`` treats every integer as a symbol.
    ``num_isyms`` / ``num_states``: sizes of the input alphabet and of the
    state set (default: the largest id met + 1)."""
    eps_in = {isyms[e] for e in EPSILON_NAMES if isyms and e in isyms}
    eps_out = {osyms[e] for e in EPSILON_NAMES if osyms and e in osyms}
    if isyms is None and epsilon is not None:
        eps_in.add(int(epsilon))
    if osyms is None and epsilon is not None:
        eps_out.add(int(epsilon))

    def label(tok, table, n, what):
        if table is not None:
            if tok not in table:
                raise ValueError(f"line {n}: {what} label {tok!r} is not in the symbol table")
            return table[tok]
        try:
            v = int(tok)
        except ValueError:
            raise ValueError(f"line {n}: {what} label {tok!r} is not an integer (no symbol table given)") from None
        if v < 0:
            raise ValueError(f"line {n}: negative {what} label {v}")
        return v

    src, dst, il, ol, w = [], [], [], [], []
    finals = {}
    start = None
    arc_fields = (3, 4) if acceptor else (4, 5)
    for n, line in enumerate(_lines(source), 1):
        f = line.split()
        if not f:
            continue
        try:
            s0 = int(f[0])
        except ValueError:
            raise ValueError(f"line {n}: state {f[0]!r} is not an integer") from None
        if s0 < 0:
            raise ValueError(f"line {n}: negative state {s0}")
        if start is None:
            start = s0
        if len(f) in (1, 2):
            finals[s0] = _cost(f[1], n) if len(f) == 2 else 0.0
            continue
        if len(f) not in arc_fields:
            raise ValueError(f"line {n}: expected {'src dst label' if acceptor else 'src dst ilabel olabel'}"
                             f" [weight], got {line!r}")
        d = int(f[1])
        if d < 0:
            raise ValueError(f"line {n}: negative state {d}")
        a = label(f[2], isyms, n, "input")
        b = a if acceptor else label(f[3], osyms if osyms is not None else None, n, "output")
        if a in eps_in or (not acceptor and b in eps_out):
            raise ValueError(f"line {n}: epsilon arc (the method handles epsilon-free FSTs only)")
        src.append(s0)
        dst.append(d)
        il.append(a)
        ol.append(b)
        k = 4 if not acceptor else 3
        w.append(_cost(f[k], n) if len(f) > k else 0.0)
    if start is None:
        raise ValueError("empty FST: no arcs and no final states")
    q = max([start] + src + dst + list(finals)) + 1
    if num_states is not None:
        if num_states < q:
            raise ValueError(f"num_states={num_states} is below the largest state + 1 = {q}")
        q = num_states
    m = max(il, default=-1) + 1
    if isyms:
        m = max(m, max(isyms.values()) + 1)
    if num_isyms is not None:
        if num_isyms < m:
            raise ValueError(f"num_isyms={num_isyms} is below the largest input label + 1 = {m}")
        m = num_isyms
    n_out = max(ol, default=-1) + 1
    if osyms:
        n_out = max(n_out, max(osyms.values()) + 1)
    start_w = np.full(q, np.inf, np.float32)
    start_w[start] = 0.0
    final_w = np.full(q, np.inf, np.float32)
    for s, c in finals.items():
        final_w[s] = c
    return FstArrays(q, max(m, 1), max(n_out, 1), np.array(src, np.int32), np.array(dst, np.int32),
                     np.array(il, np.int32), np.array(ol, np.int32), np.array(w, np.float32), start_w, final_w)


def write_att(fst: FstArrays, dest=None, isyms: dict | None = None, osyms: dict | None = None) -> str:
    """The FST as AT&T text (returned, and written to ``dest`` if given).

    The format has one start state of weight 0: an FST with several start
    states, or a start weight other than 0, cannot be written.  Arcs out of
    the start state come first (the first line names the start state), the
    others follow in caller order; weights are written with 9 significant
    digits, enough to read float32 back exactly."""
    starts = np.flatnonzero(np.isfinite(fst.start_weight))
    if len(starts) != 1 or fst.start_weight[starts[0]] != 0:
        raise ValueError("AT&T text needs exactly one start state with weight 0")
    q0 = int(starts[0])
    inv_i = {v: k for k, v in isyms.items()} if isyms else None
    inv_o = {v: k for k, v in osyms.items()} if osyms else None
    from_start = list(np.flatnonzero(fst.src == q0))
    order = from_start + list(np.flatnonzero(fst.src != q0))
    out = io.StringIO()
    finals = np.flatnonzero(np.isfinite(fst.final_weight))
    fin = sorted(int(s) for s in finals)
    if not from_start:
        if q0 not in fin:
            raise ValueError("the start state has no arcs and is not final: no line can name it")
        fin.remove(q0)
        out.write(f"{q0}\t{float(fst.final_weight[q0]) + 0.0:.9g}\n")
    for k in order:
        a = inv_i[int(fst.ilabel[k])] if inv_i else int(fst.ilabel[k])
        b = inv_o[int(fst.olabel[k])] if inv_o else int(fst.olabel[k])
        out.write(f"{int(fst.src[k])}\t{int(fst.dst[k])}\t{a}\t{b}\t{float(fst.weight[k]) + 0.0:.9g}\n")
    for s in fin:
        out.write(f"{s}\t{float(fst.final_weight[s]) + 0.0:.9g}\n")
    text = out.getvalue()
    if dest is not None:
        with open(dest, "w") as fh:
            fh.write(text)
    return text


def encode(tokens, isyms: dict) -> np.ndarray:
    """Input symbol ids of a sequence of names."""
    try:
        return np.array([isyms[t] for t in tokens], np.int32)
    except KeyError as e:
        raise ValueError(f"symbol {e.args[0]!r} is not in the input table") from None
