#!/usr/bin/env python
"""Benchmark of the FST decoding hot path on the synthetic workloads.

Default workload (the 20M-arc batching workload): one step is one pass of
the whole hot path over one batch -- Viterbi (relax, final reduction,
backtrace) and forward-backward (forward relax, log Z, backward relax fused
with arc posteriors, counts back to arc order) for all 4,096 strings of the
200,000-state, 20,000-symbol, 20,000,000-arc FST (lengths U[5, 200],
random-walk strings, seeded).  Inputs are resident in HBM when the timed
region starts and are larger than the L2 cache.

Other workloads (``--workload``):
  c1  one 50-symbol string on a 1,000-state FST, plain method (latency);
  c2  1,000 strings on a 5,000,000-arc FST, plain method, one string at a
      time (one launch per position), the batched method timed beside it;
  c4  a training step on a 2,000,000-arc FST: log Z of 1,024 strings
      through autograd, loss.backward() (the fused backward pass) and an
      SGD update of the arc weights;
  c5  64 strings of length 1,000 on a 100,000,000-arc FST, batched.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead, on a bounded sample of the same workload.
``--ingest-traffic CSV JSONLINE`` turns an ncu launch list (DRAM bytes per
launch) of a small run into the per-pass traffic figures of
profiles/traffic.json.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "arc-relaxations/s & sentences/s, batched vs plain, % of HBM roofline"
UNIT = "arc-relaxations/s"
WORKLOADS = {
    "c1": ("plain", "1,000 states, 50 input / 20 output symbols, 20,000 arcs (uniform laws, Dirichlet(1) "
                    "weights), one string of length 50; plain method, Viterbi + forward-backward with posteriors"),
    "c2": ("plain", "50,000 states, 10,000 symbols, 5,000,000 arcs (Zipf arcs per symbol, lognormal out-degree "
                    "mean 100, Dirichlet(0.5)), 1,000 strings of length U[10,60]; plain method, one string at a "
                    "time, Viterbi + forward-backward with posteriors"),
    "c3": ("batch", "batched: 200,000 states, 20,000 input symbols, 20,000,000 arcs (Zipf arcs per symbol, "
                    "lognormal out-degree mean 100, Dirichlet(0.5) weights), 4,096 random-walk strings of length "
                    "U[5,200]; Viterbi + forward-backward with arc posteriors per step"),
    "c4": ("train", "training: 100,000 states, 5,000 symbols, 2,000,000 arc weights with requires_grad, 1,024 "
                    "strings of length U[10,100]; loss = sum log Z, backward = expected counts, SGD update"),
    "c5": ("batch", "batched: 1,000,000 states, 5,000 symbols, 100,000,000 arcs (uniform laws, Dirichlet(1)), "
                    "64 strings of length 1,000; Viterbi + forward-backward with arc posteriors per step"),
}
PERSIST_NAMES = {"vit": "k_vit_persist", "fwd": "k_fwd_persist", "bwd": "k_bwd_persist"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
# the files that decide what the step kernels read and write
KERNEL_SOURCES = ("kernels.cu", "kernels.cuh", "store.cu", "fst_internal.cuh")  # the device code of the batched passes
PASS_KERNELS = {"vit": ("vit_first", "vit_step"), "fwd": ("fwd_first", "fwd_sum", "fwd_step"),
                "bwd": ("bwd_step",)}
KERNEL_NAMES = {"vit_first": "k_vit_first", "vit_step": "k_vit_step", "fwd_first": "k_fwd_first",
                "fwd_sum": "k_fwd_sum", "fwd_step": "k_fwd_step", "bwd_step": "k_bwd_step",
                "vit_final": "k_vit_final", "backtrace": "k_backtrace", "fb_final": "k_fb_final",
                "counts": "k_counts_out"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--budget-gb", type=float, default=48.0, help="plan storage budget (waves)")
    ap.add_argument("--plain-sample", type=int, default=48, help="strings timed on the plain path (batch workloads)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--slice-sample", type=int, default=16,
                    help="strings decoded with the paper's slice-wide relaxation for comparison")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--strings", type=int, default=0, help="use only the first N strings (profiling captures)")
    ap.add_argument("--parts-vit", type=int, default=0,
                    help="stream-parallel parts of the Viterbi plan (0 = the batch calls' rule: one per 32 "
                         "strings, at most 2 and 400 / the longest string)")
    ap.add_argument("--parts-fb", type=int, default=0,
                    help="stream-parallel parts of the forward-backward plan (0 = one per 8 strings, at most 8 "
                         "and 1,600 / the longest string)")
    ap.add_argument("--pull", type=int, default=0,
                    help="direction switch of the forward pass: live states from which a token pulls "
                         "(0 = off, the library default; -1 = half the states)")
    ap.add_argument("--acc", default="dense", choices=["dense", "compact"],
                    help="accumulators of the batched plans: dense per-string arrays (FST_PLAN_DENSE_ACC, the "
                         "faster) or the library's default hash tables (a third of the memory)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps from the host, not a CUDA graph")
    ap.add_argument("--driver", default="graph", choices=["graph", "persistent", "persistent-all", "autotune"],
                    help="graph: one launch per position, the step replayed as a CUDA graph; persistent: the "
                         "forward-backward plan as persistent passes (one cooperative launch each), the Viterbi "
                         "plan beside it on its own stream; persistent-all: both plans persistent, one after the "
                         "other; autotune: each plan's driver and grid chosen by fst_plan_autotune")
    ap.add_argument("--ingest-traffic", nargs=2, metavar=("NCU_CSV", "BENCH_JSON"),
                    help="write profiles/traffic.json from an ncu launch list of a small run and that run's line")
    args = ap.parse_args(argv)
    args.dense_acc = args.acc == "dense"
    return args


def auto_parts(args, B, tmax):
    """The plan parts of the graph-replayed device step: the arguments, or
    by batch size: one Viterbi part per 32 strings, at most 2 and at most
    400 / tmax position launches' worth (tmax the longest string), and one
    forward-backward part per 256 strings, at most 16.  A graph replays the
    parts' launches without host threads, so it takes more
    forward-backward parts than the batch calls, which issue them from
    host threads and stop at 4.  Measured on c3 (Viterbi / forward-backward
    parts, ms a step): 2 / 8 15.6, 4 / 12 15.1, 2 / 16 14.2, 4 / 16 14.2,
    2 / 24 14.1."""
    tmax = max(int(tmax), 1)
    pv = args.parts_vit if args.parts_vit > 0 else max(1, min(2, B // 32, 400 // tmax))
    pf = args.parts_fb if args.parts_fb > 0 else max(1, min(16, B // 256))
    return pv, pf


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- replicas
def max_over_ranks(x: float, device) -> float:
    """The job's time: the slowest rank's (every rank runs the same work on
    its own GPU, so the whole job ends when the slowest replica does)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: the units all ranks processed over the job's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------ byte models
def live_bytes(entries: int, arcs: int) -> dict:
    """Algorithmic bytes of the work the kernels do in one pass, with the
    per-step coefficients of the byte model (12 B per arc record, 4 B per
    source or destination value, 8 B per count read-modify-write) applied to
    the live work: each live state is a destination once and a source once,
    and every arc out of a live state is relaxed once per pass.
      Viterbi  12 P + 4 E (sources) + 8 E (value and backpointer)
      forward  12 P + 4 E + 4 E
      backward 20 P + 8 E + 4 E (arcs, counts, alpha and beta, beta out)"""
    e, p = float(entries), float(max(arcs, 0))
    return {"vit": 12 * p + 12 * e, "fwd": 12 * p + 8 * e, "bwd": 20 * p + 12 * e}


def slice_bytes(stats, ids) -> dict:
    """The same model over every arc of every slice (the paper's relaxation,
    which the frontier kernels do not perform): per token Viterbi
    12|A|+4U+8D, forward 12|A|+4U+4D, backward 20|A|+8U+4D."""
    A, D, U = (s.astype(np.float64)[ids] for s in stats)
    return {"vit": float((12 * A + 4 * U + 8 * D).sum()), "fwd": float((12 * A + 4 * U + 4 * D).sum()),
            "bwd": float((20 * A + 8 * U + 4 * D).sum())}


def load_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1701_03038_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def acc_mode(line_or_args):
    """'dense' or 'compact': the accumulator layout of a bench line or of the arguments."""
    if isinstance(line_or_args, dict):
        return "dense" if str(line_or_args.get("config", {}).get("accumulators", "")).startswith("dense") else "compact"
    return "dense" if line_or_args.dense_acc else "compact"


def load_traffic(mode):
    """Per-pass DRAM bytes per algorithmic byte for accumulator layout
    ``mode``, measured by ncu on a small run of the current kernels; None
    when the kernel sources changed since (or that layout was not measured)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d.get("modes", {}).get(mode)


def roofline(prof, live, peak, peak_src, traffic, stats=None, ids=None, persistent=()):
    """Roofline of the dominant pass (the pass with the most kernel time).
    ``persistent``: the passes that ran as one persistent kernel each."""
    pass_ms = {k: sum(prof[x][0] for x in ks) for k, ks in PASS_KERNELS.items()}
    pass_ms = {k: v for k, v in pass_ms.items() if v > 0}
    dom = max(pass_ms, key=pass_ms.get)
    alg = live_bytes(live["entries"], live["arcs"])
    sec = pass_ms[dom] / 1000.0
    achieved = alg[dom] / sec / 1e9
    tr = None
    if traffic is not None and dom in traffic.get("passes", {}):
        tr = traffic["passes"][dom]["dram_per_algorithmic_byte"] * alg[dom]
    r = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
         "frac": round(achieved / peak, 5), "traffic": None if tr is None else int(tr),
         "per": f"{dom} pass (all its launches)",
         "kernel": (PERSIST_NAMES[dom] if dom in persistent
                    else " + ".join(KERNEL_NAMES[x] for x in PASS_KERNELS[dom])),
         "launches": sum(prof[x][1] for x in PASS_KERNELS[dom]), "pass_ms": round(pass_ms[dom], 3),
         "algorithmic_bytes": int(alg[dom]),
         "bytes_model": "live work: Viterbi 12P+12E, forward 12P+8E, backward 20P+12E (P arcs out of live states, "
                        "E live states), the per-step coefficients of the byte model",
         "peak_source": peak_src}
    if tr is not None:
        r["dram_gbs"] = round(tr / sec / 1e9, 1)
        r["dram_frac"] = round(tr / sec / 1e9 / peak, 4)
        r["wasted_traffic_ratio"] = round(tr / alg[dom], 2)
        r["traffic_source"] = traffic.get("note", "")
    if stats is not None:
        sl = slice_bytes(stats, ids)
        r["slice_model_gbs"] = round(sl[dom] / sec / 1e9, 1)
    passes = {}
    for k, v in pass_ms.items():
        passes[k] = {"ms": round(v, 3), "algorithmic_gbs": round(alg[k] / (v / 1000.0) / 1e9, 2)}
        if traffic is not None and k in traffic.get("passes", {}):
            t = traffic["passes"][k]["dram_per_algorithmic_byte"] * alg[k]
            passes[k]["dram_gbs"] = round(t / (v / 1000.0) / 1e9, 1)
    return r, passes


# ---------------------------------------------------------- CPU oracle leg
def host_mem_bytes() -> int:
    try:
        return int(os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE"))
    except (ValueError, OSError, AttributeError):
        return 16 << 30


def oracle_threads(fa, strs, sel):
    """Threads for the oracle's batch calls: every string in flight keeps
    (n+1) x Q float64 forward and backward tables, and every thread a
    float64 count per arc; use at most a third of the free host memory."""
    cores = os.cpu_count() or 1
    nmax = max(len(strs.get(b)) for b in sel) if len(sel) else 1
    per = 16 * (nmax + 1) * fa.num_states + 8 * fa.num_arcs
    return max(1, min(cores, len(sel), host_mem_bytes() // 3 // max(per, 1)))


def cpu_oracle_run(fa, strs, sel, kind):
    """One oracle pass over strings ``sel``: Viterbi + forward-backward with
    counts (the step of the batch and plain workloads; the training step is
    forward-backward with counts).  Returns (seconds, relaxations, threads)."""
    import oracle
    o = oracle.Fst(fa)
    ids = np.concatenate([strs.get(b) for b in sel]).astype(np.int32)
    off = np.zeros(len(sel) + 1, np.int64)
    off[1:] = np.cumsum([len(strs.get(b)) for b in sel])
    th = oracle_threads(fa, strs, sel)
    A = np.bincount(fa.ilabel, minlength=fa.num_isyms)
    t0 = time.perf_counter()
    if kind != "train":
        o.viterbi_batch(ids, off, nthreads=th)
    o.fb_batch(ids, off, nthreads=th)
    dt = time.perf_counter() - t0
    passes = 2 if kind == "train" else 3
    return dt, passes * int(A[ids].sum()), th


def cpu_baseline(fa, strs, kind, target_s, min_s=2.0):
    """The oracle timed on a bounded sample of the workload (about target_s
    seconds of one pass); a whole workload that takes under min_s (c1: one
    string) is timed over repeated passes until min_s have gone by."""
    sel = cpu_sample(fa, strs, kind, target_s)
    dt, rx, th = cpu_oracle_run(fa, strs, sel, kind)
    reps = 1
    while len(sel) == strs.count and dt < min_s:
        d2, r2, _ = cpu_oracle_run(fa, strs, sel, kind)
        dt, rx, reps = dt + d2, rx + r2, reps + 1
    what = "forward-backward with counts" if kind == "train" else "Viterbi + forward-backward with counts"
    return {"value": rx / dt, "unit": UNIT, "cores": th, "kind": "oracle",
            "sentences_per_s": reps * len(sel) / dt,
            "sample": f"first {len(sel)} strings of the workload{f' ({reps} passes)' if reps > 1 else ''}, "
                      f"{what}, {th} threads, {dt:.1f} s"}


def cpu_sample(fa, strs, kind, target_s):
    """Strings of a bounded oracle sample: grow it until one pass takes about
    target_s seconds (at least one string)."""
    n = 1
    dt, _, _ = cpu_oracle_run(fa, strs, [0], kind)
    if dt > 0:
        n = int(max(1, min(strs.count, target_s / dt * min(os.cpu_count() or 1, 8))))
    return list(range(n))


# ------------------------------------------------------------- reference arm
def workload_config(name, fa, strs):
    return {"workload": name + ": " + WORKLOADS[name][1], "strings": strs.count, "tokens": int(len(strs.ids)),
            "states": int(fa.num_states), "arcs": int(fa.num_arcs)}


def make_workload(args):
    from paper_1701_03038_gb300 import synth
    fa, strs = synth.make_config(args.workload)
    if args.strings and args.strings < strs.count:
        strs = synth.Strings(strs.ids[:strs.offsets[args.strings]].copy(), strs.offsets[:args.strings + 1].copy())
    return fa, strs


def run_reference(args, rank):
    if rank != 0:
        return
    fa, strs = make_workload(args)
    kind = WORKLOADS[args.workload][0]
    sel = cpu_sample(fa, strs, kind, min(args.cpu_seconds, 3.0))
    times, relax, th = [], 0, 1
    for k in range(args.warmup + args.steps):
        dt, rx, th = cpu_oracle_run(fa, strs, sel, kind)
        if k >= args.warmup:
            times.append(dt)
            relax += rx
    tot = sum(times)
    value = relax / tot
    sample = (f"{len(sel)} of {strs.count} strings per step ({args.workload}), "
              f"{'forward-backward with counts' if kind == 'train' else 'Viterbi + forward-backward with counts'}, "
              f"{th} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": workload_config(args.workload, fa, strs),
        "sentences_per_s": len(sel) * len(times) / tot,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------- traffic ingest
def ingest_traffic(csv_path, line_path):
    """profiles/traffic.json from an ncu launch list (per launch
    dram__bytes_read.sum and dram__bytes_write.sum) of a small run, and that
    run's bench line (its live work): DRAM bytes per algorithmic byte per
    pass, which bench.py multiplies by the algorithmic bytes of the full
    run.  DRAM traffic is taken to grow in proportion to the live work."""
    by_kernel = {}
    with open(csv_path) as fh:
        rows = [r for r in csv.reader(fh) if r]
    head = None
    for r in rows:
        if "Kernel Name" in r and "Metric Name" in r:
            head = r
            continue
        if head is None or len(r) != len(head):
            continue
        d = dict(zip(head, r))
        m = re.search(r"\b(k_[A-Za-z0-9_]+)", d["Kernel Name"])
        if not m:
            continue
        name = m.group(1)
        if d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            v = float(d["Metric Value"].replace(",", ""))
            unit = d.get("Metric Unit", "byte").lower()
            v *= {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9}.get(unit, 1)
            by_kernel[name] = by_kernel.get(name, 0.0) + v
    with open(line_path) as fh:
        line = json.loads([x for x in fh.read().splitlines() if x.startswith("{")][-1])
    live = line["live_work"]
    alg = live_bytes(live["entries"], live["arcs"])
    passes = {}
    for p, ks in PASS_KERNELS.items():
        tot = sum(by_kernel.get(KERNEL_NAMES[k], 0.0) for k in ks) + by_kernel.get(PERSIST_NAMES[p], 0.0)
        if tot > 0:
            passes[p] = {"dram_bytes": int(tot), "algorithmic_bytes": int(alg[p]),
                         "dram_per_algorithmic_byte": tot / alg[p]}
    mode = acc_mode(line)
    out = {"source_hash": source_hash(), "modes": {},
           "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every launch of one step of a small run "
                   "(--cache-control none), per algorithmic byte of its live work, by accumulator layout; "
                   "scaled by the live work"}
    try:
        with open(TRAFFIC_FILE) as fh:
            old = json.load(fh)
        if old.get("source_hash") == out["source_hash"]:
            out["modes"].update(old.get("modes", {}))
    except (OSError, ValueError):
        pass
    out["modes"][mode] = {"workload": line["config"]["workload"][:60], "strings": line["config"]["strings"],
                          "live_work": live, "passes": passes}
    with open(TRAFFIC_FILE, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


# ------------------------------------------------------------------ our arm
def init(args):
    import torch
    import torch.distributed as dist
    from paper_1701_03038_gb300 import build as gbuild
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one rank builds (when the in-tree library is stale) while the others
    # wait, so that no two ranks write the same object files
    if rank == 0:
        gbuild.build()
    if world > 1:
        dist.barrier()
        gbuild.build()
    return rank, world, local, torch.device("cuda", local)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def timed(run_step, args, world, dev, clocks):
    """W untimed steps, then K steps timed by CUDA events on the current
    stream with a barrier and a synchronize on both sides; max over ranks."""
    import torch
    for _ in range(max(3, args.warmup)):
        run_step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # an NVTX range around the timed steps: an ncu launch list of exactly
    # them is `ncu --nvtx --nvtx-include "timed_steps/" ...`
    torch.cuda.nvtx.range_push("timed_steps")
    ev0.record()
    for _ in range(args.steps):
        run_step()
    ev1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    return max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev), clk


def base_line(args, world, fa, strs, ms, relax_step, clk, launches):
    return {"metric": METRIC, "value": job_throughput(relax_step, world, ms / 1000.0), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.workload, fa, strs),
            "sentences_per_s": job_throughput(strs.count, world, ms / 1000.0), "clocks": clk,
            "gpu_launches": launches}


def bench_batch(args, rank, world, dev, fa, strs, f, stats):
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
    # the Viterbi pass and forward-backward are independent: one plan each on
    # its own stream, each cut into stream-parallel parts (FST_PLAN_PARTS),
    # so that their latency-bound launches overlap
    budget = int(args.budget_gb * (1 << 30))
    ids = torch.from_numpy(strs.ids).to(dev)
    off = torch.from_numpy(strs.offsets).to(dev)
    acc = _lib.PLAN_DENSE_ACC if args.dense_acc else 0
    args.parts_vit, args.parts_fb = auto_parts(args, strs.count, int(np.diff(strs.offsets).max(initial=1)))
    plans_v = [f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_FB | acc, parts=args.parts_vit)]
    plans_f = [f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_VITERBI | acc, parts=args.parts_fb)]
    for p in plans_f:
        p.set_pull(args.pull)
    tuned = {}
    if args.driver in ("persistent", "persistent-all"):
        for p in plans_f:
            p.set_driver(_lib.DRIVER_PERSISTENT)
    if args.driver == "persistent-all":
        for p in plans_v:
            p.set_driver(_lib.DRIVER_PERSISTENT)
    if args.driver == "autotune":
        tuned = {"viterbi": [p.autotune() for p in plans_v], "forward_backward": [p.autotune() for p in plans_f]}
    infos_v, infos_f = [p.info() for p in plans_v], [p.info() for p in plans_f]
    relax_pass = sum(i["relaxations"] for i in infos_v)
    allp = plans_v + plans_f
    streams = [torch.cuda.Stream(device=dev) for _ in allp]
    # two persistent (cooperative) passes never run at the same time
    serial = sum(1 for p in allp if p.driver()[0] == _lib.DRIVER_PERSISTENT) > 1

    def run(p, st):
        if p in plans_v:
            p.viterbi(stream=st)
        else:
            p.forward_backward(stream=st)

    def step():
        main = torch.cuda.current_stream()
        if serial:
            for p in allp:
                run(p, main)
            return
        fork = torch.cuda.Event()
        fork.record(main)
        for st in streams:
            st.wait_event(fork)
        for p, st in zip(allp, streams):
            run(p, st)
        for st in streams:
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # the step's launches replay as one CUDA graph (every stream)
    graph = None
    if not args.no_graph:
        s_c = torch.cuda.Stream(device=dev)
        s_c.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=s_c):
                step()
            torch.cuda.synchronize()
        except RuntimeError as e:  # a launch kind that cannot be captured: host launches
            print(f"graph capture failed ({e}); timing host launches", file=sys.stderr)
            graph = None
            torch.cuda.synchronize()
    run_step = graph.replay if graph is not None else step
    ms, clk = timed(run_step, args, world, dev, ClockSampler(int(str(dev).split(":")[-1])))
    launches = sum(i["viterbi_launches"] for i in infos_v) + sum(i["fb_launches"] for i in infos_f)
    out = base_line(args, world, fa, strs, ms, 3 * relax_pass, clk, args.steps * launches)

    # per-kernel device time of one more step, with events around every
    # launch; the passes run one after the other here so that each kernel's
    # time is its own
    for p in allp:
        p.profile(True)
    for p in allp:
        run(p, torch.cuda.current_stream())
    torch.cuda.synchronize()
    prof = None
    for p in allp:
        r = p.profile_read()
        prof = r if prof is None else {k: (prof[k][0] + r[k][0], prof[k][1] + r[k][1]) for k in r}
        p.profile(False)
    lws = [p.live_work() for p in plans_f]
    live = {"entries": sum(x["entries"] for x in lws), "arcs": sum(x["arcs"] for x in lws)}
    peak, peak_src = load_peak()
    persistent = (("vit",) if plans_v[0].driver()[0] else ()) + (("fwd", "bwd") if plans_f[0].driver()[0] else ())
    rl, passes = roofline(prof, live, peak, peak_src, load_traffic(acc_mode(args)), stats, strs.ids, persistent)
    performed = 3 * max(live["arcs"], 0)
    plan_bytes = sum(i["device_bytes"] for i in infos_v + infos_f)
    out["config"].update({
        "relaxations_per_pass": relax_pass, "waves": max(i["waves"] for i in infos_v + infos_f),
        "plan_gb": round(plan_bytes / 2**30, 2),
        "accumulators": ("dense per-string arrays (FST_PLAN_DENSE_ACC)" if args.dense_acc else
                         "hash tables of %d slots per part (Viterbi) and %d (forward-backward)"
                         % (plans_v[0].table_slots(), plans_f[0].table_slots())),
        "parallelism": "replicas" if world > 1 else "1 GPU",
        "streams": f"a Viterbi plan of {args.parts_vit} and a forward-backward plan of {args.parts_fb} "
                   "stream-parallel parts; per-kernel times from one more step run serially",
        "launch": "CUDA graph replay" if graph is not None else "host launches",
        "driver": {"viterbi": "persistent" if plans_v[0].driver()[0] else "one launch per position",
                   "forward_backward": "persistent" if plans_f[0].driver()[0] else "one launch per position",
                   "grid": {"viterbi": plans_v[0].driver()[1], "forward_backward": plans_f[0].driver()[1]},
                   "concurrent": not serial, "autotune": tuned or None},
        "l2": "no flush: inputs larger than L2 (arc store and hash "
              f"{(fa.num_arcs * 24) / 2**30:.2f} GiB, plan storage {plan_bytes / 2**30:.1f} GiB)"})
    out.update({"relaxations_performed_per_s": job_throughput(performed, world, ms / 1000.0),
                "live_work": live, "roofline": rl, "passes": passes,
                "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]}})
    s_v, s_f = streams[0], streams[len(plans_v)]

    # plain method (one string at a time, one launch per position) on a sample
    if not args.no_plain and rank == 0:
        n = min(args.plain_sample, strs.count)
        for b in range(min(2, strs.count)):
            f.viterbi(strs.get(b))
            f.forward_backward(strs.get(b))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rx = 0
        for b in range(n):
            x = strs.get(b)
            f.viterbi(x)
            f.forward_backward(x)
            rx += 3 * int(stats[0][x].sum())
        dt = time.perf_counter() - t0
        out["plain"] = {"value": rx / dt, "unit": UNIT, "sentences_per_s": n / dt,
                        "sample": f"first {n} strings, host API (fst_viterbi + fst_forward_backward)"}
        out["batched_over_plain_sentences"] = out["sentences_per_s"] / world / (n / dt)
        out["paper_design"] = paper_design(f, strs, args.slice_sample)

    # end to end through the public batch API with host buffers (the batch
    # calls' plans get the same storage budget as the timed plans)
    if not args.no_e2e:
        f.set_batch_budget(budget)
        out["e2e"] = e2e_batch(args, world, dev, fa, strs, f, s_v, s_f, 3 * relax_pass)
    return out


def paper_design(f, strs, k):
    """The paper's slice-wide relaxation (every arc of every slice, one thread
    per arc; Viterbi by packed atomicMax, forward-backward by float32 atomic
    log-add-exp) in both arc orders within a slice, against the frontier
    plain path, one string at a time on the first k strings (sentences/s)."""
    import torch
    from paper_1701_03038_gb300 import _lib
    xs = [strs.get(b) for b in range(min(k, strs.count))]

    def rate(fn):
        fn(xs[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for x in xs:
            fn(x)
        return len(xs) / (time.perf_counter() - t0)

    out = {"sample": f"first {len(xs)} strings, one string at a time (host API)",
           "frontier": {"viterbi_sentences_per_s": rate(f.viterbi),
                        "fb_sentences_per_s": rate(f.forward_backward)}}
    for name, order in (("by_destination", _lib.SLICE_BY_DESTINATION), ("by_source", _lib.SLICE_BY_SOURCE)):
        f.set_slice_order(order)
        out["slice_" + name] = {"viterbi_sentences_per_s": rate(f.viterbi_slice),
                                "fb_sentences_per_s": rate(f.forward_backward_slice)}
    f.set_slice_order(_lib.SLICE_BY_DESTINATION)
    out["viterbi_frontier_over_slice"] = (out["frontier"]["viterbi_sentences_per_s"]
                                          / out["slice_by_destination"]["viterbi_sentences_per_s"])
    out["fb_frontier_over_slice"] = (out["frontier"]["fb_sentences_per_s"]
                                     / out["slice_by_destination"]["fb_sentences_per_s"])
    return out


def e2e_batch(args, world, dev, fa, strs, f, s_v, s_f, relax_step):
    import threading

    import torch
    h_ids = torch.from_numpy(strs.ids).pin_memory()
    h_off = torch.from_numpy(strs.offsets).pin_memory()
    h_scores = torch.empty(strs.count, dtype=torch.float32).pin_memory()
    h_paths = torch.empty(len(strs.ids), dtype=torch.int32).pin_memory()
    h_logz = torch.empty(strs.count, dtype=torch.float64).pin_memory()
    h_counts = torch.empty(fa.num_arcs, dtype=torch.float32).pin_memory()

    def e2e_vit(st):
        with torch.cuda.stream(st):
            d_ids = h_ids.to(dev, non_blocking=True)
            d_off = h_off.to(dev, non_blocking=True)
            v = f.viterbi_batch(d_ids, d_off, stream=st)
            h_scores.copy_(v["scores"], non_blocking=True)
            h_paths.copy_(v["paths"], non_blocking=True)
            st.synchronize()

    def e2e_fb(st):
        with torch.cuda.stream(st):
            d_ids = h_ids.to(dev, non_blocking=True)
            d_off = h_off.to(dev, non_blocking=True)
            r = f.forward_backward_batch(d_ids, d_off, stream=st)
            h_logz.copy_(r["logz"], non_blocking=True)
            h_counts.copy_(r["counts"], non_blocking=True)
            st.synchronize()

    def e2e_step():
        # the two batch calls from two host threads on two streams: their
        # plan builds overlap on the host and their kernels on the GPU
        th = threading.Thread(target=e2e_fb, args=(s_f,))
        th.start()
        e2e_vit(s_v)
        th.join()

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dev)
    barrier(world)
    h2d = strs.ids.nbytes + strs.offsets.nbytes
    d2h = 4 * strs.count + 4 * len(strs.ids) + 8 * strs.count + 4 * fa.num_arcs
    return {"value": job_throughput(relax_step, world, dt), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * dt,
            "api": "Fst.viterbi_batch and Fst.forward_backward_batch from two host threads on two streams (plans "
                   "built per call; device storage kept from the previous call of the same kind)"}


def plain_launches(f, strs, stats, coef) -> int:
    """Kernel launches of one plain step, from the method and driver the
    handle takes (fst_get_plain_method) and the launch sites of each: the
    one-block kernels one launch for Viterbi and, for forward-backward, the
    forward and backward blocks, the posteriors (non-empty strings) and
    their conversion (arcs > 0); the slice-wide Viterbi one per
    non-empty slice + final + output labels; the frontier Viterbi first +
    n steps + final + backtrace (one persistent pass + 2 with that
    driver); the frontier forward-backward first + n (sum + step) + final
    + n backward steps + counts (persistent: 2 passes + 2)."""
    from paper_1701_03038_gb300 import _lib
    pm = f.plain_method()
    if pm["method"] == _lib.PLAIN_BLOCK:
        lens = np.diff(strs.offsets)
        return int(strs.count * (3 if f.num_arcs > 0 else 2) + (lens > 0).sum())
    persist = pm["driver"] == _lib.DRIVER_PERSISTENT
    total = 0
    for b in range(strs.count):
        x = strs.get(b)
        n = len(x)
        arcs = int(stats[0][x].sum())
        slice_vit = pm["method"] == _lib.PLAIN_SLICE or (
            pm["method"] == _lib.PLAIN_AUTO and coef[2] + coef[3] * n + coef[4] * arcs < coef[0] + coef[1] * n)
        if slice_vit:
            total += int((stats[0][x] > 0).sum()) + 1 + (n > 0)
        else:
            total += (3 if n >= 1 else 2) if persist else n + 3 - (n == 0)
        total += (4 if n >= 1 else 2) if persist else 3 * n + 3 - (n == 0)
    return total


def bench_plain(args, rank, world, dev, fa, strs, f, stats):
    """The plain method: one string at a time through the host API
    (fst_viterbi + fst_forward_backward with posteriors), one launch per
    position; a step is every string of the workload.  The host API copies
    each string in and its results out, so the step is end to end; each
    string's posteriors go to one pinned host buffer reused by every call."""
    import torch
    from paper_1701_03038_gb300 import _lib
    relax_step = 3 * int(stats[0][strs.ids].sum())
    # the single-string Viterbi takes the cheaper of the frontier and the
    # slice-wide kernels, by a cost model calibrated on the first strings
    k = min(16, strs.count)
    coef = f.autotune_plain(strs.ids[:strs.offsets[k]], strs.offsets[:k + 1])
    # the posteriors of each string are read into one pinned host buffer
    # (the batched e2e leg reads its results into pinned buffers too)
    h_post = torch.empty(max(fa.num_arcs, 1), dtype=torch.float32).pin_memory().numpy()

    def step():
        for b in range(strs.count):
            x = strs.get(b)
            f.viterbi(x)
            f.forward_backward(x, out=h_post)

    ms, clk = timed(step, args, world, dev, ClockSampler(int(str(dev).split(":")[-1])))
    launches = plain_launches(f, strs, stats, coef)
    out = base_line(args, world, fa, strs, ms, relax_step, clk, args.steps * launches)
    out["config"].update({"parallelism": "replicas" if world > 1 else "1 GPU",
                          "launch": "host launches, one string at a time (fst_viterbi, fst_forward_backward; posteriors into a pinned host buffer)",
                          "l2": "no flush: the step streams every string's slices; consecutive strings share "
                                "L2-resident arcs, as a decoding loop would"})
    h2d = strs.ids.nbytes
    d2h = 4 * strs.count + 4 * len(strs.ids) * 2 + 8 * strs.count + 4 * fa.num_arcs * strs.count
    out["e2e"] = {"value": out["value"], "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                  "ms_per_step": ms, "api": "fst_viterbi + fst_forward_backward (host buffers, the posteriors pinned; copies inside)"}
    out["us_per_sentence"] = 1000.0 * ms / strs.count
    lens = np.diff(strs.offsets)
    sl = [bool(coef[2] + coef[3] * n + coef[4] * a < coef[0] + coef[1] * n)
          for n, a in zip(lens, [int(stats[0][strs.get(b)].sum()) for b in range(strs.count)])]
    out["plain_viterbi"] = {"method": "automatic (fst_autotune_plain on the first strings)",
                            "coef_us": [round(float(c), 4) for c in coef],
                            "strings_on_slice_kernel": int(sum(sl)), "strings": strs.count}
    # per-kernel times and live work of one more step, with events (frontier
    # kernels for both passes, so that every relaxation is profiled)
    f.set_plain_method(_lib.PLAIN_FRONTIER)
    f.profile(True)
    entries = arcs = 0
    for b in range(strs.count):
        x = strs.get(b)
        f.viterbi(x)
        f.forward_backward(x)
        lw = f.live_work()
        entries += lw["entries"]
        arcs += max(lw["arcs"], 0)
    prof = f.profile_read()
    f.profile(False)
    f.set_plain_method(_lib.PLAIN_AUTO)
    live = {"entries": entries, "arcs": arcs}
    peak, peak_src = load_peak()
    rl, passes = roofline(prof, live, peak, peak_src, None, stats, strs.ids)
    out.update({"relaxations_performed_per_s": job_throughput(3 * arcs, world, ms / 1000.0), "live_work": live,
                "roofline": rl, "passes": passes,
                "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]}})
    # the batched method on the same strings, for comparison
    if strs.count > 1 and rank == 0:
        import torch
        from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI
        ids = torch.from_numpy(strs.ids).to(dev)
        off = torch.from_numpy(strs.offsets).to(dev)
        pv = f.plan(ids, off, flags=PLAN_NO_FB)
        pf = f.plan(ids, off, flags=PLAN_NO_VITERBI)
        for _ in range(3):
            pv.viterbi()
            pf.forward_backward()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(5):
            pv.viterbi()
            pf.forward_backward()
        ev1.record()
        torch.cuda.synchronize()
        bms = ev0.elapsed_time(ev1) / 5
        out["batched"] = {"ms_per_step": bms, "sentences_per_s": strs.count / (bms / 1000.0),
                          "value": relax_step / (bms / 1000.0), "unit": UNIT,
                          "how": "the same strings as one plan each for Viterbi and forward-backward, host launches"}
        out["batched_over_plain_sentences"] = out["batched"]["sentences_per_s"] / (out["sentences_per_s"] / world)
    # the paper's slice-wide relaxation on the same strings
    if rank == 0:
        out["paper_design"] = paper_design(f, strs, args.slice_sample)
    return out


def bench_train(args, rank, world, dev, fa, strs, f, stats):
    """A training step: log Z of every string through autograd (forward
    pass), loss = -sum log Z / B, loss.backward() (the fused backward pass:
    the gradient is minus the expected counts), and an SGD update of the
    arc log-weights (written back to the FST by the next forward)."""
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300._lib import PLAN_SINGLE_WAVE
    from paper_1701_03038_gb300.autograd import LogZModule
    ids = torch.from_numpy(strs.ids).to(dev)
    off = torch.from_numpy(strs.offsets).to(dev)
    plan = f.plan(ids, off, mem_budget=int(args.budget_gb * (1 << 30)),
                  flags=PLAN_SINGLE_WAVE | (_lib.PLAN_DENSE_ACC if args.dense_acc else 0))
    from paper_1701_03038_gb300 import _lib
    tuned = None
    if args.driver in ("persistent", "persistent-all"):
        plan.set_driver(_lib.DRIVER_PERSISTENT)
    elif args.driver == "autotune":
        tuned = plan.autotune()
    info = plan.info()
    mod = LogZModule(f, -torch.from_numpy(fa.weight.astype(np.float32)))
    opt = torch.optim.SGD(mod.parameters(), lr=1e-3)
    B = strs.count

    def step():
        opt.zero_grad(set_to_none=False)
        loss = -mod(plan).sum() / B
        loss.backward()
        opt.step()

    ms, clk = timed(step, args, world, dev, ClockSampler(int(str(dev).split(":")[-1])))
    relax_pass = info["relaxations"]
    out = base_line(args, world, fa, strs, ms, 2 * relax_pass, clk, args.steps * info["fb_launches"])
    out["config"].update({"relaxations_per_pass": relax_pass, "plan_gb": round(info["device_bytes"] / 2**30, 2),
                          "parallelism": "replicas" if world > 1 else "1 GPU",
                          "launch": "host launches (fst_set_weights between steps is synchronous)",
                          "driver": {"forward_backward": "persistent" if plan.driver()[0] else "one launch per position",
                                     "grid": plan.driver()[1], "autotune": tuned},
                          "l2": "no flush: arc store, plan storage and the 2M-arc count vector exceed L2"})
    plan.profile(True)
    step()
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    live = plan.live_work()
    peak, peak_src = load_peak()
    rl, passes = roofline(prof, live, peak, peak_src, load_traffic(acc_mode(args)), stats, strs.ids,
                          ("fwd", "bwd") if plan.driver()[0] else ())
    out.update({"relaxations_performed_per_s": job_throughput(2 * max(live["arcs"], 0), world, ms / 1000.0),
                "live_work": live, "roofline": rl, "passes": passes,
                "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]}})
    if not args.no_e2e:
        out["e2e"] = e2e_train(args, world, dev, fa, strs, f, 2 * relax_pass)
    return out


def e2e_train(args, world, dev, fa, strs, f, relax_step):
    """The training step end to end through the public API, its batch
    copied in every step: ids and offsets from pinned host memory,
    fst_set_weights of the current log-weights, fst_forward_backward_batch
    with per-string weights 1/B (its counts are then minus the gradient of
    the mean -log Z, the loss), the SGD update of the log-weights on the
    device, and the loss read back into pinned memory.  The same step as the
    device-timed one, which keeps its batch in a plan."""
    import torch
    h_ids = torch.from_numpy(strs.ids).pin_memory()
    h_off = torch.from_numpy(strs.offsets).pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    B = strs.count
    theta = torch.from_numpy(-fa.weight.astype(np.float32)).to(dev)
    w = torch.full((B,), 1.0 / B, dtype=torch.float32, device=dev)
    st = torch.cuda.Stream(device=dev)

    def step():
        with torch.cuda.stream(st):
            d_ids = h_ids.to(dev, non_blocking=True)
            d_off = h_off.to(dev, non_blocking=True)
            f.set_weights(theta, "log")
            r = f.forward_backward_batch(d_ids, d_off, weights=w, stream=st)
            h_loss.copy_(-(r["logz"].sum() / B).reshape(1), non_blocking=True)
            theta.add_(r["counts"], alpha=1e-3)  # SGD, learning rate 1e-3: theta -= lr * (-counts)
            st.synchronize()

    step()  # the batch call's storage, kept for the next call
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step()
    dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dev)
    barrier(world)
    return {"value": job_throughput(relax_step, world, dt), "unit": UNIT,
            "h2d_bytes_per_step": int(strs.ids.nbytes + strs.offsets.nbytes), "d2h_bytes_per_step": 8,
            "ms_per_step": 1000 * dt,
            "api": "fst_set_weights, Fst.forward_backward_batch with per-string weights 1/B (counts = minus the "
                   "gradient of the mean -log Z), SGD on the device, the loss read back; ids and offsets from "
                   "pinned memory every step"}


def main():
    args = parse_args()
    if args.ingest_traffic:
        ingest_traffic(*args.ingest_traffic)
        return
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    rank, world, local, dev = init(args)
    from paper_1701_03038_gb300.fst import Fst
    fa, strs = make_workload(args)
    f = Fst.from_arrays(fa, device=dev)
    stats = f.symbol_stats()
    kind = WORKLOADS[args.workload][0]
    fn = {"batch": bench_batch, "plain": bench_plain, "train": bench_train}[kind]
    out = fn(args, rank, world, dev, fa, strs, f, stats)

    # CPU oracle on the host cores, bounded sample (rank 0, N = 1 only)
    if not args.no_cpu and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(fa, strs, kind, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
