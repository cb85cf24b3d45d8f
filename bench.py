#!/usr/bin/env python
"""Benchmark: batched Viterbi + forward-backward on the 20M-arc workload.

One step = one pass of the whole hot path over one batch: Viterbi (relax,
final reduction, backtrace) and forward-backward (forward relax, log Z,
backward relax fused with arc posteriors, counts back to arc order) for all
4,096 strings of the 200,000-state, 20,000-symbol, 20,000,000-arc synthetic
FST (lengths U[5, 200], random-walk strings, seeded).  Inputs are resident
in HBM when the timed region starts and are larger than the L2 cache.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
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
    "c3": "batched: 200,000 states, 20,000 input symbols, 20,000,000 arcs (Zipf arcs per symbol, lognormal "
          "out-degree mean 100, Dirichlet(0.5) weights), 4,096 random-walk strings of length U[5,200]; "
          "Viterbi + forward-backward with arc posteriors per step",
    "c2": "plain-shaped: 50,000 states, 10,000 symbols, 5,000,000 arcs, 1,000 strings of length U[10,60]",
    "c4": "100,000 states, 5,000 symbols, 2,000,000 arcs, 1,024 strings of length U[10,100]",
    "c5": "1,000,000 states, 5,000 symbols, 100,000,000 arcs, 64 strings of length 1,000",
    "c1": "1,000 states, 50 symbols, 20,000 arcs, one string of length 50",
}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "traffic.json")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--budget-gb", type=float, default=48.0, help="plan storage budget (waves)")
    ap.add_argument("--plain-sample", type=int, default=48, help="strings timed on the plain path")
    ap.add_argument("--cpu-sample", type=int, default=16, help="strings timed on the CPU oracle")
    ap.add_argument("--slice-sample", type=int, default=16,
                    help="strings decoded with the paper's slice-wide relaxation for comparison")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--strings", type=int, default=0, help="use only the first N strings (profiling captures)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps from the host, not a CUDA graph")
    return ap.parse_args()


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


# ---------------------------------------------------------------- models
PASS_KERNELS = {"vit": ("vit_first", "vit_step"), "fwd": ("fwd_first", "fwd_sum", "fwd_step"),
                "bwd": ("bwd_step",)}
KERNEL_NAMES = {"vit_first": "k_vit_first", "vit_step": "k_vit_step", "fwd_first": "k_fwd_first",
                "fwd_sum": "k_fwd_sum", "fwd_step": "k_fwd_step", "bwd_step": "k_bwd_step"}


def bytes_model(stats, ids):
    """Algorithmic bytes per pass (sum over tokens of the per-step figures):
    Viterbi 12|A|+4U+8D, forward 12|A|+4U+4D, backward+posterior 20|A|+8U+4D."""
    A, D, U = (s.astype(np.float64)[ids] for s in stats)
    return {
        "vit": float((12 * A + 4 * U + 8 * D).sum()),
        "fwd": float((12 * A + 4 * U + 4 * D).sum()),
        "bwd": float((20 * A + 8 * U + 4 * D).sum()),
    }


# Dependent random 8-byte loads over buffers larger than L2 saturate near
# this rate on a GB300 (measured with a pointer-chasing probe, 131,072
# chains: 33-39 G/s for buffers of 1-32 GB).
RANDOM_ACCESS_PEAK = 35.0


def load_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def load_traffic(pass_name: str, workload: str):
    """ncu DRAM bytes (read + write) of one whole pass, the same unit as the
    model bytes behind `achieved`; None once the kernel sources changed."""
    try:
        with open(PROFILE_SUMMARY) as fh:
            d = json.load(fh)
        e = d.get(workload, {}).get(pass_name)
        if e and e.get("source_hash") == source_hash():
            return e.get("dram_bytes_per_pass")
    except (OSError, ValueError):
        pass
    return None


# the files that decide what the step kernels read and write
KERNEL_SOURCES = ("kernels.cu", "kernels.cuh", "store.cu")


def source_hash():
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1701_03038_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    from paper_1701_03038_gb300 import synth
    fa, strs = synth.make_config(args.workload)
    o = oracle.Fst(fa)
    cores = os.cpu_count() or 1
    sample = max(1, min(args.cpu_sample, strs.count))
    A = np.bincount(fa.ilabel, minlength=fa.num_isyms)
    times = []
    relax = 0
    for k in range(args.warmup + args.steps):
        b0 = (k * sample) % strs.count
        sel = [(b0 + i) % strs.count for i in range(sample)]
        ids = np.concatenate([strs.get(b) for b in sel]).astype(np.int32)
        off = np.zeros(sample + 1, np.int64)
        off[1:] = np.cumsum([len(strs.get(b)) for b in sel])
        t0 = time.perf_counter()
        o.viterbi_batch(ids, off, nthreads=cores)
        o.fb_batch(ids, off, nthreads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            relax += 3 * int(A[ids].sum())
    tot = sum(times)
    value = relax / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload + ": " + WORKLOADS[args.workload],
                   "reference": "CPU oracle (plain C; Viterbi float32, forward-backward float64)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} strings per step of the {args.workload} batch, "
                                   f"Viterbi + forward-backward with counts, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_1701_03038_gb300 import build as gbuild
    from paper_1701_03038_gb300 import synth
    from paper_1701_03038_gb300.fst import Fst
    from paper_1701_03038_gb300._lib import PLAN_NO_FB, PLAN_NO_VITERBI

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
    dev = torch.device("cuda", local)

    fa, strs = synth.make_config(args.workload)
    if args.strings and args.strings < strs.count:
        strs = synth.Strings(strs.ids[:strs.offsets[args.strings]].copy(), strs.offsets[:args.strings + 1].copy())
    f = Fst.from_arrays(fa, device=dev)
    stats = f.symbol_stats()
    ids = torch.from_numpy(strs.ids).to(dev)
    off = torch.from_numpy(strs.offsets).to(dev)
    # the Viterbi pass and forward-backward are independent: one plan each,
    # run on two streams so that their latency-bound launches overlap
    budget = int(args.budget_gb * (1 << 30))
    plan_v = f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_FB)
    plan_f = f.plan(ids, off, mem_budget=budget, flags=PLAN_NO_VITERBI)
    info_v, info_f = plan_v.info(), plan_f.info()
    info = {"waves": max(info_v["waves"], info_f["waves"]), "device_bytes": info_v["device_bytes"] + info_f["device_bytes"],
            "viterbi_launches": info_v["viterbi_launches"], "fb_launches": info_f["fb_launches"]}
    relax_pass = info_v["relaxations"]
    relax_step = 3 * relax_pass  # Viterbi, forward and backward each relax every slice
    s_v, s_f = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def step():
        main = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(main)
        s_v.wait_event(fork)
        s_f.wait_event(fork)
        plan_v.viterbi(stream=s_v)
        plan_f.forward_backward(stream=s_f)
        for st in (s_v, s_f):
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)

    def step_serial():
        plan_v.viterbi()
        plan_f.forward_backward()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # the step's ~800 launches replay as one CUDA graph (both streams)
    graph = None
    if not args.no_graph:
        s_c = torch.cuda.Stream(device=dev)
        s_c.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s_c):
            step()
        torch.cuda.synchronize()
        for _ in range(max(3, args.warmup)):
            graph.replay()
        torch.cuda.synchronize()
    run_step = graph.replay if graph is not None else step

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        run_step()
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    value = job_throughput(relax_step, world, ms / 1000.0)
    sent_s = job_throughput(strs.count, world, ms / 1000.0)

    # per-kernel device time of one more step, with events around every
    # launch; the passes run one after the other here so that each kernel's
    # time is its own
    plan_v.profile(True)
    plan_f.profile(True)
    step_serial()
    torch.cuda.synchronize()
    pv, pf = plan_v.profile_read(), plan_f.profile_read()
    prof = {k: (pv[k][0] + pf[k][0], pv[k][1] + pf[k][1]) for k in pv}
    plan_v.profile(False)
    plan_f.profile(False)
    live = plan_f.live_work()
    model = bytes_model(stats, strs.ids)
    # a pass is its first-position push plus its kernels per position (Viterbi
    # one, forward two, backward one); the byte model is per pass, so the
    # roofline is taken over the pass's kernels
    pass_ms = {k: sum(prof[x][0] for x in ks) for k, ks in PASS_KERNELS.items()}
    dom = max(pass_ms, key=pass_ms.get)
    peak, peak_src = load_peak()
    achieved = model[dom] / (pass_ms[dom] / 1000.0) / 1e9
    kernels = {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items()}
    passes = {k: {"ms": round(v, 3), "model_gbs": round(model[k] / (v / 1000.0) / 1e9, 1) if v > 0 else None}
              for k, v in pass_ms.items()}
    traffic = load_traffic(dom, args.workload)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "per": f"{dom} pass",
                "kernel": " + ".join(KERNEL_NAMES[x] for x in PASS_KERNELS[dom]),
                "launches": sum(prof[x][1] for x in PASS_KERNELS[dom]),
                "bytes_model": "per token: Viterbi 12|A|+4U+8D, forward 12|A|+4U+4D, "
                "backward+posterior 20|A|+8U+4D (every arc of the slice, as the paper relaxes it)",
                "peak_source": peak_src}

    # the work the frontier-driven kernels actually do, against the bound
    # that applies to it: random accesses (a pool entry or an arc each costs
    # a few loads or atomics at unrelated addresses)
    acc_model = {  # random accesses per live entry and per pushed arc
        "vit": (5, 2),  # accumulator, hash probe, arc source, state map read and write; arc, atomicMax
        "fwd": (2, 4),  # accumulator line, hash probe; arc and atomicMax, then arc and fixed-point add
        "bwd": (1, 3),  # backward value; arc, backward value of the destination, count atomic
    }
    live_passes = {}
    for k, (pe, pa) in acc_model.items():
        acc = pe * live["entries"] + pa * max(live["arcs"], 0)
        gps = acc / (pass_ms[k] / 1000.0) / 1e9 if pass_ms[k] > 0 else None
        tr = load_traffic(k, args.workload)
        live_passes[k] = {"accesses": acc, "g_accesses_per_s": round(gps, 2) if gps else None,
                          "frac": round(gps / RANDOM_ACCESS_PEAK, 4) if gps else None,
                          "dram_gbs": round(tr / (pass_ms[k] / 1000.0) / 1e9, 1) if tr and pass_ms[k] > 0 else None}
    roofline_live = {"bound": "random DRAM accesses", "unit": "G accesses/s", "peak": RANDOM_ACCESS_PEAK,
                     "peak_source": "pointer-chasing probe on a GB300 (profiles/launches_c3.md)",
                     "live_entries_per_pass": live["entries"], "live_arcs_per_pass": live["arcs"],
                     "model": "random accesses per live entry / per pushed arc: Viterbi 5/2, forward 2/4, "
                              "backward 1/3", "passes": live_passes}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload + ": " + WORKLOADS[args.workload], "strings": strs.count,
                      "tokens": int(len(strs.ids)), "relaxations_per_pass": relax_pass, "waves": info["waves"],
                      "plan_gb": round(info["device_bytes"] / 2**30, 2), "parallelism": "replicas" if world > 1 else "1 GPU",
                      "streams": "a Viterbi plan and a forward-backward plan on two CUDA streams; per-kernel "
                                 "times from one more step run serially",
                      "launch": "CUDA graph replay" if graph is not None else "host launches",
                      "l2": "no flush: inputs larger than L2 (arc store "
                            f"{(fa.num_arcs * 24) / 2**30:.2f} GiB, frontiers and per-step storage "
                            f"{info['device_bytes'] / 2**30:.1f} GiB)"},
           "sentences_per_s": sent_s, "roofline": roofline, "roofline_live": roofline_live, "passes": passes, "kernels": kernels, "clocks": clk,
           "gpu_launches": args.steps * (info["viterbi_launches"] + info["fb_launches"])}

    # plain method (one string at a time, one launch per position) on a sample
    if not args.no_plain and rank == 0:
        n = min(args.plain_sample, strs.count)
        for b in range(2):
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
        out["batched_over_plain_sentences"] = sent_s / world / (n / dt)
        # the paper's own relaxation (every arc of every slice, one thread
        # per arc, packed atomicMax) against the frontier-driven plain path,
        # Viterbi only, on the first strings
        k = min(args.slice_sample, strs.count)
        f.viterbi_slice(strs.get(0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in range(k):
            f.viterbi_slice(strs.get(b))
        dt_slice = time.perf_counter() - t0
        t0 = time.perf_counter()
        for b in range(k):
            f.viterbi(strs.get(b))
        dt_ours = time.perf_counter() - t0
        out["paper_design"] = {"sample": f"first {k} strings, Viterbi, one string at a time",
                               "slice_relaxation_sentences_per_s": k / dt_slice,
                               "frontier_plain_sentences_per_s": k / dt_ours,
                               "speedup": dt_slice / dt_ours}

    # end to end through the public batch API with host buffers
    if not args.no_e2e:
        h_ids = torch.from_numpy(strs.ids).pin_memory()
        h_off = torch.from_numpy(strs.offsets).pin_memory()
        h_scores = torch.empty(strs.count, dtype=torch.float32).pin_memory()
        h_paths = torch.empty(len(strs.ids), dtype=torch.int32).pin_memory()
        h_logz = torch.empty(strs.count, dtype=torch.float64).pin_memory()
        h_counts = torch.empty(fa.num_arcs, dtype=torch.float32).pin_memory()

        import threading

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
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dev)
        barrier()
        h2d = strs.ids.nbytes + strs.offsets.nbytes
        d2h = 4 * strs.count + 4 * len(strs.ids) + 8 * strs.count + 4 * fa.num_arcs
        out["e2e"] = {"value": job_throughput(relax_step, world, dt), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * dt,
                      "api": "Fst.viterbi_batch and Fst.forward_backward_batch from two host threads on two "
                             "streams (plans built per call; device storage kept from the previous call of the same kind)"}

    # CPU oracle on the host cores, bounded sample (rank 0, N = 1 only)
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        o = oracle.Fst(fa)
        cores = os.cpu_count() or 1
        n = min(args.cpu_sample, strs.count)
        sel_ids = np.concatenate([strs.get(b) for b in range(n)]).astype(np.int32)
        sel_off = strs.offsets[:n + 1].copy()
        t0 = time.perf_counter()
        o.viterbi_batch(sel_ids, sel_off, nthreads=cores)
        o.fb_batch(sel_ids, sel_off, nthreads=cores)
        dt = time.perf_counter() - t0
        rx = 3 * int(stats[0][sel_ids].sum())
        out["cpu_baseline"] = {"value": rx / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {n} strings of the batch, Viterbi + forward-backward with "
                                         f"counts, {cores} threads, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
