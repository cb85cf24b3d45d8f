"""Host logic of the bench's launch accounting for the plain method: the
kernels one fst_viterbi + fst_forward_backward (with posteriors) call pair
launches, by the method and driver the handle reports.  The expected
sequences are written out launch by launch, in the order the single-string
entry points issue them."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1701_03038_gb300 import _lib, synth  # noqa: E402


class FakeFst:
    def __init__(self, method, driver, num_arcs=10):
        self.m = {"method": method, "driver": driver, "grid_blocks": 0}
        self.num_arcs = num_arcs

    def plain_method(self):
        return dict(self.m)


def frontier_viterbi(n, persistent):
    seq = []
    if persistent and n >= 1:
        seq.append("k_vit_persist")
    else:
        if n >= 1:
            seq.append("k_vit_first")
        seq += ["k_vit_step"] * n
    return seq + ["k_vit_final", "k_backtrace"]


def frontier_fb(n, persistent):
    seq = []
    if persistent and n >= 1:
        seq.append("k_fwd_persist")
    else:
        if n >= 1:
            seq.append("k_fwd_first")
        seq += ["k_fwd_sum", "k_fwd_step"] * n
    seq.append("k_fb_final")
    seq += ["k_bwd_persist"] if persistent and n >= 1 else ["k_bwd_step"] * n
    return seq + ["k_counts_out"]


def slice_viterbi(x, arcs_per_symbol):
    seq = ["k_slice_relax" for a in x if arcs_per_symbol[a] > 0]
    seq.append("k_slice_final")
    if len(x) > 0:
        seq.append("k_gather_olabels")
    return seq


def block_pair(n, num_arcs):
    seq = ["k_block_viterbi", "k_block_fb"]
    if n > 0:
        seq.append("k_block_post")
    if num_arcs > 0:
        seq.append("k_block_post_out")
    return seq


def _case():
    arcs_per_symbol = np.array([3, 0, 5, 1], np.int64)  # symbol 1 has no arcs
    xs = [np.zeros(0, np.int32), np.array([0, 1, 2], np.int32), np.array([1, 1], np.int32),
          np.array([2, 3, 0, 2, 1], np.int32)]
    off = np.zeros(len(xs) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in xs])
    strs = synth.Strings(np.concatenate(xs).astype(np.int32), off)
    return xs, strs, (arcs_per_symbol,)


def test_block_method_counts():
    xs, strs, stats = _case()
    for num_arcs in (10, 0):
        f = FakeFst(_lib.PLAIN_BLOCK, _lib.DRIVER_LAUNCH, num_arcs)
        want = sum(len(block_pair(len(x), num_arcs)) for x in xs)
        assert bench.plain_launches(f, strs, stats, np.zeros(5)) == want


def test_frontier_counts_both_drivers():
    xs, strs, stats = _case()
    for driver in (_lib.DRIVER_LAUNCH, _lib.DRIVER_PERSISTENT):
        p = driver == _lib.DRIVER_PERSISTENT
        f = FakeFst(_lib.PLAIN_FRONTIER, driver)
        want = sum(len(frontier_viterbi(len(x), p)) + len(frontier_fb(len(x), p)) for x in xs)
        assert bench.plain_launches(f, strs, stats, np.zeros(5)) == want


def test_slice_and_auto_counts():
    xs, strs, stats = _case()
    f = FakeFst(_lib.PLAIN_SLICE, _lib.DRIVER_LAUNCH)
    want = sum(len(slice_viterbi(x, stats[0])) + len(frontier_fb(len(x), False)) for x in xs)
    assert bench.plain_launches(f, strs, stats, np.zeros(5)) == want
    # the calibrated choice: slice when c0 + c1 n + c2 S < d0 + d1 n
    coef = np.array([0.0, 10.0, 5.0, 0.0, 1.0])  # frontier 10 n, slice 5 + S
    f = FakeFst(_lib.PLAIN_AUTO, _lib.DRIVER_LAUNCH)
    want = 0
    for x in xs:
        n, S = len(x), int(stats[0][x].sum())
        v = slice_viterbi(x, stats[0]) if 5.0 + S < 10.0 * n else frontier_viterbi(n, False)
        want += len(v) + len(frontier_fb(n, False))
    assert bench.plain_launches(f, strs, stats, coef) == want


def test_graph_step_parts_rule():
    # the graph-replayed batched step: one Viterbi part per 32 strings (at
    # most 2, at most 400 / tmax), one forward-backward part per 256 strings
    # (at most 16); explicit arguments win
    class A:
        parts_vit = 0
        parts_fb = 0
    assert bench.auto_parts(A, 4096, 200) == (2, 16)   # c3
    assert bench.auto_parts(A, 64, 1000) == (1, 1)     # c5
    assert bench.auto_parts(A, 1000, 60) == (2, 3)     # c2's strings batched
    assert bench.auto_parts(A, 1, 50) == (1, 1)        # c1
    A.parts_vit, A.parts_fb = 3, 5
    assert bench.auto_parts(A, 4096, 200) == (3, 5)


def _ncu_csv(path, rows):
    import csv
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for i, (k, m, u, v) in enumerate(rows):
            w.writerow([str(i), k, m, u, v])


def test_traffic_ingest_and_staleness(tmp_path, monkeypatch):
    # per-pass DRAM bytes from an ncu launch list (units scaled, write and
    # read summed over every launch of the pass's kernels, other kernels
    # ignored), divided by the live-work byte model of the run's bench line;
    # read back only for the layout measured and only while the device code
    # is the one it was measured on
    import json
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "traffic.json"))
    rows = [("fstgpu::(anonymous namespace)::k_vit_step(LayoutView)", "dram__bytes_read.sum", "Mbyte", "1.5"),
            ("fstgpu::(anonymous namespace)::k_vit_step(LayoutView)", "dram__bytes_write.sum", "Kbyte", "500"),
            ("k_vit_first", "dram__bytes_read.sum", "byte", "1,000"),
            ("k_fwd_sum", "dram__bytes_read.sum", "byte", "3000"),
            ("k_fwd_step", "dram__bytes_write.sum", "byte", "7000"),
            ("k_fwd_step", "gpu__time_duration.sum", "nsecond", "12345"),
            ("k_bwd_step", "dram__bytes_read.sum", "Gbyte", "0.000004"),
            ("k_counts_out", "dram__bytes_read.sum", "byte", "999999")]
    _ncu_csv(tmp_path / "l.csv", rows)
    E, P = 100, 250
    line = {"live_work": {"entries": E, "arcs": P},
            "config": {"workload": "tiny", "strings": 3, "accumulators": "dense per-string arrays"}}
    (tmp_path / "b.json").write_text("noise\n" + json.dumps(line) + "\n")
    bench.ingest_traffic(str(tmp_path / "l.csv"), str(tmp_path / "b.json"))
    d = json.load(open(tmp_path / "traffic.json"))
    assert d["source_hash"] == bench.source_hash()
    p = d["modes"]["dense"]["passes"]
    alg = {"vit": 12 * P + 12 * E, "fwd": 12 * P + 8 * E, "bwd": 20 * P + 12 * E}
    assert p["vit"]["dram_bytes"] == 1_500_000 + 500_000 + 1_000
    assert p["fwd"]["dram_bytes"] == 10_000 and p["bwd"]["dram_bytes"] == 4_000
    for k in alg:
        assert p[k]["algorithmic_bytes"] == alg[k]
        assert abs(p[k]["dram_per_algorithmic_byte"] - p[k]["dram_bytes"] / alg[k]) < 1e-12
    assert bench.load_traffic("dense")["passes"]["vit"]["dram_bytes"] == 2_001_000
    assert bench.load_traffic("compact") is None
    # a second layout joins the first while the hash holds
    line["config"]["accumulators"] = "hash tables"
    (tmp_path / "b.json").write_text(json.dumps(line) + "\n")
    bench.ingest_traffic(str(tmp_path / "l.csv"), str(tmp_path / "b.json"))
    assert bench.load_traffic("dense") is not None and bench.load_traffic("compact") is not None
    monkeypatch.setattr(bench, "source_hash", lambda: "another")
    assert bench.load_traffic("dense") is None


def test_roofline_of_the_dominant_pass():
    # the pass with the most summed kernel time; achieved = its live-work
    # algorithmic bytes over that time, frac against the peak, traffic the
    # measured DRAM-per-algorithmic-byte ratio times those bytes
    kinds = ["vit_first", "vit_step", "vit_final", "backtrace", "fwd_first", "fwd_sum", "fwd_step", "fb_final",
             "bwd_step", "counts"]
    prof = {k: (0.0, 0) for k in kinds}
    prof.update({"vit_step": (2.0, 10), "vit_first": (0.5, 1), "fwd_sum": (3.0, 10), "fwd_step": (4.0, 10),
                 "fwd_first": (0.25, 1), "bwd_step": (1.0, 10)})
    E, P = 1_000_000, 2_000_000
    traffic = {"passes": {"fwd": {"dram_per_algorithmic_byte": 10.0}}, "note": "n"}
    r, passes = bench.roofline(prof, {"entries": E, "arcs": P}, 1000.0, "src", traffic)
    fwd_bytes = 12 * P + 8 * E
    sec = (3.0 + 4.0 + 0.25) / 1000.0
    assert r["per"].startswith("fwd") and r["launches"] == 21 and r["pass_ms"] == 7.25
    assert r["kernel"] == "k_fwd_first + k_fwd_sum + k_fwd_step"
    assert r["algorithmic_bytes"] == fwd_bytes
    assert abs(r["achieved"] - round(fwd_bytes / sec / 1e9, 2)) < 1e-9
    assert abs(r["frac"] - round(fwd_bytes / sec / 1e9 / 1000.0, 5)) < 1e-12
    assert r["traffic"] == int(10.0 * fwd_bytes) and r["wasted_traffic_ratio"] == 10.0
    assert set(passes) == {"vit", "fwd", "bwd"} and passes["vit"]["ms"] == 2.5
    # without a capture for the pass there is no traffic figure
    r2, _ = bench.roofline(prof, {"entries": E, "arcs": P}, 1000.0, "src", None)
    assert r2["traffic"] is None and "wasted_traffic_ratio" not in r2
    # a persistent pass is named by its one kernel
    r3, _ = bench.roofline(prof, {"entries": E, "arcs": P}, 1000.0, "src", None, persistent=("fwd",))
    assert r3["kernel"] == "k_fwd_persist"


def test_cpu_baseline_sample_and_repeats():
    # the oracle leg: a bounded sample of the workload's first strings; a
    # whole workload shorter than the minimum is repeated until it has run
    # that long, and the rates count every pass
    rng = np.random.default_rng(5)
    fa = synth.tiny_fst(rng, max_states=5, max_syms=3)
    xs = [rng.integers(0, fa.num_isyms, size=4).astype(np.int32) for _ in range(3)]
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([4, 4, 4])
    strs = synth.Strings(np.concatenate(xs), off)
    r = bench.cpu_baseline(fa, strs, "batch", target_s=0.01, min_s=0.05)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
    assert "passes)" in r["sample"] and r["sentences_per_s"] > 0
    # relaxations of one pass: every arc of every slice, three passes
    per_pass = 3 * int(np.bincount(fa.ilabel, minlength=fa.num_isyms)[strs.ids].sum())
    dt, rx, _ = bench.cpu_oracle_run(fa, strs, list(range(strs.count)), "batch")
    assert rx == per_pass and dt > 0


def test_reference_arm_line(capsys):
    # bench.py --impl reference: the oracle on the host cores, one JSON line
    # with the contract's keys, its own cpu_baseline and an e2e that moves no
    # bytes; ranks other than 0 print nothing
    import json
    args = bench.parse_args(["--impl", "reference", "--workload", "c1", "--steps", "2", "--warmup", "3"])
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["config"]["workload"].startswith("c1")
