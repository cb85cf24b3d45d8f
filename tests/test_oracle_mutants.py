"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins catch every one of them."""
import os
import shutil
import subprocess

import pytest

import oracle

import pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = {
    "viterbi_gathers_dst": ("prev[f->src[k]] + f->theta[k]", "prev[f->dst[k]] + f->theta[k]"),
    "viterbi_highest_id_on_ties": ("if (c > cur[q2])", "if (c >= cur[q2])"),
    "viterbi_drops_final_weight": ("const float c = prev[q] + f->theta_f[q];", "const float c = prev[q];"),
    "viterbi_highest_final_on_ties": ("if (c > best) { best = c; qb = q; }", "if (c >= best) { best = c; qb = q; }"),
    "viterbi_ignores_start_vector": ("prev[q] = f->theta_s[q];", "prev[q] = (q == 0) ? 0.0f : -INFINITY;"),
    "fb_drops_arc_weight": ("const double v = in[from[k]] + (double)f->theta[k];", "const double v = in[from[k]];"),
    "fb_max_instead_of_sum": ("out[to[k]] += exp(v - mx[to[k]]);", "out[to[k]] = 1.0;"),
    "fb_backward_not_reversed": ("const int32_t *from = reverse ? f->dst : f->src;", "const int32_t *from = f->src;"),
    "counts_drop_beta": ("+ be[(size_t)t * Q + f->dst[k]] - logz;", "- logz;"),
    "counts_alpha_off_by_one": ("const double e = al[(size_t)(t - 1) * Q + f->src[k]]", "const double e = al[(size_t)t * Q + f->src[k]]"),
    "em_reads_one_states_total": ("const double t = total[src[k]];", "const double t = total[0];"),
    "em_drops_pseudo_count_in_total": ("total[src[k]] += counts[k] + alpha;", "total[src[k]] += counts[k];"),
    "em_unused_states_get_minus_inf": (": (double)theta[k];", ": -INFINITY;"),
    "logz_drops_final_weight": ("s += exp(al[(size_t)n * Q + q] + (double)f->theta_f[q] - m);", "s += exp(al[(size_t)n * Q + q] - m);"),
}


def _run_pins(lib):
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(lib)
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            failed.append((pin.__name__, type(e).__name__))
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(text.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", *oracle.CFLAGS, str(mut), "-o", str(so), "-lm"], check=True)
    lib = oracle.load(str(so))
    failed = _run_pins(lib)
    assert failed, f"mutant {name} passed every pin"


def test_unmutated_passes_all(tmp_path):
    assert _run_pins(oracle.load()) == []
