"""The oracle's pins catch plausible mistakes in the oracle.

Each case below plants one mistake in a copy of ``oracle/lbg_oracle.c`` (a
dropped term, a wrong sign, a transposed index, another reading of a rule
the paper fixes), compiles the copy, and runs the pins of
``tests/test_oracle.py`` against it in a child process.  The mistake must make
at least one pin fail.  The unmodified source, compiled the same way, must
pass every pin, so a failure of a planted copy is the pins' doing and not the
harness's.  Every planted mistake keeps all memory accesses in bounds.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbg_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle.py")

# name -> [(text in lbg_oracle.c, text that replaces it), ...]; each text occurs once.
MUTANTS = {
    # Sec. 2.2 distance: squared Euclidean (reading R7)
    "distance_not_squared": [("    return s;\n}\n\n/* Initial codebook",
                              "    return sqrt(s);\n}\n\n/* Initial codebook")],
    "distance_abs_not_square": [("        s += d * d;", "        s += fabs(d);")],
    "distance_drops_last_dim": [("    for (int32_t l = 0; l < L; ++l) {\n        double d =",
                                 "    for (int32_t l = 0; l < L - 1; ++l) {\n        double d =")],
    # Alg. 1 centroid(input)
    "mean_divides_by_m_minus_1": [("c_out[l] /= (double)M;", "c_out[l] /= (double)(M - 1);")],
    "mean_transposed": [("c_out[l] += (double)X[m * L + l];",
                         "c_out[L - 1 - l] += (double)X[m * L + l];")],
    # Alg. 1 codebook splitting (readings R5, R6) and variant V1
    "split_children_swapped": [(": c + delta;", ": c - DELTA_TMP;"),
                               (": c - delta;", ": c + delta;"),
                               ("c - DELTA_TMP;", "c - delta;")],
    "split_plus_child_dropped": [(": c + delta;", ": c;")],
    "split_mult_minus_as_divide": [("c * (1.0 - delta)", "c / (1.0 + delta)")],
    # cell allocation: ties to the lowest index (R9) and the near-tie gap
    "tie_goes_to_highest_index": [("if (d < d1) {", "if (d <= d1) {")],
    "second_best_not_tracked": [("} else if (d < d2) {", "} else if (d < d1) {")],
    "gap_relative_to_second": [("gap[m] = (d2 - d1) / d1;", "gap[m] = (d2 - d1) / d2;")],
    "gap_zero_distance_rule": [("gap[m] = (d2 > 0.0) ? INFINITY : 0.0;",
                                "gap[m] = (d2 > 0.0) ? 0.0 : INFINITY;")],
    # integration of distortions
    "distortion_drops_first_term": [("for (int64_t m = 0; m < M; ++m) s += e[m];",
                                     "for (int64_t m = 1; m < M; ++m) s += e[m];")],
    # updation (R10)
    "update_divides_by_count_plus_1": [("sum[i] / (double)cnt[n]",
                                        "sum[i] / (double)(cnt[n] + 1)")],
    "update_empty_cell_zeroed": [(": C_in[i];", ": 0.0;")],
    "update_transposed": [("sum[(int64_t)n * L + l] += (double)X[m * L + l];",
                           "sum[(int64_t)n * L + l] += (double)X[m * L + (L - 1 - l)];")],
    # stop test (readings R1, R2) and the stage loop (R3, R4, R11)
    "stop_divides_by_previous": [("((D_prev - D) / D <= theta)",
                                  "((D_prev - D) / D_prev <= theta)")],
    "stop_strict_less": [("((D_prev - D) / D <= theta)", "((D_prev - D) / D < theta)")],
    "stop_no_zero_rule": [("int done = (D == 0.0) || ", "int done = ")],
    "d_prev_not_reset_per_stage": [("    for (;;) {\n        double D_prev = INFINITY;",
                                    "    double D_prev = INFINITY;\n    for (;;) {")],
    "halt_keeps_updated_codebook": [
        ("            if (done) break;",
         "            if (done) {\n"
         "                oracle_update(X, M, L, a_out, n, C, Cn, cnt);\n"
         "                memcpy(C, Cn, (size_t)n * L * sizeof(double));\n"
         "                break;\n"
         "            }")],
    "pass_cap_off_by_one": [("if (pass + 1 >= max_passes)", "if (pass >= max_passes)")],
    # variant V2 re-seeding
    "reseed_takes_smallest_cell": [("if (counts[n] > counts[b]) b = n;",
                                    "if (counts[n] < counts[b] && counts[n] > 1) b = n;")],
    "reseed_rounds_half_up": [("counts[e] = counts[b] / 2;", "counts[e] = (counts[b] + 1) / 2;")],
    "train_ignores_multiplicative": [("oracle_split_mode(C, n, L, delta, split_mult, Cn);",
                                      "oracle_split_mode(C, n, L, delta, 0, Cn);")],
    "train_ignores_reseed": [("if (reseed) oracle_reseed(Cn, cnt, n, L, delta);",
                              "(void)reseed;")],
    "near_tie_count_strict": [("near += gap[m] <= near_tol;", "near += gap[m] < near_tol;")],
    "assign_skips_first_row": [("for (int64_t m = 0; m < M; ++m) {\n        const float *x = X",
                                "for (int64_t m = 1; m < M; ++m) {\n        const float *x = X")],
    "update_counts_doubled": [("        cnt[n] += 1;\n        for (int32_t l = 0; l < L; ++l) sum[",
                               "        cnt[n] += 2;\n        for (int32_t l = 0; l < L; ++l) sum[")],
    "mean_not_zeroed": [("for (int32_t l = 0; l < L; ++l) c_out[l] = 0.0;",
                         "for (int32_t l = 0; l < L; ++l) c_out[l] += 0.0;")],
    "update_keeps_singleton_cells": [("C_out[i] = cnt[n] > 0 ?", "C_out[i] = cnt[n] > 1 ?")],
    "second_best_not_shifted": [("                d2 = d1;\n", "")],
    "d_prev_not_updated": [("            D_prev = D;\n", "")],
    "reseed_splits_singletons": [("if (counts[b] < 2) break;", "if (counts[b] < 1) break;")],
    "distance_accumulates_in_fp32": [("{\n    double s = 0.0;\n    for (int32_t l = 0; l < L; ++l) {\n        double d =",
                                      "{\n    float s = 0.0f;\n    for (int32_t l = 0; l < L; ++l) {\n        double d =")],
    "update_reads_column_major": [("sum[(int64_t)n * L + l] += (double)X[m * L + l];",
                                   "sum[(int64_t)n * L + l] += (double)X[m + (int64_t)l * M];")],
    "pass_counter_starts_at_1": [("for (int32_t pass = 0;; ++pass)", "for (int32_t pass = 1;; ++pass)")],
    # gradient at a fixed cell table
    "grad_c_wrong_sign": [("gC[i] = 2.0 * ((double)cnt[n] * C[i] + gC[i]);",
                           "gC[i] = 2.0 * ((double)cnt[n] * C[i] - gC[i]);")],
    "grad_c_count_dropped": [("gC[i] = 2.0 * ((double)cnt[n] * C[i] + gC[i]);",
                              "gC[i] = 2.0 * (C[i] + gC[i]);")],
    "grad_x_factor_dropped": [("gX[m * L + l] = 2.0 *", "gX[m * L + l] = 1.0 *")],
    "grad_x_wrong_sign": [("2.0 * ((double)X[m * L + l] - C[(int64_t)a[m] * L + l])",
                           "2.0 * (C[(int64_t)a[m] * L + l] - (double)X[m * L + l])")],
}


def _plant(src: str, edits) -> str:
    for old, new in edits:
        assert src.count(old) == 1, f"the text to replace occurs {src.count(old)} times: {old!r}"
        src = src.replace(old, new)
    return src


def _run_pins(lib: str):
    env = dict(os.environ)
    env[oracle.LIBRARY_ENV] = lib
    env["OMP_NUM_THREADS"] = "2"
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_fail_on_every_planted_mistake(tmp_path):
    with open(SRC) as f:
        src = f.read()
    jobs = {"unmodified": src}
    for name, edits in MUTANTS.items():
        jobs[name] = _plant(src, edits)
    libs = {}
    for name, text in jobs.items():
        c = tmp_path / f"{name}.c"
        c.write_text(text)
        libs[name] = oracle.compile_source(str(c), str(tmp_path / f"lib{name}.so"))
    workers = max(1, min(len(libs), (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as pool:
        res = dict(zip(libs, pool.map(_run_pins, libs.values())))
    base = res.pop("unmodified")
    assert base.returncode == 0, base.stdout[-2000:] + base.stderr[-2000:]
    # returncode 1: pytest ran and a pin failed (not a crash or a collection error)
    missed = {n: r.returncode for n, r in res.items() if r.returncode != 1}
    assert not missed, f"planted mistakes no pin caught (pytest exit codes): {missed}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_text_is_present(name):
    """Every planted mistake still applies to the current oracle source."""
    with open(SRC) as f:
        _plant(f.read(), MUTANTS[name])
