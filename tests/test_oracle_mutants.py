"""The oracle's pins catch plausible mistakes (CPU).

Each case below plants one mistake in a copy of ``oracle/gk_oracle.c`` (a flipped
sign, a dropped term, a wrong index, a step out of order: the kinds of error a
restatement of Algorithms 1-2 and Eq. 1-3 could contain), builds that copy into a
library of its own in a temporary directory, and runs the oracle's pin tests
(``tests/test_oracle.py``, ``tests/test_oracle_trajectory.py``) against it in a
separate process.  The quality measures of Section 5 (``oracle/quality.py``) get the
same treatment against the CPU tests of ``tests/test_quality.py``.  The pins must fail
for every planted mistake.  The committed oracle is never modified: the copy is loaded
in place of it only inside that process.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gk_oracle.c")
HDR = os.path.join(ROOT, "oracle", "gk_oracle.h")
PINS = ["tests/test_oracle.py", "tests/test_oracle_trajectory.py"]

# name -> [(text in gk_oracle.c, its replacement), ...]; every text occurs exactly once.
# Left out as equivalent: running the movement loop to it <= maxIter (the body already
# leaves at the last iteration, so only maxIter = 0 would tell).
MUTANTS = {
    # Eq. 1 and the balance test (Section 2, Section 4.2, Algorithm 1)
    "eq1_gamma_inverted": [("double gamma = target / S[c];", "double gamma = S[c] / target;")],
    "eq1_no_root": [("factor = sqrt(gamma);", "factor = gamma;")],
    "eq1_clamp_upper": [("if (factor > 1.05) factor = 1.05;", "if (factor > 1.5) factor = 1.5;")],
    "eq1_clamp_lower": [("if (factor < 0.95) factor = 0.95;", "if (factor < 0.5) factor = 0.5;")],
    "eq1_empty_block_kept": [("factor = INFINITY;", "factor = 1.0;")],
    "eq1_target_ceiling": [("double target = W / (double)k;", "double target = ceil(W / (double)k);")],
    "bound_no_ceiling": [("return (1.0 + eps) * ceil(W / (double)k);",
                          "return (1.0 + eps) * (W / (double)k);")],
    "bound_strict": [("if (max_s <= bound) return 1;", "if (max_s < bound) return 1;")],
    "imbalance_against_target": [("if (imbalance) *imbalance = max_s / ceil_avg - 1.0;",
                                  "if (imbalance) *imbalance = max_s / (W / (double)k) - 1.0;")],
    # effective distance and argmin (Section 4.2)
    "distance_times_influence": [("double eff = sqrt(ss) / I[c];", "double eff = sqrt(ss) * I[c];")],
    "distance_squared": [("double eff = sqrt(ss) / I[c];", "double eff = ss / I[c];")],
    "ties_to_highest_index": [("if (eff < best) {", "if (eff <= best) {")],
    "runner_up_dropped": [("} else if (eff < second) {", "} else if (0) {")],
    # block weights (Algorithm 1 localBlockSizes)
    "block_weights_unweighted": [("S[A[p]] += wp;", "S[A[p]] += 1.0;")],
    # initial centers (Algorithm 2)
    "centers_without_offset": [("int64_t idx = i * n / k + n / (2 * (int64_t)k);",
                                "int64_t idx = i * n / k;")],
    # movement and beta (Algorithm 2, Eq. 2-3)
    "mean_by_count": [("C_new[c * d + j] = sx[c * d + j] / sw[c];",
                       "C_new[c * d + j] = sx[c * d + j] / (double)cnt[c];")],
    "beta_over_all_blocks": [("*beta = nonempty > 0 ? diam_sum / (double)nonempty : 0.0;",
                              "*beta = diam_sum / (double)k;")],
    "beta_squared_diagonal": [("diam_sum += sqrt(diag);", "diam_sum += diag;")],
    "delta_squared": [("delta[c] = sqrt(dd);", "delta[c] = dd;")],
    # erosion (Eq. 2-3)
    "erosion_sign": [("double t = -delta[c] / beta;", "double t = delta[c] / beta;")],
    "erosion_alpha_form": [("alpha = 2.0 / (1.0 + exp(t)) - 1.0;", "alpha = 1.0 / (1.0 + exp(t));")],
    "erosion_exponent": [("I[c] = exp((1.0 - alpha) * log(I[c]));", "I[c] = exp(alpha * log(I[c]));")],
    # the loop's composition (Algorithms 1-2 as read)
    "erode_the_used_influence": [(
        "        if (opt->erosion) or_erosion(delta, beta, k, I);\n    }\n    if (!balanced) {",
        "        if (opt->erosion) {\n"
        "            memcpy(I, I_used, (size_t)k * sizeof(double));\n"
        "            or_erosion(delta, beta, k, I);\n"
        "        }\n    }\n    if (!balanced) {")],
    "erode_before_convergence_test": [
        ("        if (max_delta < thr) {\n            res->converged = 1;",
         "        if (opt->erosion) or_erosion(delta, beta, k, I);\n"
         "        if (max_delta < thr) {\n            res->converged = 1;"),
        ("        if (opt->erosion) or_erosion(delta, beta, k, I);\n    }\n    if (!balanced) {",
         "    }\n    if (!balanced) {")],
    "move_in_last_phase": [("        if (it == opt->max_iter - 1) break;\n", "")],
    "used_influence_after_update": [(
        "            for (int c = 0; c < k; ++c) I_used[c] = I[c];\n"
        "            balanced = or_balance_update(S, W, k, d, eps, I, &imbalance);\n"
        "            if (balanced) break;\n        }\n        /* Algorithm 2",
        "            balanced = or_balance_update(S, W, k, d, eps, I, &imbalance);\n"
        "            for (int c = 0; c < k; ++c) I_used[c] = I[c];\n"
        "            if (balanced) break;\n        }\n        /* Algorithm 2")],
    "no_final_passes": [("    if (!balanced) {\n        for (int fp", "    if (0) {\n        for (int fp")],
    # Hilbert curve (Section 4.1) and its grid
    "hilbert_no_mirror": [("flip[0] ^= 1; /* mirror slot 0 */", "/* no mirror */")],
    "hilbert_no_parity": [("digit = (digit << 1) | (uint64_t)(prefix ^ parity_above);",
                           "digit = (digit << 1) | (uint64_t)prefix;")],
    "hilbert_no_exchange": [("                perm[0] = perm[i];\n                perm[i] = tp;\n",
                             "                (void)tp;\n")],
    "grid_not_tight": [("return (f == 0.5) ? e - 1 : e;", "return e;")],
    "quantise_rounds": [("return (uint32_t)floor(scaled);", "return (uint32_t)floor(scaled + 0.5);")],
    "f32_subtract_in_f64": [("float v = x[p * d + j] - lo[j]; /* one FP32 subtraction */",
                             "double v = (double)x[p * d + j] - (double)lo[j];")],
    "extent_of_the_first_axis": [(
        "    for (int j = 0; j < d; ++j)\n        if (hi[j] - lo[j] > s) s = hi[j] - lo[j];\n"
        "    int b = hilbert_bits(d);",
        "    for (int j = 0; j < 1; ++j)\n        if (hi[j] - lo[j] > s) s = hi[j] - lo[j];\n"
        "    int b = hilbert_bits(d);")],
    "top_cell_not_clamped": [("if (scaled >= top) return (uint32_t)(top - 1.0);",
                              "if (scaled > top) return (uint32_t)(top - 1.0);")],
    "box_starts_at_zero": [(
        "        lo[j] = INFINITY;\n        hi[j] = -INFINITY;\n    }\n"
        "    for (int64_t p = 0; p < n; ++p) {\n        for (int j = 0; j < d; ++j) {\n            double v",
        "        lo[j] = 0.0;\n        hi[j] = 0.0;\n    }\n"
        "    for (int64_t p = 0; p < n; ++p) {\n        for (int j = 0; j < d; ++j) {\n            double v")],
    "f32_extent_rounded": [("        double e = (double)hi[j] - (double)lo[j];",
                            "        double e = (double)(hi[j] - lo[j]);")],
    # sort (Algorithm 2 sortGlobal)
    "sort_unstable": [("if (keys[a[j]] < keys[a[i]])", "if (keys[a[j]] <= keys[a[i]])")],
    # the bootstrap's data movement and the loop bounds (Algorithm 2)
    "scatter_inverted": [(
        "    int st = or_balanced_kmeans(xs, ws, n, d, k, eps, opt, C_out, I, I_out, NULL, As, res);\n"
        "    for (int64_t i = 0; i < n; ++i) A_out[perm[i]] = As[i];",
        "    int st = or_balanced_kmeans(xs, ws, n, d, k, eps, opt, C_out, I, I_out, NULL, As, res);\n"
        "    for (int64_t i = 0; i < n; ++i) A_out[i] = As[perm[i]];")],
    "weights_not_permuted": [("        if (ws) ws[i] = w[perm[i]];\n    }\n    double *I",
                              "        if (ws) ws[i] = w[i];\n    }\n    double *I")],
    "centers_from_unsorted_points": [(
        "    or_sfc_centers(xs, n, d, k, C_out);\n    for (int c = 0; c < k; ++c) I[c] = 1.0;\n    int st",
        "    or_sfc_centers(xd, n, d, k, C_out);\n    for (int c = 0; c < k; ++c) I[c] = 1.0;\n    int st")],
    "influence_starts_at_two": [(
        "    or_sfc_centers(xs, n, d, k, C_out);\n    for (int c = 0; c < k; ++c) I[c] = 1.0;\n    int st",
        "    or_sfc_centers(xs, n, d, k, C_out);\n    for (int c = 0; c < k; ++c) I[c] = 2.0;\n    int st")],
    "hilbert_bits_3d": [("return d == 2 ? 32 : 21;", "return d == 2 ? 32 : 20;")],
    "delta_threshold_scale": [("opt->delta_threshold : 1e-4 * extent;", "opt->delta_threshold : 1e-3 * extent;")],
    "one_balance_pass_more": [(
        "        for (int bp = 0; bp < opt->max_balance_iter; ++bp) {\n"
        "            or_assign(x, n, d, C, I, k, A, NULL, NULL, opt->threads);",
        "        for (int bp = 0; bp <= opt->max_balance_iter; ++bp) {\n"
        "            or_assign(x, n, d, C, I, k, A, NULL, NULL, opt->threads);")],
    # random initialization (Section 4.5)
    "sample_by_input_index": [("mark[rank[order[i]]] = 1;", "mark[order[i]] = 1;")],
    "sample_rounds_one_more": [("while (r < 62 && (m0 << r) < n) ++r;",
                                "while (r < 62 && (m0 << r) <= n) ++r;")],
    "sample_first_not_100k": [("int64_t m0 = sample0 > 0 ? sample0 : 100 * (int64_t)k;",
                               "int64_t m0 = sample0 > 0 ? sample0 : 10 * (int64_t)k;")],
    "sample_unweighted": [("            if (wr) wr[j] = ws[pos];", "            if (wr) wr[j] = 1.0;")],
    "sample_round_without_erosion": [(
        "        if (opt->erosion) or_erosion(delta, beta, k, I);\n    }\n    or_options rest",
        "    }\n    or_options rest")],
    "sampled_iterations_not_shared": [("rest.max_iter = opt->max_iter - R;",
                                       "rest.max_iter = opt->max_iter;")],
}


QSRC = os.path.join(ROOT, "oracle", "quality.py")
QPINS = ["tests/test_quality.py"]

# mistakes in the quality measures (Section 5) and the diameter sweeps as read.  Left out
# as equivalent (no input tells them apart): counting self-loops (never foreign, never a
# new vertex), the bound from the last sweep only (every sweep starts at a vertex the one
# before reached last, so eccentricities do not decrease), and dropping the empty-block
# case (an empty block is "connected" with bound 0 anyway).
QMUTANTS = {
    "edge_cut_not_halved": [('"edge_cut": int(ext.sum() // 2)', '"edge_cut": int(ext.sum())')],
    "comm_counts_edges": [("pairs = np.unique(np.stack([v[foreign], bu[foreign]], axis=1), axis=0)",
                           "pairs = np.stack([v[foreign], bu[foreign]], axis=1)")],
    "comm_credited_to_other_block": [("comm = np.bincount(block[pairs[:, 0]], minlength=k)",
                                      "comm = np.bincount(pairs[:, 1], minlength=k)")],
    "comm_includes_own_block": [("pairs = np.unique(np.stack([v[foreign], bu[foreign]], axis=1), axis=0)",
                                 "pairs = np.unique(np.stack([v, bu], axis=1), axis=0)")],
    "bfs_leaves_the_block": [("fresh = (block[u] == block[tail]) & (dist[u] < 0)",
                              "fresh = dist[u] < 0")],
    "first_start_largest_index": [(
        "    start = np.full(k, n, dtype=np.int64)\n    np.minimum.at(start, block, ids)",
        "    start = np.full(k, -1, dtype=np.int64)\n    np.maximum.at(start, block, ids)")],
    "next_start_largest_index": [(
        "        start = np.full(k, n, dtype=np.int64)\n        np.minimum.at(start, block[last], last)",
        "        start = np.full(k, -1, dtype=np.int64)\n        np.maximum.at(start, block[last], last)")],
    "next_start_not_farthest": [("last = np.nonzero(dist == ecc[block])[0]",
                                 "last = np.nonzero(dist == 0)[0]")],
    "harmonic_without_disconnected": [("m = int(big.sum())", "m = int(pos.sum())")],
    "harmonic_over_single_vertices": [("big = size >= 2", "big = size >= 1")],
    "arithmetic_mean": [("hm = 0.0 if m == 0 else (np.inf if s == 0.0 else m / s)",
                         "hm = 0.0 if m == 0 else float(diam[pos].sum()) / m")],
}


def _mutant_source(name):
    text = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert text.count(old) == 1, f"{name}: the text to replace occurs {text.count(old)} times"
        text = text.replace(old, new)
    return text


def _qmutant_source(name):
    text = open(QSRC).read()
    for old, new in QMUTANTS[name]:
        assert text.count(old) == 1, f"{name}: the text to replace occurs {text.count(old)} times"
        text = text.replace(old, new)
    return text


def test_every_mutant_applies_to_the_current_oracle():
    for name in MUTANTS:
        assert _mutant_source(name) != open(SRC).read()
    for name in QMUTANTS:
        assert _qmutant_source(name) != open(QSRC).read()


_RUNNER = """
import sys
import oracle
oracle._SRC = sys.argv[1]
oracle._LIB_PATH = sys.argv[2]
import pytest
sys.exit(pytest.main(["-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + sys.argv[3:]))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(name, tmp_path):
    src = tmp_path / "gk_oracle.c"
    src.write_text(_mutant_source(name))
    shutil.copy(HDR, tmp_path / "gk_oracle.h")
    lib = tmp_path / "liboracle.so"
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _RUNNER, str(src), str(lib), *PINS], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert lib.exists(), r.stdout[-2000:] + r.stderr[-2000:]
    # exit status 1: tests ran and at least one failed (not a crash, not a collection error)
    assert r.returncode == 1, f"{name} was not caught:\n{r.stdout[-1500:]}"


_QRUNNER = """
import importlib.util
import sys
import oracle
spec = importlib.util.spec_from_file_location("oracle.quality", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
sys.modules["oracle.quality"] = mod
oracle.quality = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + sys.argv[2:]))
"""


@pytest.mark.parametrize("name", sorted(QMUTANTS))
def test_quality_pins_reject_planted_mistake(name, tmp_path):
    src = tmp_path / "quality.py"
    src.write_text(_qmutant_source(name))
    r = subprocess.run([sys.executable, "-c", _QRUNNER, str(src), *QPINS], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"{name} was not caught:\n{r.stdout[-1500:]}{r.stderr[-800:]}"
