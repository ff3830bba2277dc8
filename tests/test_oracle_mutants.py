"""The oracle's pins catch planted mistakes.

Each mutant is a copy of the oracle's C source with one plausible mistake,
compiled into a temporary library.  The committed pin suite
(test_oracle_pins.py, test_oracle_flips.py) then runs against that copy in a child process
(ORACLE_LIB points the binding at it) and must fail.  The mistakes are
planted in the oracle on the CPU only; nothing here touches the CUDA library.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cse_oracle.c")

# (name, the passage the planted mistake violates, original text, mutated text)
MUTANTS = [
    ("philox_multiplier", "Philox4x32-10 round constant",
     "uint64_t p0 = (uint64_t)0xD2511F53u * c0;", "uint64_t p0 = (uint64_t)0xD2511F57u * c0;"),
    ("philox_output_order", "Philox4x32-10 round output",
     "uint32_t n1 = (uint32_t)p1;", "uint32_t n1 = (uint32_t)p0;"),
    ("naive_counts_nnz", "Section 3.2.1: A_naive adds nnz - 1 per row",
     "        s += nnz - 1;", "        s += nnz;"),
    ("pair_sign_from_one_entry", "Section 3.2.1: the pair's sign is alpha_i alpha_j",
     "KEY(i, j, row[i] * row[j] < 0)", "KEY(i, j, row[i] < 0)"),
    ("substitution_ignores_sign", "Section 3.2.1: rows hold x_i + s x_j up to a common sign",
     "row[j] == s * row[i]", "row[j] == row[i]"),
    ("substitution_keeps_x_j", "Algorithm 1: both coefficients of the pair are cleared",
     "            row[i] = 0;\n            row[j] = 0;\n", "            row[i] = 0;\n"),
    ("cost_without_fresh_variables", "Section 3.2.1: Cost = n_f + A_naive",
     "return P->nf + naive_rows(P->coef, M->rows, P->ncols, S->cap);",
     "return naive_rows(P->coef, M->rows, P->ncols, S->cap);"),
    ("single_occurrences_are_candidates", "Algorithm 1: only pairs with c > 1 are substituted",
     "count_pairs(P->coef, M->rows, P->ncols, S->cap, 2,", "count_pairs(P->coef, M->rows, P->ncols, S->cap, 1,"),
    ("greedy_ties_to_last", "Greedy: lowest canonical key among the maxima",
     "if (cnt[t] > cnt[best]) best = t;", "if (cnt[t] >= cnt[best]) best = t;"),
    ("ga_index_off_by_one", "Greedy-Alternative: uniform over the ties",
     "uint32_t want = scale(u, (uint64_t)ties);", "uint32_t want = scale(u, (uint64_t)ties - 1);"),
    ("wr_boundary", "Weighted-Random: probability proportional to c - 1",
     "if (acc > x) return t;", "if (acc >= x) return t;"),
    ("gr_even_coin", "Greedy-Random: ga with probability 0.75",
     "coin < 0xC0000000u ?", "coin < 0x80000000u ?"),
    ("mix_cut", "Mixed: gi, ga, gr, wr in proportions 8:4:2:1",
     "return r < 8 ? OR_GI : r < 12", "return r < 7 ? OR_GI : r < 12"),
    ("gi_disjoint_sum_keeps_p", "Section 3.4.2: the sum runs over q != p",
     "int64_t d = total - wp - inter;", "int64_t d = total - inter;"),
    ("gi_coin_for_p_itself", "Section 3.4.2: the sum runs over q != p",
     "if (q != p) coin = coin_at(cs, p, q, 0, pos0);", "coin = coin_at(cs, p, q, 0, pos0);"),
    ("gi_beta_as_alpha", "Section 3.4.2: intersecting terms weigh beta (c_q - 1)",
     "(d << 16) + (int64_t)b * x)", "(d << 16) + (int64_t)a * x)"),
    ("gi_ties_to_last", "Greedy-Intersections: lowest canonical key on equal scores",
     "        if (best < 0 || s > best_s) {", "        if (best < 0 || s >= best_s) {"),
    ("gp_counts_single_pairs", "Greedy-Potential: new pairs that occur at least twice",
     "pot += (b - a) >= 2;", "pot += (b - a) >= 1;"),
    ("share_prefix_whole_list", "Section 3.5.2: a prefix of 1 to 3/4 of the shared list",
     "int32_t big_k = (3 * M->snap_len) / 4;", "int32_t big_k = M->snap_len;"),
    ("shared_coin_word", "shared coins: bit q & 31 of word (q >> 5) & 3",
     "o[(q >> 5) & 3]", "o[(q >> 5) & 1]"),
    ("brent_drops_k_index", "Section 3.1: the Brent equations",
     "int64_t want = (j == j2 && i == i2 && k == k2) ? 1 : 0;", "int64_t want = (j == j2 && i == i2) ? 1 : 0;"),
    ("alpha_half_open", "Section 3.4.2: alpha in [0, 0.5]",
     "int32_t oracle_alpha(uint32_t u) { return (int32_t)scale(u, 32769); }",
     "int32_t oracle_alpha(uint32_t u) { return (int32_t)scale(u, 32768); }"),
    ("beta_from_zero", "Section 3.4.2: beta in [0.5, 1]",
     "int32_t oracle_beta(uint32_t u) { return 32768 + (int32_t)scale(u, 32769); }",
     "int32_t oracle_beta(uint32_t u) { return (int32_t)scale(u, 65537); }"),
    ("run_strategy_boundary", "Section 3.5.1: strategy drawn in proportion to its weight",
     "            if (x < acc) {", "            if (x <= acc) {"),
    ("best_record_replaced_on_ties", "Section 3.5.2: a process keeps its lowest-cost run",
     "    if (c < P->best_cost) {", "    if (c <= P->best_cost) {"),
    ("fresh_variable_takes_x_j_sign", "Section 3.2.1: the row keeps its sign through x_k",
     "            row[k] = row[i];", "            row[k] = row[j];"),
    ("wr_total_counts_c", "Weighted-Random: weights c - 1",
     "for (int32_t t = 0; t < m; t++) total += (uint64_t)(cnt[t] - 1);",
     "for (int32_t t = 0; t < m; t++) total += (uint64_t)cnt[t];"),
    ("shared_coin_bit", "shared coins: bit q & 31 of word (q >> 5) & 3",
     "(q & 31)) & 1u)", "(q & 15)) & 1u)"),
    ("process_zero_not_greedy", "Section 3.5.1: process 0 starts with Greedy",
     "    if (pi == 0 && t == 0) {", "    if (pi == 0 && t < 0) {"),
    ("share_probability_scale", "Section 3.5.2: a run starts from a shared prefix with probability 40%",
     "uint64_t thr = ((uint64_t)S->permille << 32) / 1000u;", "uint64_t thr = ((uint64_t)S->permille << 32) / 100u;"),
    ("gp_score_ignores_count", "Greedy-Potential: (c - 1) first, then alpha times the potential",
     "int64_t sc = ((int64_t)(cnt[p] - 1) << 16) + (int64_t)a * pot;",
     "int64_t sc = (int64_t)a * pot;"),
    ("snapshot_replaced_on_ties", "Section 3.5.2: the shared solution changes only when beaten",
     "M->procs[win].best_cost < M->snap_cost", "M->procs[win].best_cost <= M->snap_cost"),
    ("gi_coins_same_every_step", "reading R9: coins drawn afresh at every step",
     "draw4(cs->seed, cs->proc, cs->t, cs->mat, PU_GI, (uint32_t)blk, cs->keys[p], cs->block);",
     "draw4(cs->seed, cs->proc, 0, cs->mat, PU_GI, (uint32_t)blk, cs->keys[p], cs->block);"),
    ("gi_coins_shared_by_all_p", "reading R9: coins independent per scored candidate p",
     "draw4(cs->seed, cs->proc, cs->t, cs->mat, PU_GI, (uint32_t)blk, cs->keys[p], cs->block);",
     "draw4(cs->seed, cs->proc, cs->t, cs->mat, PU_GI, (uint32_t)blk, 0, cs->block);"),
    ("gi_coin_biased", "Section 3.4.2: each intersecting term kept with probability 1/2",
     "return (int)((w >> (rho & 63)) & 1u);", "return (int)(((w >> (rho & 63)) & 3u) != 0);"),
    ("flip_sign_ignored", "Section 3.5.3: a flip of terms whose shared factor differs in sign",
     "const int sigma = same ? 1 : -1;", "const int sigma = 1;"),
    ("flip_z_unchanged", "Section 3.5.3: a flip rewrites two factors of two terms",
     "    for (int32_t i = 0; i < len[z]; i++) zm[i] = (int8_t)(zm[i] - zl[i]);\n", "\n"),
    ("flip_not_ternary", "Section 3.5.3: ternary flips keep every coefficient in {-1, 0, 1}",
     "        if (v < -1 || v > 1) return 0;\n        ynz |= v != 0;", "        ynz |= v != 0;"),
    ("mops_rewrite_words", "the method op count (R15): 6 per 64-bit word of a rewrite",
     "P->mops += 6 * (int64_t)((M->rows + 63) / 64) + rows_nnz_of_pair(", "P->mops += 6 * (int64_t)((M->rows + 31) / 32) + rows_nnz_of_pair("),
    ("mops_rows_after_rewrite", "the method op count (R15): nnz of the rewritten rows before the rewrite",
     "for (int32_t v = 0; v < ncols; v++) n += row[v] != 0;", "for (int32_t v = 0; v < ncols; v++) n += row[v] != 0 && v != i;"),
    ("mops_gi_terms_once", "the method op count (R15): 2 per intersect term",
     "(cs->shared ? 4 * (int64_t)m : 2 * terms)", "(cs->shared ? 4 * (int64_t)m : terms)"),
    ("mops_no_scan", "the method op count (R15): every selection scans m",
     "case OR_G: P->ops += 2 * (int64_t)P->m; P->mops += P->m;", "case OR_G: P->ops += 2 * (int64_t)P->m;"),
    ("ops_rewrite_term", "the op count: 10 per word for the rewrite",
     "P->ops += 10 * (int64_t)M->w32 + 5 * (int64_t)M->w32 * (nij + nu);",
     "P->ops += 8 * (int64_t)M->w32 + 5 * (int64_t)M->w32 * (nij + nu);"),
    ("ops_gi_terms", "the op count: 3 per intersecting term of gi",
     "ops += 3 * (int64_t)n_inter + 8 +", "ops += 2 * (int64_t)n_inter + 8 +"),
    ("ops_selection_scan", "the op count: 2 per candidate for g, ga, gr, wr",
     "case OR_G: P->ops += 2 * (int64_t)P->m;", "case OR_G: P->ops += (int64_t)P->m;"),
    ("patience_one_late", "Section 4: stop after 10 iterations without improvement",
     "if (patience > 0 && stale >= patience) break;", "if (patience > 0 && stale > patience) break;"),
]


def _build(tmp, name, old=None, new=None):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"{name}: the original text must occur exactly once"
        src = src.replace(old, new)
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src)
    lib = os.path.join(tmp, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I", os.path.dirname(SRC), "-o", lib, path,
                           "-lpthread"])
    return lib


def _run_pins(lib):
    env = dict(os.environ, ORACLE_LIB=lib)
    try:
        out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                              os.path.join(ROOT, "tests", "test_oracle_flips.py"),
                              "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                             cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return "timeout", ""
    return out.returncode, out.stdout[-2000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("mutants"))
    # the unchanged source, built the same way: the control that passes
    libs = {"unchanged": _build(tmp, "unchanged")}
    libs.update({name: _build(tmp, name, old, new) for name, _, old, new in MUTANTS})
    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        return dict(zip(libs, ex.map(_run_pins, libs.values())))


def test_unchanged_copy_passes_the_pins(results):
    rc, tail = results["unchanged"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(results, name):
    rc, tail = results[name]
    assert rc != 0, f"mutant {name} passed every pin:\n{tail}"
