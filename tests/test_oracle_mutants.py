"""The oracle's pins must reject plausible mistakes.  Each case plants one
mistake in a temporary copy of oracle.c (a dropped term, a wrong bound, a
reversed comparison ...), builds it, routes the oracle through it and checks
that some pin of tests/test_oracle_pins.py fails.  CPU only."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = [
    ("separation_off_by_one", "for (uint32_t z = x + 1; z <= y; z++) {\n        const uint32_t q",
     "for (uint32_t z = x + 1; z < y; z++) {\n        const uint32_t q"),
    ("block_barrier_orders_blocks", "if (!grid_only || p->slot_level[k] == 1) return 1;", "return 1;"),
    ("shared_arrays_cross_blocks", "const int open_cross = !shared && ", "const int open_cross = "),
    ("same_thread_races", "if (same && t1 == t2) continue;", ""),
    ("clause_range_shifted", "if (orc_pos(p, k) == st[z] - 1u) m |= 1u << k;",
     "if (orc_pos(p, k) == st[z] % 24u) m |= 1u << k;"),
    ("inter_clause_not_grid_only", "clauses[n++] = orc_slots_between(p, st, x, y) & grid;",
     "clauses[n++] = orc_slots_between(p, st, x, y);"),
    ("tie_break_reversed", "(wt == best_w && x < best_x)", "(wt == best_w && x > best_x)"),
    ("forbidden_ignored", "if (x & forbidden) continue;", ""),
    ("negative_clause_wrong", "if ((x & neg[c]) == neg[c]) ok = 0;", "if ((x & neg[c]) != 0) ok = 0;"),
    ("divergence_ignores_mask", "if (!((mask >> k) & 1u) || p->slot_guard_k[k] == 0) continue;",
     "if (p->slot_guard_k[k] == 0) continue;"),
    ("probe_returned", "if (!any && !probe) {", "if (!any) {"),
    ("existing_not_forced", "const uint32_t forced = mode == 0 ? p->existing_mask : 0;",
     "const uint32_t forced = 0;"),
    ("divergence_not_forbidden", "forbidden |= w.diverge;", ""),
    ("perm_offset_dropped", "((uint64_t)tid + (uint64_t)p->c[s] * blk + p->b[s] + d) % M;",
     "((uint64_t)tid + (uint64_t)p->c[s] * blk + d) % M;"),
    ("block_term_dropped", "(((uint64_t)p->a[s] * tid + (uint64_t)p->c[s] * blk + p->b[s] + d) % M)",
     "(((uint64_t)p->a[s] * tid + p->b[s] + d) % M)"),
    ("read_read_pairs", "if (p->op[i] != 1 && p->op[j] != 1) continue;", ""),
    ("guard_negated", "return k == 0 || tid % k == r;", "return k == 0 || tid % k != r;"),
    ("weight_of_all_slots", "if ((x >> k) & 1u) wt += w[k];", "wt += w[k];"),
    ("greedy_tie_to_higher_index", "(uint64_t)hits * w[best] > (uint64_t)best_hits * w[k]",
     "(uint64_t)hits * w[best] >= (uint64_t)best_hits * w[k]"),
    ("greedy_not_minimal", "        if (ok) x = y;", "        (void)ok;"),
    ("pairs_double_counted",
     "if (x == y && (uint64_t)b2 * T + t2 < (uint64_t)b1 * T + t1) continue;", ""),
    # counted loops
    ("loop_counter_term_dropped", "const uint64_t d = p->iter_coef ? (uint64_t)p->iter_coef[s] * it : 0;",
     "const uint64_t d = 0;"),
    ("instance_index_taken_for_statement", "const uint32_t q = st[z] - 1;", "const uint32_t q = z - 1;"),
    ("loop_trips_off_by_one", "for (uint32_t t2 = 0; t2 < p->loop_trips[l]; t2++)",
     "for (uint32_t t2 = 0; t2 + 1 < p->loop_trips[l]; t2++)"),
    ("inner_statements_use_outer_counter", "orc_emit(p, p->loop_lo[l], p->loop_hi[l], l, t2, st, it, n);",
     "orc_emit(p, p->loop_lo[l], p->loop_hi[l], l, t, st, it, n);"),
    ("loop_rows_past_statements_ignored",
     "for (uint32_t i = 0; i < 32; i++)\n            if (w.intra[i] | w.inter[i]) any = 1;",
     "for (uint32_t i = 0; i < p->n_stmts; i++)\n            if (w.intra[i] | w.inter[i]) any = 1;"),
    ("negative_clauses_ignored", "clauses, n_cl, p->neg, p->n_neg, forced, forbidden, &m, &wt)",
     "clauses, n_cl, NULL, 0, forced, forbidden, &m, &wt)"),
    ("greedy_negative_check_skipped", "                if ((m & p->neg[c]) == p->neg[c]) ok = 0;", ""),
    ("head_slot_taken_after_statement", "if (orc_pos(p, k) == st[z] - 1u) m |= 1u << k;",
     "if (orc_pos(p, k) == st[z - 1]) m |= 1u << k;"),
    ("slot_position_ignored", "return p->slot_pos ? p->slot_pos[k] : k;", "return k;"),
    ("clauses_kept_as_multiset", "if (u == 0 || clauses[u - 1] != clauses[t]) clauses[u++] = clauses[t];",
     "clauses[u++] = clauses[t];"),
    # the word-grouped check
    ("words_same_thread_races", "if (same && ax[a].tid == ay[c].tid) continue; /* one thread */", ""),
    ("words_pairs_count_same_thread", "out->access_pairs += bb * (nx * ny - nxy);",
     "out->access_pairs += bb * nx * ny;"),
    ("words_unordered_cross_pairs_doubled", "out->access_pairs += bb * (bb - 1) / 2 * nx * nx;",
     "out->access_pairs += bb * (bb - 1) * nx * nx;"),
    ("words_merge_skips_a_word", "u = u1;\n                    v = v1;", "u = u1;\n                    v = v1 + 1;"),
    ("words_stops_at_first_scope", "(open_same > found_same || open_cross > found_cross)",
     "(open_same > found_same && open_cross > found_cross)"),
]


def _all_pins():
    for case in pins.GOLD["cases"]:
        yield lambda c=case: pins.test_listing_checks(c)
        yield lambda c=case: pins.test_listing_repairs(c)
    for case in pins.GOLD["solver_cases"]:
        yield lambda c=case: pins.test_solver_paper_example(c)
    yield pins.test_greedy_paper_example
    for case in pins.GOLD["greedy_cases"]:
        yield lambda c=case: pins.test_greedy_worked_cases(c)
    for case in pins.GOLD["loop_cases"]:
        yield lambda c=case: pins.test_loop_cases(c)
    for case in pins.GOLD["neg_cases"]:
        yield lambda c=case: pins.test_neg_cases(c)
    for case in pins.GOLD["site_cases"]:
        yield lambda c=case: pins.test_site_cases(c)
    for s in range(16):
        yield lambda s=s: pins.test_check_matches_flag_reset_detector(s)
        yield lambda s=s: pins.test_check_matches_affine_closed_form(s)
        yield lambda s=s: pins.test_access_pairs_closed_form(s)
        yield lambda s=s: pins.test_solve_matches_interval_dp(s)
        yield lambda s=s: pins.test_solve_matches_milp(s)
        yield lambda s=s: pins.test_check_antitone_in_mask(s)
        yield lambda s=s: pins.test_clause_is_exact_filter(s)
        yield lambda s=s: pins.test_repair_path_independence(s)
        yield lambda s=s: pins.test_greedy_minimal_and_within_johnson_bound(s)
        yield lambda s=s: pins.test_loop_check_matches_interpreter(s)
        yield lambda s=s: pins.test_loop_repair_path_independence(s)
        yield lambda s=s: pins.test_loop_clause_is_exact_filter(s)
        yield lambda s=s: pins.test_repair_path_independence_with_negative_clauses(s)
        yield lambda s=s: pins.test_site_check_matches_interpreter(s)
        yield lambda s=s: pins.test_site_repair_path_independence(s)
        yield lambda s=s: pins.test_check_words_matches_check(s)
        yield lambda s=s: pins.test_repair_words_matches_repair(s)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(name, old, new, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) >= 1, "mutation site must exist"  # every copy of the site is mutated
    mutated = tmp_path / "oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o",
                           str(lib), str(mutated)])
    killed = False
    with oracle.using_library(str(lib)):
        for pin in _all_pins():
            try:
                pin()
            except AssertionError:
                killed = True
                break
    assert killed, f"no pin rejects the planted mistake '{name}'"
