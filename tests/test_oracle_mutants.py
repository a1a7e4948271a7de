"""Plants plausible mistakes in a copy of the oracle (CPU only) and checks that
the pins of test_oracle_pins.py catch every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "amg_oracle.c")

# (name, original text, mutated text, pins expected to fail)
MUTANTS = [
    ("prolongation_sign", "x[i] = x[i] + xc[l->agg[i]];", "x[i] = x[i] - xc[l->agg[i]];",
     "test_vcycle_closed_form_on_2x2_blocks"),
    ("restriction_drops_term", "else fc[I] = fc[I] + t[i];", "else fc[I] = t[i];",
     "test_vcycle_closed_form_on_2x2_blocks"),
    ("jacobi_without_omega", "x[i] = x[i] + omega * (f[i] - t[i]) / l->diag[i];",
     "x[i] = x[i] + (f[i] - t[i]) / l->diag[i];", "test_vcycle_closed_form_on_2x2_blocks"),
    ("galerkin_drops_term", "val_c[slot[J]] = val_c[slot[J]] + val[e];", "val_c[slot[J]] = val_c[slot[J]];",
     "test_worked_example_matches_paper"),
    ("tie_break_larger_index", "if (a->u != b->u) return a->u < b->u ? -1 : 1;",
     "if (a->u != b->u) return a->u > b->u ? -1 : 1;", "test_greedy_matching_bruteforce"),
    ("rounds_tie_break", "(tie_break == 1 ? j > pick[i] : j < pick[i])", "(tie_break == 1 ? j > pick[i] : j > pick[i])",
     "test_handshake_rounds_reach_greedy_matching"),
    ("numbering_by_largest", "if (mate[i] < 0 || i < mate[i]) agg[i] = C++;",
     "if (mate[i] < 0 || i > mate[i]) agg[i] = C++;", "test_aggregates_partition_and_numbering"),
    ("pcg_residual_sign", "r[i] = r[i] - alpha * q[i];", "r[i] = r[i] + alpha * q[i];",
     "test_pcg_matches_dense_solve_to_1e10"),
    ("bicgstab_p_update", "p[i] = r[i] + beta * (p[i] - omega * v[i]);", "p[i] = r[i] + beta * p[i];",
     "test_krylov_finite_termination_two_eigenvalues"),
    ("coarse_cg_steepest_descent", "      double beta = rz_new / rz;\n", "      double beta = 0.0 * rz_new / rz;\n",
     "test_coarse_cg_solver_agrees_with_dense or test_coarse_cg_finite_termination_two_eigenvalues"),
    ("coarse_cg_residual_sign", "x[i] += alpha * p[i]; r[i] -= alpha * q[i];",
     "x[i] += alpha * p[i]; r[i] += alpha * q[i];",
     "test_coarse_cg_solver_agrees_with_dense or test_coarse_cg_finite_termination_two_eigenvalues"),
    ("flexible_beta_sign", "beta = s / rz;", "beta = -s / rz;",
     "test_flexible_beta_keeps_consecutive_directions_a_conjugate"),
    ("flexible_beta_is_fletcher_reeves", "s += z[i] * (r[i] - rold[i]);", "s += z[i] * r[i];",
     "test_flexible_beta_keeps_consecutive_directions_a_conjugate"),
    ("nhem_never_descending", "nc = orc_nhem_dir(n, rp, ci, val, pass_index % 2, agg);",
     "nc = orc_nhem_dir(n, rp, ci, val, 0, agg);", "test_alternating_node_based_hierarchy"),
    ("nhem_descending_scan_wrong", "const int i = descending ? n - 1 - s : s;", "const int i = s;",
     "test_node_based_matching_scans_both_ways_by_hand"),
    ("stall_rule_not_strict", "if ((double)cur_n / (double)f->n > prm->stall_ratio) {",
     "if ((double)cur_n / (double)f->n >= prm->stall_ratio) {", "test_hierarchy_stops_before_a_stalled_level"),
    ("stall_ratio_against_finest", "if ((double)cur_n / (double)f->n > prm->stall_ratio) {",
     "if ((double)cur_n / (double)h->lev[0].n > prm->stall_ratio) {", "test_hierarchy_stops_before_a_stalled_level"),
    ("lu_no_pivoting", "if (fabs(a[(size_t)i * n + k]) > best)", "if (0 && fabs(a[(size_t)i * n + k]) > best)",
     "test_dense_lu_matches_numpy"),
    ("desc_tie_order_wrong_direction", "if (a->v != b->v) return a->v > b->v ? -1 : 1;",
     "if (a->v != b->v) return a->v < b->v ? -1 : 1;", "test_descending_tie_order_bruteforce"),
    ("scaled_weight_without_sqrt", "return fabs(a_ij) / sqrt(d[i] * d[j]);", "return fabs(a_ij) / (d[i] * d[j]);",
     "test_scaled_weight_bruteforce_and_invariance"),
    ("w_second_cycle_from_zero", "kind == 1) mg_cycle(h, k + 1, fc, xc, 1, 0);",
     "kind == 1) mg_cycle(h, k + 1, fc, xc, 1, 1);", "test_cycles_match_error_propagation_recursion"),
    ("w_single_coarse_cycle", "if (k + 1 < h->L && kind == 1)", "if (0 && k + 1 < h->L && kind == 1)",
     "test_cycles_match_error_propagation_recursion"),
    ("f_second_cycle_is_f", "kind == 2) mg_cycle(h, k + 1, fc, xc, 0, 0);",
     "kind == 2) mg_cycle(h, k + 1, fc, xc, 2, 0);", "test_cycles_match_error_propagation_recursion"),
    ("amg_solver_correction_sign", "x[i] = x[i] + z[i];", "x[i] = x[i] - z[i];",
     "test_amg_solver_iterates_closed_form"),
    ("amg_solver_stale_residual", "    orc_spmv(n, l->rp, l->ci, l->val, x, r);\n    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];\n    ++it;",
     "    ++it;", "test_amg_solver_iterates_closed_form"),
]


@pytest.mark.parametrize("name,orig,mut,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, mut, pins):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor for {name} not unique"
    bad = tmp_path / "amg_oracle_mutant.c"
    bad.write_text(src.replace(orig, mut))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(bad), "-lm"])
    env = dict(os.environ, AMG_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
