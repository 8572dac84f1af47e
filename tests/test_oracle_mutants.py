"""The pins must catch plausible mistakes. Each case plants one mistake in a
copy of the oracle's C source (on the CPU, never in the product), builds it,
and runs the pin and invariant tests against it: at least one must fail."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "biolog_oracle.c")

MUTANTS = {
    "drop_hq_to_first_field_su_leg": ("if (k == 0) { ra.LSU[g] += c->D[(size_t)prev_anchor * N + fn]; ops += 2; }",
                                      "if (k == 0) { ops += 2; }"),
    "single_shuttle_leg": ("shuttle += 2.0 * (double)nf", "shuttle += 1.0 * (double)nf"),
    "su_route_not_multiplied": ("(double)nsu * ra.LSU[g]", "ra.LSU[g]"),
    "hu_route_not_multiplied": ("(double)nhu * ra.LHU[g]", "ra.LHU[g]"),
    "mean_over_fields_not_bps": ("dsum += sb / (double)p->blen[b];", "dsum += sb; nbp += p->blen[b] - 1;"),
    "ceil_off_at_integers": ("int64_t nf = ceil_ratio(c->supply[f] * (double)nsu, capsum);",
                             "int64_t nf = (int64_t)floor(c->supply[f] * (double)nsu / capsum) + 1;"),
    "hu_accept_sign": ("if (tmx < ref || is_last) {\n                moved = h;",
                       "if (tmx > ref || is_last) {\n                moved = h;"),
    "critical_su_smallest": ("if (star < 0 || c->su_fill[s] > c->su_fill[star]) star = s;",
                             "if (star < 0) star = s;"),
    "no_demand_check": ("if (!(s >= c->demand[b])) { res->ops = ops; return; }", "(void)s;"),
    "philox_multiplier": ("M1 = 0xCD9E8D57u", "M1 = 0xCD9E8D55u"),
    "init_ties_to_highest": ("if (best < 0 || d < bd) { best = b; bd = d; }\n        }\n        chain[k]",
                             "if (best < 0 || d <= bd) { best = b; bd = d; }\n        }\n        chain[k]"),
    "gate_inclusive": ("(gate == 1 && tmax > tmax_star)", "(gate == 1 && tmax >= tmax_star)"),
    "no_termination_undo": ("if (!(nm < old_max)) {\n            hu_tour[moved] = gmin;",
                            "if (0) {\n            hu_tour[moved] = gmin;"),
    "slot_range_short": ("mv[3] = (int16_t)draw_below(r[2], (uint32_t)(len + 1));\n    } else {",
                         "mv[3] = (int16_t)draw_below(r[2], (uint32_t)(len > 0 ? len : 1));\n    } else {"),
    "hu_round_robin_reversed": ("for (int k = 0; k < c->H; ++k) hu_tour[c->hu_sorted[k]] = act[k % na];",
                                "for (int k = 0; k < c->H; ++k) hu_tour[c->hu_sorted[k]] = act[na - 1 - k % na];"),
    "wait_fill_sign": ("return drive - fill;", "return drive + fill;"),
    # decision margins (the gaps that decide which candidates escape the strict FP32-FP64 comparison)
    "margin_pick_smaller_scale": ("if (g != a) note_gap(site0, margin, val[a], val[g], fmax(scale[a], scale[g]));",
                                  "if (g != a) note_gap(site0, margin, val[a], val[g], fmin(scale[a], scale[g]));"),
    "margin_min_pick_wrong_operand": ("note_gap(site0 + 2, margin, val[m], val[g], fmax(scale[m], scale[g]));",
                                      "note_gap(site0 + 2, margin, val[a2], val[g], fmax(scale[a2], scale[g]));"),
    "margin_hu_accept_dropped": ("if (!is_last) note_gap(GAP_HU_ACCEPT, margin, tmx, ref, fmax(tmx, ref));",
                                 "(void)is_last;"),
    "margin_su_accept_counts_last": ("if (!is_last) note_gap(GAP_SU_ACCEPT,", "note_gap(GAP_SU_ACCEPT,"),
    "margin_su_accept_wrong_scale": ("fmax(sc_mx, ref_scale)", "fmax(sc_mn, ref_scale)"),
    "margin_hu_stop_wrong_operand": ("note_gap(GAP_HU_STOP, margin, nm, old_max, fmax(nm, old_max));",
                                     "note_gap(GAP_HU_STOP, margin, nm, Tc[gmax2], fmax(nm, Tc[gmax2]));"),
    "margin_su_stop_new_scale": ("fmax(nm_scale, sscmx)", "nm_scale"),
    "margin_gate_dropped": ("note_gap(GAP_GATE, &margin, tmax, tmax_star, fmax(tmax, tmax_star));", "(void)0;"),
    "margin_keeps_largest": ("if (m < *margin) *margin = m;", "if (m > *margin || isinf(*margin)) *margin = m;"),
    # chained moves (Step 8 repeated)
    "second_move_drawn_on_base": ("draw_move(c, prm, iter, i, j, out, mv + 4 * j);",
                                  "draw_move(c, prm, iter, i, j, base, mv + 4 * j);"),
    "move_counter_word3_shared": ("return j == 0 ? 0u : (uint32_t)j + 1u;", "return (uint32_t)j;"),
    "margin_su_scale_max_of_terms": ("if (scale) *scale = fabs(drive) + fabs(fill);",
                                     "if (scale) *scale = fmax(fabs(drive), fabs(fill));"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=gnu11", "-O1", "-fPIC", "-shared", "-fopenmp", "-w", "-o", str(so), str(mutant),
                    "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_invariants.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
