"""Planted mistakes: each mutant is a copy of the oracle with one plausible
error (a wrong sign, an off-by-one, a dropped or extra term, another search
order).  The pins in test_oracle_pins.py and test_oracle_search_pins.py must
fail on every one of them.  Mutants are built and
run on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pccp_oracle.c")

MUTANTS = {
    "temporal_ub_sign": ("r.value = ub[y] - d;", "r.value = ub[y] + d;"),
    "temporal_lb_off_by_one": ("r.value = lb[x] + d;", "r.value = lb[x] + d - 1;"),
    "reified_entailed_B_off_by_one": ("int ent_B = ub[y] <= lb[x] + d - 1;",
                                      "int ent_B = ub[y] <= lb[x] + d;"),
    "reified_B_lower_off_by_one": ("t.value = lb[y] - d + 1; }", "t.value = lb[y] - d; }"),
    "reified_rule2_drops_conjunct": ("if (ent_A && ent_B)", "if (ent_A)"),
    "reified_notA_strictness": ("t.value = lb[y] + 1; }", "t.value = lb[y]; }"),
    "reified_notB_over_tightens": ("t.var = y; t.value = lb[x] + d; } break;",
                                   "t.var = y; t.value = lb[x] + d + 1; } break;"),
    "reified_swapped_operands": ("int ent_notA = lb[x] >= ub[y] + 1;",
                                 "int ent_notA = lb[y] >= ub[x] + 1;"),
    "linear_keeps_self_term": ("if (j == k) continue;", ""),
    "linear_wrong_min_term": ("(a > 0) ? a * lb[v] : a * ub[v]", "(a > 0) ? a * ub[v] : a * lb[v]"),
    "floor_div_truncates": ("if ((a % b != 0) && (a < 0)) q -= 1;", ""),
    "ceil_for_negative_coef": ("t.value = ceil_div(-slack, -a);", "t.value = floor_div(-slack, -a);"),
    "jacobi_failure_check_skipped": ("if (empty_at(lb, ub, t.var)) { status = OM_FAILED; goto done; }\n        }\n      }\n    } else",
                                     "}\n      }\n    } else"),
    "sequential_failure_check_skipped": ("if (empty_at(lb, ub, t.var)) { status = OM_FAILED; goto done; }\n        }\n      }\n    }\n    if (!changed)",
                                         "}\n      }\n    }\n    if (!changed)"),
    "solve_records_nonimproving": ("if (s->o->mode == OM_OPTIMISE) record = 1;",
                                   "if (s->o->mode == OM_OPTIMISE) record = (s->r->solutions == 1);"),
    # search order: tie-break, split point, child order
    "first_fail_ties_to_higher_index": ("if (best < 0 || w < best_w)", "if (best < 0 || w <= best_w)"),
    "split_at_one_third": ("i64 mid = l + (u - l) / 2;", "i64 mid = l + (u - l) / 3;"),
    "split_left_takes_smaller_half": ("i64 mid = l + (u - l) / 2;", "i64 mid = l + (u - l - 1) / 2;"),
    "split_drops_lower_bound": ("i64 mid = l + (u - l) / 2;", "i64 mid = (u - l) / 2 > l ? (u - l) / 2 : l;"),
    "right_child_first": (
        """  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_UB; s->dval[depth] = mid;
  dfs(s, depth + 1);
  if (s->stop) return;
  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_LB; s->dval[depth] = mid + 1;
  dfs(s, depth + 1);""",
        """  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_LB; s->dval[depth] = mid + 1;
  dfs(s, depth + 1);
  if (s->stop) return;
  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_UB; s->dval[depth] = mid;
  dfs(s, depth + 1);"""),
}

PIN_FILES = ("test_oracle_pins.py", "test_oracle_search_pins.py")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    mut = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    so = tmp_path / "mutant.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so)])
    env = dict(os.environ, PCCP_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + [os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
