"""Writes search_traces.json: the oracle's depth-first search traces of a
few models small enough to follow by hand.  Calls only the oracle.

Each case is a model (plain rows), the search options and the trace the
oracle returns: one record per node in depth-first preorder,
(depth, decision variable, side, value, outcome, chosen variable) with side
0 = left child (ub <= value), 1 = right child (lb >= value), outcome
0 failed / 1 solution / 2 branching, and the variable a branching node
splits.  tests/test_oracle_search_pins.py checks every stored trace against
the one derived by hand from the search rule (split [l, u] at
m = l + (u - l) / 2, left child first; input order: lowest-index unfixed
branch variable; first-fail: smallest ub - lb, ties to the lower index;
Sec. 5 of the paper for the propagate-and-branch loop, whose rule it leaves
open) and the oracle against the stored traces.

    python tests/golden/make_search_traces.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

# name: (lb0, ub0, temporal, linear, reified, objective, branch, mode, strategy)
CASES = {
    "first_fail_ties_to_lower_index": (
        [0, 0], [1, 1], [], [], [], -1, [0, 1], oracle.COUNT_ALL, oracle.FIRST_FAIL),
    "split_point_odd_width": (
        [1], [6], [], [], [], -1, [0], oracle.COUNT_ALL, oracle.INPUT_ORDER),
    "incumbent_bound_prunes": (
        [0, 0], [3, 10], [(0, 1, 2)], [], [], 1, [0], oracle.OPTIMISE, oracle.INPUT_ORDER),
    "first_fail_after_propagation": (
        [0, 4], [6, 9], [(0, 1, 3)], [], [], -1, [0, 1], oracle.OPTIMISE, oracle.FIRST_FAIL),
    "linear_row_first_fail_count": (
        [0, 0], [3, 3], [], [(3, [(1, 0), (1, 1)])], [], -1, [0, 1], oracle.COUNT_ALL,
        oracle.FIRST_FAIL),
    "reified_not_equal_count": (
        [0, 0, 0], [2, 2, 0], [], [], [(2, 0, 1, 1)], -1, [0, 1], oracle.COUNT_ALL,
        oracle.INPUT_ORDER),
}


def run_case(case):
    lb0, ub0, temporal, linear, reified, objective, branch, mode, strategy = case
    m = oracle.Model(lb0, ub0, temporal, linear, reified, objective, branch)
    r = oracle.solve(m, mode=mode, strategy=strategy, trace_cap=1000)
    return {"nodes": r["nodes"], "fails": r["fails"], "solutions": r["solutions"],
            "objective": r["objective"],
            "witness": None if r["witness"] is None else [int(x) for x in r["witness"]],
            "trace": [list(t) for t in r["trace"]]}


def main():
    oracle.build()
    out = {"about": "oracle depth-first search traces; see make_search_traces.py",
           "fields": ["depth", "decision_var", "side", "value", "outcome", "chosen_var"],
           "cases": {}}
    for name, case in CASES.items():
        lb0, ub0, temporal, linear, reified, objective, branch, mode, strategy = case
        out["cases"][name] = {
            "model": {"lb0": lb0, "ub0": ub0, "temporal": temporal, "linear": linear,
                      "reified": reified, "objective": objective, "branch": branch},
            "mode": mode, "strategy": strategy, "result": run_case(case)}
    with open(os.path.join(HERE, "search_traces.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
