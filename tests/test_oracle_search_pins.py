"""Pins for the oracle's search order (which variable, which split point,
which child first), each compared with something other than the oracle.

The paper leaves the branching rule open (Sec. 5 runs propagate-and-branch
with full recomputation); the readings pinned here are: input order = the
lowest-index unfixed branch variable; first-fail = the smallest ub - lb,
ties to the lower index; split [l, u] at m = l + (u - l) / 2 (floor), left
child ub <= m explored first, right child lb >= m + 1; a node is every store
propagated; after a solution of objective z every later node is told
ub(obj) <= z - 1.

1. Hand-derived traces (tests/golden/search_traces.json, written by
   tests/golden/make_search_traces.py from the oracle) must equal the traces
   below, each worked out by hand from the rule above; the oracle must
   reproduce the stored file.
2. On brute-forced tiny schedules, input-order depth-first search visits
   leaves in lexicographic order of the start vector, so its first solution
   is the lexicographically smallest feasible start vector, and branch and
   bound ends on the lexicographically smallest optimal one.  Both come from
   enumeration alone.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model
from synthetic.rcpsp import RcpspDistribution, draw_rcpsp

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "search_traces.json")

F, S, B = oracle.NODE_FAILED, oracle.NODE_SOLUTION, oracle.NODE_BRANCH
ROOT = (0, -1, -1, 0)

# Records: (depth, decision var, side, value, outcome, chosen var); side 0 is
# the left child (ub <= value), 1 the right child (lb >= value).
HAND = {
    # x0, x1 in [0, 1], no rows, count all, first-fail.  Both widths are 1 at
    # the root: the tie goes to x0, m = 0.  Under x0 <= 0 only x1 is open
    # (m = 0), giving (0,0), (0,1); then x0 >= 1 and (1,0), (1,1).
    "first_fail_ties_to_lower_index": dict(nodes=7, fails=0, solutions=4, witness=[0, 0], trace=[
        ROOT + (B, 0), (1, 0, 0, 0, B, 1), (2, 1, 0, 0, S, -1), (2, 1, 1, 1, S, -1),
        (1, 0, 1, 1, B, 1), (2, 1, 0, 0, S, -1), (2, 1, 1, 1, S, -1)]),
    # x0 in [1, 6], count all.  m = 1 + 5/2 = 3; [1,3]: m = 2; [1,2]: m = 1
    # -> 1, 2; then 3; [4,6]: m = 5; [4,5]: m = 4 -> 4, 5; then 6.
    "split_point_odd_width": dict(nodes=11, fails=0, solutions=6, witness=[1], trace=[
        ROOT + (B, 0), (1, 0, 0, 3, B, 0), (2, 0, 0, 2, B, 0), (3, 0, 0, 1, S, -1),
        (3, 0, 1, 2, S, -1), (2, 0, 1, 3, S, -1), (1, 0, 1, 4, B, 0), (2, 0, 0, 5, B, 0),
        (3, 0, 0, 4, S, -1), (3, 0, 1, 5, S, -1), (2, 0, 1, 6, S, -1)]),
    # x0 in [0, 3], M = x1 in [0, 10], x0 + 2 <= M, minimise M, branch on x0.
    # Root: M in [2, 10]; m = 1.  [0,1]: m = 0.  x0 = 0: solution, M = 2.
    # Later nodes get ub(M) <= 1 while lb(M) >= lb(x0) + 2 >= 3: x0 = 1
    # fails, and so does the root's right child x0 >= 2.
    "incumbent_bound_prunes": dict(nodes=5, fails=2, solutions=1, witness=[0, 2], trace=[
        ROOT + (B, 0), (1, 0, 0, 1, B, 0), (2, 0, 0, 0, S, -1), (2, 0, 1, 1, F, -1),
        (1, 0, 1, 2, F, -1)]),
    # x0 in [0, 6], x1 in [4, 9], x0 + 3 <= x1, first solution, first-fail.
    # Root: widths 6 and 5 -> x1, m = 6.  x1 in [4,6] makes ub(x0) = 3:
    # widths 3, 2 -> x1, m = 5.  x1 in [4,5], ub(x0) = 2: widths 2, 1 -> x1,
    # m = 4.  x1 = 4, x0 in [0,1] -> x0, m = 0: x0 = 0 is the solution.
    "first_fail_after_propagation": dict(nodes=5, fails=0, solutions=1, witness=[0, 4], trace=[
        ROOT + (B, 1), (1, 1, 0, 6, B, 1), (2, 1, 0, 5, B, 1), (3, 1, 0, 4, B, 0),
        (4, 0, 0, 0, S, -1)]),
    # x0, x1 in [0, 3], x0 + x1 <= 3, count all, first-fail.  Root tie -> x0,
    # m = 1; [0,1] (width 1 < 3) -> x0, m = 0; x0 = 0: x1 in [0,3], m = 1,
    # then [0,1] m = 0 and [2,3] m = 2: (0,0) (0,1) (0,2) (0,3).  x0 = 1:
    # x1 <= 2, m = 1: [0,1] m = 0 -> (1,0) (1,1); x1 = 2.  Root right child
    # x0 in [2,3] makes x1 <= 1: tie of widths 1 -> x0, m = 2; x0 = 2: x1
    # m = 0 -> (2,0) (2,1); x0 = 3 fixes x1 = 0.  10 solutions (the pairs
    # with x0 + x1 <= 3).
    "linear_row_first_fail_count": dict(nodes=19, fails=0, solutions=10, witness=[0, 0], trace=[
        ROOT + (B, 0), (1, 0, 0, 1, B, 0), (2, 0, 0, 0, B, 1), (3, 1, 0, 1, B, 1),
        (4, 1, 0, 0, S, -1), (4, 1, 1, 1, S, -1), (3, 1, 1, 2, B, 1), (4, 1, 0, 2, S, -1),
        (4, 1, 1, 3, S, -1), (2, 0, 1, 1, B, 1), (3, 1, 0, 1, B, 1), (4, 1, 0, 0, S, -1),
        (4, 1, 1, 1, S, -1), (3, 1, 1, 2, S, -1), (1, 0, 1, 2, B, 0), (2, 0, 0, 2, B, 1),
        (3, 1, 0, 0, S, -1), (3, 1, 1, 1, S, -1), (2, 0, 1, 3, S, -1)]),
    # x0, x1 in [0, 2], b = x2 fixed to 0, b <=> (x0 <= x1 and x1 < x0 + 1),
    # i.e. x0 != x1; count all, input order.  x0 = 0 entails x0 <= x1, so
    # not(x1 < x0 + 1): x1 >= 1, m = 1 -> (0,1) (0,2).  x0 = 1: x1 in [0,2],
    # m = 1; x1 <= 1 entails x1 <= x0, so not(x0 <= x1): x1 <= 0, a solution
    # at once; x1 = 2.  x0 = 2 entails x1 <= x0, so x1 <= 1, m = 0 -> (2,0)
    # (2,1).  6 solutions.
    "reified_not_equal_count": dict(nodes=11, fails=0, solutions=6, witness=[0, 1, 0], trace=[
        ROOT + (B, 0), (1, 0, 0, 1, B, 0), (2, 0, 0, 0, B, 1), (3, 1, 0, 1, S, -1),
        (3, 1, 1, 2, S, -1), (2, 0, 1, 1, B, 1), (3, 1, 0, 1, S, -1), (3, 1, 1, 2, S, -1),
        (1, 0, 1, 2, B, 1), (2, 1, 0, 0, S, -1), (2, 1, 1, 1, S, -1)]),
}


def _load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _model(spec):
    m = spec["model"]
    return oracle.Model(m["lb0"], m["ub0"], [tuple(t) for t in m["temporal"]],
                        [(c, [tuple(t) for t in terms]) for c, terms in m["linear"]],
                        [tuple(r) for r in m["reified"]], m["objective"], m["branch"])


def test_every_hand_case_is_stored():
    assert sorted(_load_golden()) == sorted(HAND)


@pytest.mark.parametrize("name", sorted(HAND))
def test_stored_trace_matches_hand_derivation(name):
    stored = _load_golden()[name]["result"]
    hand = HAND[name]
    assert [tuple(t) for t in stored["trace"]] == hand["trace"]
    assert (stored["nodes"], stored["fails"], stored["solutions"]) == \
        (hand["nodes"], hand["fails"], hand["solutions"])
    assert stored["witness"] == hand["witness"]
    # a node is every store propagated: the trace has one record per node
    assert len(hand["trace"]) == hand["nodes"]


@pytest.mark.parametrize("name", sorted(HAND))
def test_oracle_reproduces_hand_trace(name):
    spec = _load_golden()[name]
    r = oracle.solve(_model(spec), mode=spec["mode"], strategy=spec["strategy"], trace_cap=1000)
    hand = HAND[name]
    assert r["trace"] == hand["trace"]
    assert (r["nodes"], r["fails"], r["solutions"]) == (hand["nodes"], hand["fails"],
                                                        hand["solutions"])
    assert [int(x) for x in r["witness"]] == hand["witness"]


def _lexmin(rows):
    rows = np.asarray(rows)
    order = np.lexsort(rows.T[::-1])
    return [int(x) for x in rows[order[0]]]


TINY = RcpspDistribution(3, 5, 2, (1, 3), (0, 2), (2, 3), 0.25)


@pytest.mark.parametrize("seed", range(40))
def test_input_order_first_solution_is_lexicographic_minimum(seed):
    """Input order with left children first enumerates leaves in
    lexicographic order of the start vector, whatever the split points, so
    in count-all mode (objective bounded by the optimum K) the first
    solution recorded is the lexicographically smallest start vector with
    makespan <= K among the brute-force enumeration."""
    inst = draw_rcpsp(TINY, 5000 + seed)
    om = rcpsp_model(inst)
    opt = oracle.solve(om)["objective"]
    sols = brute.rcpsp_enumerate(inst, opt)
    assert len(sols) > 0
    c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=opt)
    assert [int(x) for x in c["witness"][: inst.n]] == _lexmin(sols)


@pytest.mark.parametrize("seed", range(40))
def test_branch_and_bound_ends_on_lexicographic_minimum_optimum(seed):
    """Branch and bound in input order records a solution only when it
    improves; the optimal leaf that comes first in lexicographic order is
    never pruned (the bound is still above the optimum when it is reached),
    and nothing after it improves, so the witness is the lexicographically
    smallest optimal start vector of the enumeration."""
    inst = draw_rcpsp(TINY, 6000 + seed)
    om = rcpsp_model(inst)
    r = oracle.solve(om)
    all_sols = brute.rcpsp_enumerate(inst, inst.horizon)
    d = np.asarray(inst.durations)
    mk = (all_sols + d[None, :]).max(axis=1)
    assert r["objective"] == int(mk.min())
    assert [int(x) for x in r["witness"][: inst.n]] == _lexmin(all_sols[mk == mk.min()])


@pytest.mark.parametrize("seed", range(20))
def test_first_fail_finds_the_same_optimum_and_solution_set(seed):
    """Reordering the tree changes node counts but not the optimum or the
    number of optimal schedules."""
    inst = draw_rcpsp(TINY, 7000 + seed)
    om = rcpsp_model(inst)
    a = oracle.solve(om)
    b = oracle.solve(om, strategy=oracle.FIRST_FAIL)
    assert a["objective"] == b["objective"]
    ca = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=a["objective"])
    cb = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=a["objective"], strategy=oracle.FIRST_FAIL)
    assert ca["solutions"] == cb["solutions"] == len(brute.rcpsp_enumerate(inst, a["objective"]))
