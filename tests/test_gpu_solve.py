"""GPU parity of pccp_solve / pccp_solve_batch with the oracle's depth-first
branch and bound: in the deterministic order the optimum, the witness and
the node, failure and solution counts are equal."""
import numpy as np
import pytest

import oracle
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from synthetic import config_instance, draw_generic_model
from tests.gpu_util import oracle_model_from_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATUS = {oracle.RES_OPTIMAL: pccp.PCCP_RES_OPTIMAL, oracle.RES_INFEASIBLE: pccp.PCCP_RES_INFEASIBLE,
          oracle.RES_LIMIT: pccp.PCCP_RES_LIMIT}


def same(r, o):
    assert r["status"] == STATUS[o["status"]], (r, o)
    assert (r["nodes"], r["fails"], r["solutions"]) == (o["nodes"], o["fails"], o["solutions"]), (r, o)
    assert r["has_solution"] == o["has_solution"]
    if o["has_solution"]:
        assert r["objective"] == o["objective"]
        assert np.array_equal(r["witness"], o["witness"])
    assert r["max_depth"] == o["max_depth"]


def test_tiny8_single_solves():
    # the library keeps these models in its own variable order: witnesses must
    # still come back in the caller's
    assert pccp.Model.from_rcpsp(config_instance("tiny8", 0)).info.reordered == 1
    for seed in range(0, 100, 5):
        inst = config_instance("tiny8", seed)
        same(pccp.solve(pccp.Model.from_rcpsp(inst)), oracle.solve(rcpsp_model(inst)))


def test_tiny8_batch_one_launch():
    insts = [config_instance("tiny8", s) for s in range(100)]
    res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts])
    for inst, r in zip(insts, res):
        same(r, oracle.solve(rcpsp_model(inst)))


@pytest.mark.parametrize("threads", [32, 128, 1024])
def test_tiny8_first_fail_and_team_sizes(threads):
    for seed in range(0, 100, 9):
        inst = config_instance("tiny8", seed)
        r = pccp.solve(pccp.Model.from_rcpsp(inst), strategy=pccp.PCCP_FIRST_FAIL, threads=threads)
        same(r, oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL))


def test_tiny8_count_all_under_optimum():
    for seed in range(0, 100, 10):
        inst = config_instance("tiny8", seed)
        o = oracle.solve(rcpsp_model(inst))
        c = oracle.solve(rcpsp_model(inst), mode=oracle.COUNT_ALL, obj_ub=o["objective"])
        r = pccp.solve(pccp.Model.from_rcpsp(inst), mode=pccp.PCCP_COUNT_ALL, obj_ub=o["objective"])
        same(r, c)
        assert r["solutions"] >= 1


def test_node_limited_j30_and_mixed_batch():
    insts = [config_instance("j30", s) for s in range(4)] + \
            [config_instance("mixed30_60", s) for s in range(12)]
    res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts], node_limit=400)
    for inst, r in zip(insts, res):
        o = oracle.solve(rcpsp_model(inst), node_limit=400)
        same(r, o)


def test_generic_models_search():
    for seed in range(40):
        gm = draw_generic_model(9000 + seed, n_int=4, n_bool=3, dom=6)
        m = pccp.Model.from_lists(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                                  gm.objective, gm.branch)
        om = oracle_model_from_lists(gm)
        same(pccp.solve(m), oracle.solve(om))
        same(pccp.solve(m, mode=pccp.PCCP_COUNT_ALL), oracle.solve(om, mode=oracle.COUNT_ALL))


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_lane_groups_for_linear_rows_are_exact(threads):
    """In the depth-first searches over tables in shared memory, short linear
    rows are summed by groups of 2, 4 or 8 lanes when the team has that many
    lanes per row and the longest row at least 6 terms per lane (30-32-task
    models: groups of 2 at 256 threads; 30-60-task models: 4 at 1024 threads;
    generic models with a few rows of up to 64 terms: 8 at 1024 threads).
    Node, failure and solution counts, optima and witnesses stay the
    oracle's."""
    insts = [config_instance("mixed30_60", s) for s in (0, 2, 3, 6, 14, 35)]
    assert sorted({i.n for i in insts}) == [32, 47, 59, 60]
    for strat, ostrat in ((pccp.PCCP_INPUT_ORDER, oracle.INPUT_ORDER),
                          (pccp.PCCP_FIRST_FAIL, oracle.FIRST_FAIL)):
        res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts], node_limit=250,
                               threads=threads, teams_per_cta=1, strategy=strat)
        for inst, r in zip(insts, res):
            same(r, oracle.solve(rcpsp_model(inst), node_limit=250, strategy=ostrat))
    long_rows = 0
    for seed in range(12):
        gm = draw_generic_model(7700 + seed, n_int=8, n_bool=56, dom=10, n_temporal=6,
                                n_linear=4, n_reified=10, max_len=64, coef=6)
        lens = [sum(1 for a, _ in row[1] if a != 0) for row in gm.linear]
        long_rows += max(lens) >= 48
        m = pccp.Model.from_lists(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                                  gm.objective, gm.branch)
        om = oracle_model_from_lists(gm)
        same(pccp.solve(m, threads=threads, node_limit=300), oracle.solve(om, node_limit=300))
    assert long_rows >= 4


# ------------------------------------------- parallel search (EPS subproblems)

from oracle import brute  # noqa: E402


def _check_rcpsp_witness(inst, r):
    n = inst.n
    s = [int(v) for v in r["witness"][:n]]
    assert brute.rcpsp_feasible(inst, s)
    mk = max(s[i] + inst.durations[i] for i in range(n))
    assert mk == r["objective"] == int(r["witness"][n + n * n])


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_parallel_tiny8_optima(threads):
    for seed in range(0, 100, 7):
        inst = config_instance("tiny8", seed)
        r = pccp.solve(pccp.Model.from_rcpsp(inst), deterministic=False, threads=threads)
        o = oracle.solve(rcpsp_model(inst))
        assert r["status"] == pccp.PCCP_RES_OPTIMAL and r["objective"] == o["objective"]
        _check_rcpsp_witness(inst, r)


def test_parallel_count_all_and_proof_trees_are_exact():
    """Without an incumbent the tree is fixed, so node, failure and solution
    counts do not depend on how it is split among teams."""
    for seed in range(0, 100, 11):
        inst = config_instance("tiny8", seed)
        m, om = pccp.Model.from_rcpsp(inst), rcpsp_model(inst)
        opt = oracle.solve(om)["objective"]
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=opt)
        r = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, obj_ub=opt, deterministic=False)
        assert (r["nodes"], r["fails"], r["solutions"]) == (c["nodes"], c["fails"], c["solutions"])
        assert r["status"] == pccp.PCCP_RES_OPTIMAL
        _check_rcpsp_witness(inst, r)
        p = oracle.solve(om, obj_ub=opt - 1)
        rp = pccp.solve(m, obj_ub=opt - 1, deterministic=False)
        assert p["status"] == oracle.RES_INFEASIBLE and rp["status"] == pccp.PCCP_RES_INFEASIBLE
        assert (rp["nodes"], rp["fails"]) == (p["nodes"], p["fails"])


def test_parallel_generic_models():
    for seed in range(30):
        gm = draw_generic_model(9000 + seed, n_int=4, n_bool=3, dom=6)
        m = pccp.Model.from_lists(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                                  gm.objective, gm.branch)
        om = oracle_model_from_lists(gm)
        o = oracle.solve(om)
        r = pccp.solve(m, deterministic=False)
        assert r["status"] == STATUS[o["status"]] and r["objective"] == o["objective"]
        if o["has_solution"]:  # the witness, as a fixed store, is stable under propagation
            w = r["witness"]
            st, flb, fub, _ = oracle.propagate(om, w, w)
            assert st == oracle.FIXPOINT
        c = oracle.solve(om, mode=oracle.COUNT_ALL)
        rc = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, deterministic=False)
        assert (rc["nodes"], rc["solutions"]) == (c["nodes"], c["solutions"])


def test_parallel_node_limited_j30():
    """A budget of ~1,600 nodes per team lets depth-first dives (about 8
    decisions per task) reach leaves; the limit is checked in batches of 64
    nodes per team, so the count may exceed it by that much per team."""
    inst = config_instance("j30", 0)
    r = pccp.solve(pccp.Model.from_rcpsp(inst), deterministic=False, node_limit=2_000_000,
                   time_limit_ms=20_000)
    assert r["status"] in (pccp.PCCP_RES_LIMIT, pccp.PCCP_RES_OPTIMAL)
    assert r["nodes"] >= 100_000 and r["has_solution"]
    _check_rcpsp_witness(inst, r)
    d = oracle.solve(rcpsp_model(inst), node_limit=2_000)  # the parallel search does better
    if d["has_solution"]:
        assert r["objective"] <= d["objective"]



# ------------------------------- skipping stable rows keeps every result exact

def test_skip_stable_search_is_exact():
    for seed in range(0, 100, 6):
        inst = config_instance("tiny8", seed)
        m, om = pccp.Model.from_rcpsp(inst), rcpsp_model(inst)
        same(pccp.solve(m, skip_stable=True), oracle.solve(om))
        same(pccp.solve(m, strategy=pccp.PCCP_FIRST_FAIL, skip_stable=True),
             oracle.solve(om, strategy=oracle.FIRST_FAIL))
    insts = [config_instance("mixed30_60", s) for s in range(8)]
    res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts], node_limit=300,
                           skip_stable=True)
    for inst, r in zip(insts, res):
        same(r, oracle.solve(rcpsp_model(inst), node_limit=300))


def test_skip_stable_parallel_counts_are_exact():
    for seed in range(0, 100, 13):
        inst = config_instance("tiny8", seed)
        m, om = pccp.Model.from_rcpsp(inst), rcpsp_model(inst)
        opt = oracle.solve(om)["objective"]
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=opt)
        r = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, obj_ub=opt, deterministic=False,
                       skip_stable=True)
        assert (r["nodes"], r["fails"], r["solutions"]) == (c["nodes"], c["fails"], c["solutions"])
        r2 = pccp.solve(m, deterministic=False, skip_stable=True)
        assert r2["objective"] == opt
        _check_rcpsp_witness(inst, r2)
