"""The parallel search over a shared queue of subproblems with work
donation (k_search_queue): teams hand the shallowest open right branch of
their path to waiting teams.  Donation splits the tree into disjoint
subtrees, so every count that does not depend on the incumbent's timing is
exact: count-all node, failure and solution counts, and the node and
failure counts of proof trees (objective bounded below the optimum);
optima equal the oracle's, and witnesses are valid schedules."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from synthetic import config_instance, draw_generic_model
from tests.gpu_util import oracle_model_from_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _check_schedule(inst, r):
    s = [int(v) for v in r["witness"][: inst.n]]
    assert brute.rcpsp_feasible(inst, s)
    assert max(s[i] + inst.durations[i] for i in range(inst.n)) == r["objective"]


@pytest.mark.parametrize("donate, gran", [(0, 1), (1, 1), (4, 4), (16, 2), (-1, 1)])
def test_donation_keeps_order_free_counts_exact(donate, gran):
    for seed in range(0, 100, 9):
        inst = config_instance("tiny8", seed)
        m, om = pccp.Model.from_rcpsp(inst), rcpsp_model(inst)
        opt = oracle.solve(om)["objective"]
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=opt)
        r = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, obj_ub=opt, deterministic=False,
                       donate_nodes=donate, queue_granularity=gran)
        assert (r["nodes"], r["fails"], r["solutions"]) == (c["nodes"], c["fails"], c["solutions"])
        assert r["status"] == pccp.PCCP_RES_OPTIMAL
        _check_schedule(inst, r)
        p = oracle.solve(om, obj_ub=opt - 1)
        rp = pccp.solve(m, obj_ub=opt - 1, deterministic=False, donate_nodes=donate,
                        queue_granularity=gran)
        assert rp["status"] == pccp.PCCP_RES_INFEASIBLE
        assert (rp["nodes"], rp["fails"]) == (p["nodes"], p["fails"])
        ro = pccp.solve(m, deterministic=False, donate_nodes=donate, queue_granularity=gran)
        assert ro["status"] == pccp.PCCP_RES_OPTIMAL and ro["objective"] == opt
        _check_schedule(inst, ro)


def test_generic_models_parallel_with_donation():
    for seed in range(24):
        gm = draw_generic_model(9100 + seed, n_int=5, n_bool=3, dom=7)
        m = pccp.Model.from_lists(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                                  gm.objective, gm.branch)
        om = oracle_model_from_lists(gm)
        c = oracle.solve(om, mode=oracle.COUNT_ALL)
        rc = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, deterministic=False, donate_nodes=1)
        assert (rc["nodes"], rc["fails"], rc["solutions"]) == (c["nodes"], c["fails"], c["solutions"])
        o = oracle.solve(om)
        r = pccp.solve(m, deterministic=False, donate_nodes=1)
        assert r["has_solution"] == o["has_solution"]
        if o["has_solution"]:
            assert r["objective"] == o["objective"]
            st, *_ = oracle.propagate(om, r["witness"], r["witness"])
            assert st == oracle.FIXPOINT


def test_parallel_batch_of_complete_solves():
    """All 256 models of the complete-solve family share one queue: every
    optimum equals the stored oracle optimum, every witness is an optimal
    schedule, and each model reports its own time to proof."""
    with open(os.path.join(HERE, "golden", "batch_complete_ff.json")) as f:
        g = json.load(f)
    insts = [config_instance(g["family"], m["seed"]) for m in g["models"]]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    res = pccp.solve_batch(models, strategy=pccp.PCCP_FIRST_FAIL, deterministic=False)
    for inst, r, o in zip(insts, res, g["models"]):
        assert r["status"] == pccp.PCCP_RES_OPTIMAL, inst.name
        assert r["objective"] == o["objective"], inst.name
        _check_schedule(inst, r)
        assert 0 < r["model_ms"] <= r["elapsed_ms"] * 1.001 + 0.01


def test_parallel_batch_counts_and_strategies():
    """Count-all and proof-tree counts of a parallel batch are the oracle's
    model by model, for input order, first-fail and a learned policy."""
    insts = [config_instance("tiny8", s) for s in range(30)]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    oms = [rcpsp_model(i) for i in insts]
    opts = [oracle.solve(om)["objective"] for om in oms]
    pol = pccp.Policy.random(5)
    for strat, ostrat, kw in ((pccp.PCCP_INPUT_ORDER, oracle.INPUT_ORDER, {}),
                              (pccp.PCCP_FIRST_FAIL, oracle.FIRST_FAIL, {}),
                              (pccp.PCCP_LEARNED, None, {"policy": pol})):
        # one obj_ub for the whole batch, the smallest optimum: models with a
        # larger optimum give proof trees, the others count optimal schedules
        ub = min(opts)
        res = pccp.solve_batch(models, strategy=strat, mode=pccp.PCCP_COUNT_ALL, obj_ub=ub,
                               deterministic=False, **kw)
        for inst, om, r in zip(insts, oms, res):
            if ostrat is not None:
                c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=ub, strategy=ostrat)
                assert (r["nodes"], r["fails"], r["solutions"]) == \
                    (c["nodes"], c["fails"], c["solutions"]), (inst.name, strat)
            else:  # the learned order: the solution set does not depend on the order
                c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=ub)
                assert r["solutions"] == c["solutions"]
            if r["has_solution"]:
                _check_schedule(inst, r)
        res = pccp.solve_batch(models, strategy=strat, deterministic=False, **kw)
        assert [r["objective"] for r in res] == opts


def test_parallel_batch_limits():
    models = [pccp.Model.from_rcpsp(config_instance("j30", s)) for s in range(4)]
    res = pccp.solve_batch(models, node_limit=500, deterministic=False)
    for r in res:
        assert r["status"] == pccp.PCCP_RES_LIMIT
        assert 500 <= r["nodes"] <= 500 + 64 * 1216
    res = pccp.solve_batch(models, time_limit_ms=300, deterministic=False)
    assert all(r["status"] == pccp.PCCP_RES_LIMIT for r in res)
    assert all(r["elapsed_ms"] < 3000 for r in res)


def test_reusable_batch_parallel_form_in_a_graph():
    """The parallel form queued by a reusable batch, captured in a CUDA graph
    and replayed twice (the queue is re-initialised by the graph itself):
    optima equal the stored oracle optima on every replay, and the
    sequential-order form of the same batch still gives the oracle's counts."""
    with open(os.path.join(HERE, "golden", "batch_complete_ff.json")) as f:
        g = json.load(f)
    rows = g["models"][:96]
    insts = [config_instance(g["family"], m["seed"]) for m in rows]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    b = pccp.Batch(models)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.solve_async(strategy=pccp.PCCP_FIRST_FAIL, deterministic=False)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        res = b.results()
        for inst, r, o in zip(insts, res, rows):
            assert r["status"] == pccp.PCCP_RES_OPTIMAL and r["objective"] == o["objective"]
            _check_schedule(inst, r)
    b.solve_async(strategy=pccp.PCCP_FIRST_FAIL, node_limit=200)
    for r, o in zip(b.results(), rows):
        if o["nodes"] <= 200:
            assert (r["nodes"], r["fails"], r["solutions"]) == (o["nodes"], o["fails"], o["solutions"])
