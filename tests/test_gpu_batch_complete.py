"""Batched complete solves (the uneven-batch configuration): 256 seeded
6-10-task models proved optimal in one persistent launch captured in a CUDA
graph, in the launch shape the autotuner picks; every model's optimum and
deterministic node, failure and solution counts equal the oracle's (stored
by tests/golden/make_batch_complete.py, which calls only the oracle).  Also:
every batched launch shape (teams per CTA, threads, rows per thread, tables
staged in a slot or read from global memory) gives the oracle's counts."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from paper_2207_12116_gb300 import autotune
from synthetic import config_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
STATUS = {oracle.RES_OPTIMAL: pccp.PCCP_RES_OPTIMAL, oracle.RES_INFEASIBLE: pccp.PCCP_RES_INFEASIBLE,
          oracle.RES_LIMIT: pccp.PCCP_RES_LIMIT}


def _golden():
    with open(os.path.join(HERE, "golden", "batch_complete_ff.json")) as f:
        return json.load(f)


def _check(r, o, inst):
    assert r["status"] == STATUS[o["status"]], (r, o)
    assert (r["nodes"], r["fails"], r["solutions"], r["max_depth"]) == \
        (o["nodes"], o["fails"], o["solutions"], o["max_depth"]), (inst.name, r, o)
    assert r["objective"] == o["objective"]
    s = [int(v) for v in r["witness"][: inst.n]]
    assert s == o["witness_starts"]
    assert brute.rcpsp_feasible(inst, s)
    assert max(s[i] + inst.durations[i] for i in range(inst.n)) == r["objective"]


def test_complete_batch_in_a_captured_graph_matches_the_oracle():
    g = _golden()
    insts = [config_instance(g["family"], m["seed"]) for m in g["models"]]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    (teams, threads), report = autotune.tune_search_shape(models, node_limit=400)
    assert report[(teams, threads)] == max(v for v in report.values() if v)
    b = pccp.Batch(models, threads=threads, teams_per_cta=teams)
    assert b.shape[:2] == (threads, teams)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.solve_async(strategy=pccp.PCCP_FIRST_FAIL)
    graph.replay()
    torch.cuda.synchronize()
    res = b.results()
    for inst, r, o in zip(insts, res, g["models"]):
        _check(r, o, inst)
        assert 0 < r["model_ms"]


def _same_as_oracle(insts, lim, shapes):
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    ref = [oracle.solve(rcpsp_model(i), strategy=oracle.FIRST_FAIL, node_limit=lim)
           for i in insts]
    for kw in shapes:
        res = pccp.solve_batch(models, strategy=pccp.PCCP_FIRST_FAIL, node_limit=lim, **kw)
        for inst, r, o in zip(insts, res, ref):
            assert r["status"] == STATUS[o["status"]], (kw, inst.name)
            assert (r["nodes"], r["fails"], r["solutions"], r["max_depth"]) == \
                (o["nodes"], o["fails"], o["solutions"], o["max_depth"]), (kw, inst.name, r, o)
            if o["has_solution"]:
                assert r["objective"] == o["objective"]
                assert np.array_equal(r["witness"], o["witness"])
    return models


def test_slot_shapes_and_table_placements_agree_with_the_oracle():
    """8-task and 30-60-task models in one launch: with several teams per CTA
    the larger tables do not fit a slot beside their stores and are read from
    global memory while the others are staged; counts are the oracle's under
    the same node limit, whatever the shape."""
    insts = [config_instance("tiny8", s) for s in range(10)] + \
            [config_instance("mixed30_60", s) for s in range(6)]
    _same_as_oracle(insts, 60, [
        dict(), dict(teams_per_cta=1, threads=1024), dict(teams_per_cta=2),
        dict(teams_per_cta=3, threads=256), dict(teams_per_cta=4, threads=128),
        dict(teams_per_cta=6, threads=64), dict(teams_per_cta=2, props_per_thread=8),
        dict(teams_per_cta=4, skip_stable=True), dict(teams_per_cta=3, skip_stable=False)])


def test_many_small_slots_and_a_large_model_alone():
    """Up to 15 one-warp teams per CTA on 8-task models; a 120-task model:
    with interval stores (116 KB, half the shared memory) with one team per
    CTA, and refused with several; with its Booleans as bits (a 4.6 KB store)
    in four teams per CTA."""
    _same_as_oracle([config_instance("tiny8", s) for s in range(40)], 300, [
        dict(teams_per_cta=8, threads=64), dict(teams_per_cta=12, threads=32),
        dict(teams_per_cta=15, threads=32)])
    _same_as_oracle([config_instance("j120", 0), config_instance("tiny8", 3)], 10, [
        dict(), dict(teams_per_cta=1, threads=512)])
    bits = [pccp.Model.from_rcpsp(config_instance("j120", 0), bool_store=1),
            pccp.Model.from_rcpsp(config_instance("tiny8", 3))]
    rb = pccp.solve_batch(bits, strategy=pccp.PCCP_FIRST_FAIL, node_limit=10, teams_per_cta=4,
                          threads=256)
    ob = oracle.solve(rcpsp_model(config_instance("j120", 0)), strategy=oracle.FIRST_FAIL,
                      node_limit=10)
    assert (rb[0]["nodes"], rb[0]["fails"]) == (ob["nodes"], ob["fails"])
    big = [pccp.Model.from_rcpsp(config_instance("j120", 0), bool_store=-1),
           pccp.Model.from_rcpsp(config_instance("tiny8", 3))]
    r = pccp.solve_batch(big, strategy=pccp.PCCP_FIRST_FAIL, node_limit=10, teams_per_cta=1)
    o = oracle.solve(rcpsp_model(config_instance("j120", 0)), strategy=oracle.FIRST_FAIL,
                     node_limit=10)
    assert (r[0]["nodes"], r[0]["fails"]) == (o["nodes"], o["fails"])
    with pytest.raises(pccp.PccpError) as e:
        pccp.solve_batch(big, node_limit=5, teams_per_cta=4)
    assert e.value.code == pccp.PCCP_ERR_SMEM


def test_batch_shape_is_reported_and_bounded():
    models = [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(5)]
    b = pccp.Batch(models, threads=64, teams_per_cta=6)
    threads, teams, ctas = b.shape
    # one CTA per model while SMs are free: models spread before teams share an SM
    assert (threads, teams) == (64, 6) and ctas == 5
    with pytest.raises(pccp.PccpError):
        pccp.Batch(models, threads=128, teams_per_cta=16)
