"""Batched search and propagation captured in CUDA graphs and replayed, and
the autotuner's choices, all checked against eager results and the oracle."""
import numpy as np
import pytest

import oracle
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from paper_2207_12116_gb300 import autotune
from synthetic import config_instance, draw_partial_assignments
from tests.gpu_util import compare_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DET = ("status", "has_solution", "objective", "nodes", "fails", "solutions", "max_depth")


def _same(a, b):
    for k in DET:
        assert a[k] == b[k], (k, a[k], b[k])
    if a["has_solution"]:
        assert np.array_equal(a["witness"], b["witness"])


def test_batched_search_graph_replay():
    models = [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(24)] + \
             [pccp.Model.from_rcpsp(config_instance("mixed30_60", s)) for s in range(8)]
    ref = pccp.solve_batch(models, node_limit=300)
    b = pccp.Batch(models, threads=128)
    b.solve_async(node_limit=300)  # eager once
    for x, y in zip(ref, b.results()):
        _same(x, y)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.solve_async(node_limit=300)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for x, y in zip(ref, b.results()):
            _same(x, y)
    # and the eager results are the oracle's under the same node limit
    for i in range(24):
        o = oracle.solve(rcpsp_model(config_instance("tiny8", i)), node_limit=300)
        assert (ref[i]["objective"], ref[i]["nodes"], ref[i]["fails"]) == \
            (o["objective"], o["nodes"], o["fails"])


def test_propagation_graph_replay():
    inst = config_instance("j30", 0)
    rows = pccp.rcpsp.build_rows(inst)
    m = pccp.Model.from_rows(rows)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 2000, seed=5)
    lb_h, ub_h = pccp.rcpsp.node_stores(rows, nodes)
    src_lb = torch.from_numpy(lb_h).cuda()
    src_ub = torch.from_numpy(ub_h).cuda()
    lb, ub = src_lb.clone(), src_ub.clone()
    st = torch.empty(len(nodes), dtype=torch.int32, device="cuda")
    it = torch.empty_like(st)
    pccp.propagate(m, lb, ub, st, it)
    torch.cuda.synchronize()
    eager = (st.cpu().numpy().copy(), lb.cpu().numpy().copy(), ub.cpu().numpy().copy())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lb.copy_(src_lb)
        ub.copy_(src_ub)
        pccp.propagate(m, lb, ub, st, it)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        s2 = st.cpu().numpy()
        assert np.array_equal(s2, eager[0])
        ok = s2 == 0
        assert np.array_equal(lb.cpu().numpy()[ok], eager[1][ok])
        assert np.array_equal(ub.cpu().numpy()[ok], eager[2][ok])


def test_autotuned_propagation_is_exact():
    inst = config_instance("j30", 1)
    rows = pccp.rcpsp.build_rows(inst)
    m = pccp.Model.from_rows(rows)
    om = rcpsp_model(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 3000, seed=9)
    lb_h, ub_h = pccp.rcpsp.node_stores(rows, nodes)
    lb, ub = torch.from_numpy(lb_h).cuda(), torch.from_numpy(ub_h).cuda()
    cfg, report = autotune.tune_propagate(m, lb, ub, trials=2)
    assert (cfg.team_threads, cfg.teams_per_cta) in report
    assert report[(cfg.team_threads, cfg.teams_per_cta)] == min(v for v in report.values() if v)
    st, _ = pccp.propagate(m, lb, ub, config=cfg)
    torch.cuda.synchronize()
    compare_batch(om, lb_h, ub_h, st.cpu().numpy(), lb.cpu().numpy(), ub.cpu().numpy(),
                  rows=range(0, 3000, 10))


def test_autotuned_search_threads():
    models = [pccp.Model.from_rcpsp(config_instance("mixed30_60", s)) for s in range(16)]
    threads, report = autotune.tune_search_threads(models, node_limit=100)
    assert threads in report and report[threads] == max(v for v in report.values() if v)
    res = pccp.solve_batch(models, node_limit=100, threads=threads)
    for inst_seed, r in zip(range(16), res):
        o = oracle.solve(rcpsp_model(config_instance("mixed30_60", inst_seed)), node_limit=100)
        assert (r["nodes"], r["fails"], r["solutions"]) == (o["nodes"], o["fails"], o["solutions"])
