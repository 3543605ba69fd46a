"""120-task models (14,521 variables, 14,280 reified rows, ~570 KB table):
the table does not fit shared memory, so every kernel reads it from the
device image while the store stays in shared memory.  Results must still be
the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model, node_store
import paper_2207_12116_gb300 as pccp
from synthetic import config_instance, draw_partial_assignments
from tests.gpu_util import compare_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_j120_table_exceeds_shared_memory():
    m = pccp.Model.from_rcpsp(config_instance("j120", 0))
    assert m.info.table_bytes > 232448  # larger than one CTA's shared memory


def test_j120_propagation_bit_exact():
    inst = config_instance("j120", 0)
    rows = pccp.rcpsp.build_rows(inst)
    m = pccp.Model.from_rows(rows)
    om = rcpsp_model(inst)
    nodes = [[]] + draw_partial_assignments(inst.n, inst.horizon, 11, seed=21)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    dlb, dub = torch.from_numpy(lb).cuda(), torch.from_numpy(ub).cuda()
    st, it = pccp.propagate(m, dlb, dub)
    torch.cuda.synchronize()
    x, f = compare_batch(om, lb, ub, st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy())
    assert x >= 5


def test_j120_search_matches_oracle_node_limited():
    inst = config_instance("j120", 1)
    r = pccp.solve_batch([pccp.Model.from_rcpsp(inst)], node_limit=12)[0]
    o = oracle.solve(rcpsp_model(inst), node_limit=12)
    assert (r["nodes"], r["fails"], r["solutions"], r["status"]) == \
        (o["nodes"], o["fails"], o["solutions"], pccp.PCCP_RES_LIMIT)


def test_j120_parallel_search_finds_valid_schedules():
    inst = config_instance("j120", 2)
    r = pccp.solve(pccp.Model.from_rcpsp(inst), deterministic=False, time_limit_ms=4000)
    assert r["nodes"] > 1000
    if r["has_solution"]:
        n = inst.n
        s = [int(v) for v in r["witness"][:n]]
        assert brute.rcpsp_feasible(inst, s)
        assert max(s[i] + inst.durations[i] for i in range(n)) == r["objective"]
