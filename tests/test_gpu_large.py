"""120-task models (14,521 variables, 14,280 reified rows, ~570 KB table):
the table does not fit shared memory, so every kernel reads it from the
device image while the store stays in shared memory.  Results must still be
the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from synthetic import config_instance, draw_partial_assignments
from tests.gpu_util import compare_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_j120_table_exceeds_shared_memory():
    m = pccp.Model.from_rcpsp(config_instance("j120", 0))
    assert m.info.table_bytes > 232448  # larger than one CTA's shared memory


@pytest.mark.parametrize("stream_table, skip_stable", [(True, None), (False, None),
                                                       (False, False), (True, False)])
def test_j120_propagation_bit_exact(stream_table, skip_stable):
    """Tables in global memory: read in place or streamed, with stable rows
    skipped (the default there) or every row every iteration."""
    inst = config_instance("j120", 0)
    rows = pccp.rcpsp.build_rows(inst)
    m = pccp.Model.from_rows(rows)
    assert m.info.n_segments > 10
    assert m.info.reordered == 1  # pair-block order: far fewer bank conflicts here
    om = rcpsp_model(inst)
    nodes = [[]] + draw_partial_assignments(inst.n, inst.horizon, 11, seed=21)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    dlb, dub = torch.from_numpy(lb).cuda(), torch.from_numpy(ub).cuda()
    cfg = pccp.launch_config(stream_table=stream_table, skip_stable=skip_stable)
    st, it = pccp.propagate(m, dlb, dub, config=cfg)
    torch.cuda.synchronize()
    x, f = compare_batch(om, lb, ub, st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy())
    assert x >= 5


@pytest.mark.parametrize("stream_table, skip_stable", [(True, None), (False, None),
                                                       (False, False)])
def test_j120_search_matches_oracle_node_limited(stream_table, skip_stable):
    inst = config_instance("j120", 1)
    r = pccp.solve_batch([pccp.Model.from_rcpsp(inst)], node_limit=12,
                         stream_table=stream_table, skip_stable=skip_stable)[0]
    o = oracle.solve(rcpsp_model(inst), node_limit=12)
    assert (r["nodes"], r["fails"], r["solutions"], r["status"]) == \
        (o["nodes"], o["fails"], o["solutions"], pccp.PCCP_RES_LIMIT)


def test_j120_batch_switches_streams_between_models():
    """One CTA searches several 120-task models in turn: each model's stream
    is closed and the next one opened on the same buffers."""
    insts = [config_instance("j120", s) for s in (3, 4, 5)]
    res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts], node_limit=6, blocks=1,
                           stream_table=True)
    for inst, r in zip(insts, res):
        o = oracle.solve(rcpsp_model(inst), node_limit=6)
        assert (r["nodes"], r["fails"], r["solutions"]) == (o["nodes"], o["fails"], o["solutions"])


@pytest.mark.parametrize("stream_table", [True, False])
def test_j120_parallel_search_finds_valid_schedules(stream_table):
    inst = config_instance("j120", 2)
    r = pccp.solve(pccp.Model.from_rcpsp(inst), deterministic=False, time_limit_ms=3000,
                   stream_table=stream_table)
    assert r["nodes"] > 1000
    if r["has_solution"]:
        n = inst.n
        s = [int(v) for v in r["witness"][:n]]
        assert brute.rcpsp_feasible(inst, s)
        assert max(s[i] + inst.durations[i] for i in range(n)) == r["objective"]


def big_generic_model(seed):
    """16,000 variables and a ~200 KB table with every kind of stream segment:
    single reified rows, temporal rows, tiles of short linear rows, long rows
    that fit a 32 KB segment and one (9,000 terms) that does not.  The long
    rows hold disjoint Booleans that nothing else uses.  Seeded inputs only."""
    g = np.random.default_rng(seed)
    n_int, n_bool = 3000, 13000
    lb0 = [int(v) for v in g.integers(0, 50, n_int)] + [0] * n_bool
    ub0 = [lb0[i] + int(w) for i, w in enumerate(g.integers(2000, 6000, n_int))] + [1] * n_bool
    temporal = []
    for _ in range(3000):
        x, y = sorted(int(v) for v in g.choice(n_int, 2, replace=False))
        temporal.append((x, y, int(g.integers(0, 4))))
    reified = [(n_int + int(g.integers(0, 500)), int(g.integers(0, n_int)),
                int(g.integers(0, n_int)), int(g.integers(1, 7))) for _ in range(8000)]
    linear = []
    for _ in range(600):  # short rows over Booleans, resource-like
        ln = int(g.integers(10, 61))
        vs = [(int(a), n_int + int(v)) for a, v in
              zip(g.integers(1, 6, ln), g.choice(500, ln, replace=False))]
        linear.append((sum(a for a, _ in vs) // 2, vs))
    for _ in range(100):  # short rows with both signs over integers
        ln = int(g.integers(2, 9))
        vs = [(int(a) if a != 0 else 1, int(v)) for a, v in
              zip(g.integers(-4, 5, ln), g.choice(n_int, ln, replace=False))]
        linear.append((int(g.integers(0, 400)) + 50 * sum(max(a, 0) for a, _ in vs), vs))
    first = n_int + 500
    for ln in (1000, 2500, 9000):  # long rows; the last exceeds one segment
        vs = [(int(a), first + k) for k, a in enumerate(g.integers(1, 4, ln))]
        linear.append((sum(a for a, _ in vs) * 3 // 5, vs))
        first += ln
    return lb0, ub0, temporal, linear, reified


def big_generic_stores(lb0, ub0, linear):
    """Six stores: the root, two with random narrowings, and three that set
    Booleans of one long row to 1 while its sum stays at most its bound - 2
    (so that its remaining terms with coefficient 3 must drop to 0)."""
    g = np.random.default_rng(11)
    lb = np.tile(np.array(lb0, dtype=np.int32), (6, 1))
    ub = np.tile(np.array(ub0, dtype=np.int32), (6, 1))
    for s in (1, 2):
        for v in g.choice(len(lb0), 30, replace=False):
            if ub[s, v] > lb[s, v]:
                if g.integers(0, 2):
                    lb[s, v] = g.integers(lb[s, v], ub[s, v] + 1)
                else:
                    ub[s, v] = g.integers(lb[s, v], ub[s, v] + 1)
    for s, (c, terms) in zip((3, 4, 5), linear[-3:]):
        tot = 0
        for a, v in terms:
            if tot + a <= c - 2:
                lb[s, v] = 1
                tot += a
    return lb, ub


@pytest.mark.parametrize("stream_table, skip_stable", [(True, None), (False, None),
                                                       (False, False), (True, False)])
def test_streamed_segments_of_every_kind_bit_exact(stream_table, skip_stable):
    lb0, ub0, temporal, linear, reified = big_generic_model(5)
    m = pccp.Model.from_lists(lb0, ub0, temporal, linear, reified, -1, list(range(3000)))
    assert m.info.table_bytes + 8 * m.n_vars > 232448  # read from global memory
    assert m.info.table_bytes > 150_000
    assert m.info.n_segments >= 8
    om = oracle.Model(lb0, ub0, temporal, linear, reified, -1, list(range(3000)))
    lb, ub = big_generic_stores(lb0, ub0, linear)
    dlb, dub = torch.from_numpy(lb).cuda(), torch.from_numpy(ub).cuda()
    cfg = pccp.launch_config(stream_table=stream_table, skip_stable=skip_stable)
    st, it = pccp.propagate(m, dlb, dub, config=cfg)
    torch.cuda.synchronize()
    x, f = compare_batch(om, lb, ub, st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy())
    assert x >= 3
