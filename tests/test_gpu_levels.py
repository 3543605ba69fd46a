"""Temporal rows walked in topological levels (pccp_launch_config /
pccp_solve_opts temporal_levels).  Only the order in which the rows run
changes, so every fixed point, status and search count equals the oracle's
with the levels forced on, forced off and left to the library, in every
team size (one warp doing both passes, two warps, more)."""
import numpy as np
import pytest

import oracle
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from synthetic import SplitMix64, config_instance, draw_partial_assignments
from tests.gpu_util import compare_batch, compare_whole_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVELS = (None, True, False)


def run(model, lb, ub, cfg=None):
    dlb = torch.from_numpy(np.ascontiguousarray(lb, dtype=np.int32)).cuda()
    dub = torch.from_numpy(np.ascontiguousarray(ub, dtype=np.int32)).cuda()
    st, it = pccp.propagate(model, dlb, dub, config=cfg)
    torch.cuda.synchronize()
    return st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy(), it.cpu().numpy()


def longest_chain_levels(n_vars, rows):
    """Levels counted by a memoised depth-first search backwards over the
    rows (not the library's queue of sources): the level of v is the number
    of rows on the longest chain of rows ending at v; the count is 1 + the
    largest level of a row's x, 0 when some chain meets itself (a cycle) or
    there are no rows."""
    into = {v: [] for v in range(n_vars)}
    for (x, y, _) in rows:
        into[y].append(x)
    memo, active = {}, set()

    def level(v):
        if v in memo:
            return memo[v]
        if v in active:
            raise ValueError("cycle")
        active.add(v)
        lv = max((1 + level(x) for x in into[v]), default=0)
        active.discard(v)
        memo[v] = lv
        return lv

    if not rows:
        return 0
    try:
        return 1 + max(level(x) for (x, _, _) in rows)
    except ValueError:
        return 0


def test_level_counts():
    chain = pccp.Model.from_lists([0] * 6, [50] * 6, temporal=[(i, i + 1, 2) for i in range(5)])
    assert chain.info.temporal_levels == 5
    cyc = pccp.Model.from_lists([0, 0, 0], [9, 9, 9], temporal=[(0, 1, 1), (1, 2, 1), (2, 0, -5)])
    assert cyc.info.temporal_levels == 0
    selfrow = pccp.Model.from_lists([0, 0], [9, 9], temporal=[(0, 1, 1), (1, 1, 0)])
    assert selfrow.info.temporal_levels == 0
    assert pccp.Model.from_lists([0], [9]).info.temporal_levels == 0
    for fam, seed in (("tiny8", 3), ("j30", 0), ("mixed30_60", 5)):
        inst = config_instance(fam, seed)
        om = rcpsp_model(inst)
        m = pccp.Model.from_rcpsp(inst)
        assert m.info.temporal_levels == longest_chain_levels(len(om.lb0), om.temporal)


def test_chain_closes_in_one_sweep():
    """A chain of 40 rows from both ends: with levels the first sweep carries
    every bound along the chain and the second finds nothing left, so each
    store takes exactly two iterations in every team size."""
    n = 41
    m = pccp.Model.from_lists([0] * n, [1000] * n, temporal=[(i, i + 1, 3) for i in range(n - 1)])
    om = oracle.Model([0] * n, [1000] * n, [(i, i + 1, 3) for i in range(n - 1)])
    lb = np.zeros((4, n), dtype=np.int32)
    ub = np.full((4, n), 1000, dtype=np.int32)
    lb[1, 0], ub[2, n - 1], lb[3, 5], ub[3, 30] = 10, 500, 7, 200
    for cfg in (pccp.launch_config(32, 1, temporal_levels=True),
                pccp.launch_config(64, 2, temporal_levels=True),
                pccp.launch_config(256, 1, temporal_levels=True),
                pccp.launch_config(128, 4, skip_stable=True, temporal_levels=True)):
        st, glb, gub, it = run(m, lb, ub, cfg)
        compare_batch(om, lb, ub, st, glb, gub)
        assert it.tolist() == [2, 2, 2, 2]


@pytest.mark.parametrize("levels", LEVELS)
@pytest.mark.parametrize("cfg", [dict(), dict(team_threads=32, teams_per_cta=4),
                                 dict(team_threads=64, teams_per_cta=2),
                                 dict(team_threads=256, teams_per_cta=2, skip_stable=True)])
def test_scheduling_fixed_points(levels, cfg):
    inst = config_instance("j30", 2)
    om = rcpsp_model(inst)
    m = pccp.Model.from_rcpsp(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 2000, seed=5)
    lb, ub = pccp.rcpsp.node_stores(pccp.rcpsp.build_rows(inst), nodes)
    st, glb, gub, _ = run(m, lb, ub, pccp.launch_config(temporal_levels=levels, **cfg))
    nx, nf = compare_whole_batch(om, lb, ub, st, glb, gub)
    assert nx > 100 and nf > 100


@pytest.mark.parametrize("levels", LEVELS)
def test_large_model_fixed_points(levels):
    """120 tasks: the table is read from global memory and the levels from
    the copy each CTA keeps in shared memory."""
    inst = config_instance("j120", 1)
    om = rcpsp_model(inst)
    m = pccp.Model.from_rcpsp(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 304, seed=8)
    lb, ub = pccp.rcpsp.node_stores(pccp.rcpsp.build_rows(inst), nodes)
    for cfg in (pccp.launch_config(temporal_levels=levels),
                pccp.launch_config(512, 1, skip_stable=False, temporal_levels=levels)):
        st, glb, gub, _ = run(m, lb, ub, cfg)
        compare_whole_batch(om, lb, ub, st, glb, gub)


def _dag_model(seed, n_int=12, n_rows=30, n_bool=6):
    """Random acyclic temporal rows (edges follow a random order of the
    variables, durations of either sign) with reified and linear rows."""
    g = SplitMix64.derive(seed, 0x7E1)
    perm = list(range(n_int))
    for i in range(n_int - 1, 0, -1):
        j = g.uniform_int(0, i)
        perm[i], perm[j] = perm[j], perm[i]
    lb0 = [g.uniform_int(-10, 5) for _ in range(n_int)] + [0] * n_bool
    ub0 = [l + g.uniform_int(5, 60) for l in lb0[:n_int]] + [1] * n_bool
    temporal = []
    for _ in range(n_rows):
        a = g.uniform_int(0, n_int - 2)
        b = g.uniform_int(a + 1, n_int - 1)
        temporal.append((perm[a], perm[b], g.uniform_int(-4, 9)))
    reified = [(n_int + g.uniform_int(0, n_bool - 1), g.uniform_int(0, n_int - 1),
                g.uniform_int(0, n_int - 1), g.uniform_int(1, 6)) for _ in range(8)]
    linear = [(g.uniform_int(2, 6), [(g.uniform_int(1, 3), n_int + g.uniform_int(0, n_bool - 1))
                                     for _ in range(3)]) for _ in range(3)]
    return lb0, ub0, temporal, linear, reified


def test_generic_dags():
    for seed in range(40):
        lb0, ub0, temporal, linear, reified = _dag_model(seed)
        m = pccp.Model.from_lists(lb0, ub0, temporal, linear, reified)
        om = oracle.Model(lb0, ub0, temporal, linear, reified)
        assert m.info.temporal_levels == longest_chain_levels(len(lb0), temporal)
        g = SplitMix64.derive(seed, 9)
        lbs, ubs = [], []
        for _ in range(48):
            lb, ub = list(lb0), list(ub0)
            for v in range(len(lb0)):
                if g.bernoulli(0.25) and ub[v] > lb[v]:
                    if g.bernoulli(0.5):
                        lb[v] = g.uniform_int(lb[v], ub[v])
                    else:
                        ub[v] = g.uniform_int(lb[v], ub[v])
            lbs.append(lb)
            ubs.append(ub)
        lb, ub = np.array(lbs), np.array(ubs)
        for cfg in (pccp.launch_config(temporal_levels=True),
                    pccp.launch_config(32, 1, temporal_levels=True),
                    pccp.launch_config(96, 2, skip_stable=True, temporal_levels=True)):
            st, glb, gub, _ = run(m, lb, ub, cfg)
            compare_batch(om, lb, ub, st, glb, gub)


@pytest.mark.parametrize("levels", LEVELS)
def test_search_counts(levels):
    """The sequential order's counts (nodes, fails, solutions, depth,
    optimum, witness) do not depend on the order rows run in."""
    insts = [config_instance("mixed30_60", s) for s in range(6)]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    res = pccp.solve_batch(models, strategy=pccp.PCCP_FIRST_FAIL, node_limit=200,
                           temporal_levels=levels)
    for inst, r in zip(insts, res):
        o = oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL, node_limit=200)
        assert (r["nodes"], r["fails"], r["solutions"], r["max_depth"]) == \
            (o["nodes"], o["fails"], o["solutions"], o["max_depth"]), inst.name
        if o["has_solution"]:
            assert r["objective"] == o["objective"] and np.array_equal(r["witness"], o["witness"])
    for s in range(0, 40, 7):
        inst = config_instance("tiny8", s)
        om = rcpsp_model(inst)
        z = oracle.solve(om)["objective"]
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=z)
        m = pccp.Model.from_rcpsp(inst)
        r = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, obj_ub=z, deterministic=False,
                       temporal_levels=levels)
        assert (r["nodes"], r["fails"], r["solutions"]) == (c["nodes"], c["fails"], c["solutions"])


def test_large_model_search_counts():
    inst = config_instance("j120", 0)
    m = pccp.Model.from_rcpsp(inst)
    o = oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL, node_limit=12)
    for levels in LEVELS:
        r = pccp.solve(m, strategy=pccp.PCCP_FIRST_FAIL, node_limit=12, temporal_levels=levels)
        assert (r["nodes"], r["fails"], r["max_depth"]) == (o["nodes"], o["fails"], o["max_depth"])
