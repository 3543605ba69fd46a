"""Booleans kept as bits (pccp_model_desc.bool_store): two bits of a shared
64-bit slot per Boolean instead of an int2, joins by atomic OR (lower bits)
and AND (upper bits).  The lattice and every result are the same as with
interval stores: fixed points, statuses, node counts and optima equal the
oracle's, with the layout forced on and off."""
import numpy as np
import pytest

import oracle
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from synthetic import SplitMix64, config_instance, draw_partial_assignments
from tests.gpu_util import compare_batch, compare_whole_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATUS = {oracle.RES_OPTIMAL: pccp.PCCP_RES_OPTIMAL, oracle.RES_INFEASIBLE: pccp.PCCP_RES_INFEASIBLE,
          oracle.RES_LIMIT: pccp.PCCP_RES_LIMIT}


def run(model, lb, ub, cfg=None):
    dlb = torch.from_numpy(np.ascontiguousarray(lb, dtype=np.int32)).cuda()
    dub = torch.from_numpy(np.ascontiguousarray(ub, dtype=np.int32)).cuda()
    st, it = pccp.propagate(model, dlb, dub, config=cfg)
    torch.cuda.synchronize()
    return st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy(), it.cpu().numpy()


def test_layout_is_reported():
    inst = config_instance("j30", 0)
    n = inst.n
    bits = pccp.Model.from_rcpsp(inst, bool_store=1)
    ints = pccp.Model.from_rcpsp(inst, bool_store=-1)
    dflt = pccp.Model.from_rcpsp(inst)
    assert bits.info.bool_vars == n * n and bits.info.store_bytes == 8 * ((n + 1) + (n * n + 31) // 32)
    assert ints.info.bool_vars == 0 and ints.info.store_bytes == 8 * (n + n * n + 1)
    assert dflt.info.bool_vars == 0  # interval stores that fit: the library keeps intervals
    big = pccp.Model.from_rcpsp(config_instance("j120", 0))
    assert big.info.bool_vars == 0  # 116 KB still fits
    huge = pccp.Model([0] * 40000, [1] * 40000)
    assert huge.info.bool_vars == 40000  # 320 KB would not: bits by default


@pytest.mark.parametrize("cfg", [None, pccp.launch_config(64, 8), pccp.launch_config(32, 1),
                                 pccp.launch_config(128, 4, skip_stable=True)])
def test_propagation_with_bits_is_bit_exact(cfg):
    inst = config_instance("j30", 3)
    om = rcpsp_model(inst)
    m = pccp.Model.from_rcpsp(inst, bool_store=1)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 3000, seed=11)
    lb, ub = pccp.rcpsp.node_stores(pccp.rcpsp.build_rows(inst), nodes)
    st, glb, gub, _ = run(m, lb, ub, cfg)
    nx, nf = compare_whole_batch(om, lb, ub, st, glb, gub)
    assert nx > 0 and nf > 0


def test_boolean_inputs_outside_zero_one():
    """Input stores may narrow a Boolean to an empty or out-of-range interval:
    the join with the root decides it, as for intervals."""
    inst = config_instance("j30", 1)
    om = rcpsp_model(inst)
    m = pccp.Model.from_rcpsp(inst, bool_store=1)
    n, nv = inst.n, inst.n + inst.n * inst.n + 1
    g = SplitMix64(99)
    lb = np.tile(om.lb0, (64, 1)).astype(np.int32)
    ub = np.tile(om.ub0, (64, 1)).astype(np.int32)
    for r in range(64):
        for _ in range(3):
            v = n + g.uniform_int(0, n * n - 1)
            kind = g.uniform_int(0, 4)
            if kind == 0:
                lb[r, v] = 1
            elif kind == 1:
                ub[r, v] = 0
            elif kind == 2:
                lb[r, v] = 2          # above the root: empty
            elif kind == 3:
                ub[r, v] = -1         # below the root: empty
            else:
                lb[r, v], ub[r, v] = -3, 5  # wider than the root: the root's box
    st, glb, gub, _ = run(m, lb, ub)
    compare_batch(om, lb, ub, st, glb, gub)


def test_sequential_search_counts_with_bits():
    for seed in range(0, 100, 7):
        inst = config_instance("tiny8", seed)
        om = rcpsp_model(inst)
        m = pccp.Model.from_rcpsp(inst, bool_store=1)
        assert m.info.bool_vars == 64
        for strat, ostrat in ((pccp.PCCP_INPUT_ORDER, oracle.INPUT_ORDER),
                              (pccp.PCCP_FIRST_FAIL, oracle.FIRST_FAIL)):
            r = pccp.solve(m, strategy=strat)
            o = oracle.solve(om, strategy=ostrat)
            assert r["status"] == STATUS[o["status"]]
            assert (r["nodes"], r["fails"], r["solutions"], r["max_depth"]) == \
                (o["nodes"], o["fails"], o["solutions"], o["max_depth"])
            assert r["objective"] == o["objective"] and np.array_equal(r["witness"], o["witness"])


@pytest.mark.parametrize("shape", [dict(), dict(teams_per_cta=2), dict(teams_per_cta=4, threads=128),
                                   dict(teams_per_cta=1, skip_stable=True)])
def test_batched_search_with_bits(shape):
    """30-60-task models with bits forced (their tables are then read from
    global memory): the sequential order's counts under a node limit equal
    the oracle's in every launch shape."""
    insts = [config_instance("mixed30_60", s) for s in range(8)]
    models = [pccp.Model.from_rcpsp(i, bool_store=1) for i in insts]
    assert all(m.info.bool_vars == i.n * i.n for m, i in zip(models, insts))
    res = pccp.solve_batch(models, strategy=pccp.PCCP_FIRST_FAIL, node_limit=150, **shape)
    for inst, r in zip(insts, res):
        o = oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL, node_limit=150)
        assert (r["nodes"], r["fails"], r["solutions"], r["max_depth"]) == \
            (o["nodes"], o["fails"], o["solutions"], o["max_depth"]), inst.name
        if o["has_solution"]:
            assert r["objective"] == o["objective"] and np.array_equal(r["witness"], o["witness"])


def test_parallel_search_with_bits():
    """Count-all and proof-tree counts are order-free, so the parallel search
    (one model shared by the CTA's teams, and many models over one queue)
    must match the oracle with bits too."""
    insts = [config_instance("tiny8", s) for s in range(0, 60, 5)]
    models = [pccp.Model.from_rcpsp(i, bool_store=1) for i in insts]
    oms = [rcpsp_model(i) for i in insts]
    opts = [oracle.solve(om)["objective"] for om in oms]
    for m, om, z in zip(models, oms, opts):
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=z)
        r = pccp.solve(m, mode=pccp.PCCP_COUNT_ALL, obj_ub=z, deterministic=False)
        assert (r["nodes"], r["fails"], r["solutions"]) == (c["nodes"], c["fails"], c["solutions"])
        p = oracle.solve(om, obj_ub=z - 1)
        rp = pccp.solve(m, obj_ub=z - 1, deterministic=False, donate_nodes=1)
        assert (rp["nodes"], rp["fails"]) == (p["nodes"], p["fails"])
    res = pccp.solve_batch(models, deterministic=False)
    assert [r["objective"] for r in res] == opts


def _qualifying_generic(seed, n_int=5, n_bool=40, n_reified=30, n_linear=6):
    """A random model whose Booleans appear only as reified b's and in
    all-positive 0/1 linear rows (so they may be kept as bits)."""
    g = SplitMix64.derive(seed, 0xB175)
    lb0 = [g.uniform_int(-6, 2) for _ in range(n_int)] + [0] * n_bool
    ub0 = [l + g.uniform_int(2, 12) for l in lb0[:n_int]] + [1] * n_bool
    for k in range(n_bool):
        r = g.uniform_int(0, 9)
        if r == 0:
            lb0[n_int + k] = 1
        elif r == 1:
            ub0[n_int + k] = 0
    temporal = [(g.uniform_int(0, n_int - 1), g.uniform_int(0, n_int - 1), g.uniform_int(-5, 3))
                for _ in range(4)]
    reified = [(n_int + g.uniform_int(0, n_bool - 1), g.uniform_int(0, n_int - 1),
                g.uniform_int(0, n_int - 1), g.uniform_int(1, 5)) for _ in range(n_reified)]
    linear = []
    for _ in range(n_linear):
        ln = g.uniform_int(2, 40 if g.uniform_int(0, 2) else 80)
        terms = [(g.uniform_int(1, 6), n_int + g.uniform_int(0, n_bool - 1)) for _ in range(ln)]
        linear.append((g.uniform_int(3, 30), terms))
    return lb0, ub0, temporal, linear, reified


def test_generic_models_with_bits():
    for seed in range(30):
        lb0, ub0, temporal, linear, reified = _qualifying_generic(seed)
        m = pccp.Model.from_lists(lb0, ub0, temporal, linear, reified, bool_store=1)
        assert m.info.bool_vars > 0
        om = oracle.Model(lb0, ub0, temporal, linear, reified)
        g = SplitMix64.derive(seed, 5)
        lbs, ubs = [], []
        for _ in range(40):
            lb, ub = list(lb0), list(ub0)
            for v in range(len(lb0)):
                if g.bernoulli(0.2) and ub[v] > lb[v]:
                    if g.bernoulli(0.5):
                        lb[v] = g.uniform_int(lb[v], ub[v])
                    else:
                        ub[v] = g.uniform_int(lb[v], ub[v])
            lbs.append(lb)
            ubs.append(ub)
        lb, ub = np.array(lbs), np.array(ubs)
        for cfg in (None, pccp.launch_config(32, 1), pccp.launch_config(64, 4, skip_stable=True)):
            st, glb, gub, _ = run(m, lb, ub, cfg)
            compare_batch(om, lb, ub, st, glb, gub)
