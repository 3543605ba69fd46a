"""GPU parity of pccp_propagate (through the C ABI) with the CPU oracle:
bit-exact lb/ub on every store that reaches a fixed point, equal status on
every store (the fixed point is unique for any fair order: Theorem 1 and the
fix D = fix O theorem; the load/store soundness and completeness theorems
carry it to the lock-free GPU execution)."""
import numpy as np
import pytest

import oracle
from oracle.rcpsp import rcpsp_model, node_store
import paper_2207_12116_gb300 as pccp
from synthetic import (config_instance, draw_generic_model, draw_generic_store,
                       draw_partial_assignments, SplitMix64)
from tests.gpu_util import compare_batch, compare_whole_batch, oracle_model_from_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(model, lb, ub, cfg=None):
    dlb = torch.from_numpy(np.ascontiguousarray(lb, dtype=np.int32)).cuda()
    dub = torch.from_numpy(np.ascontiguousarray(ub, dtype=np.int32)).cuda()
    st, it = pccp.propagate(model, dlb, dub, config=cfg)
    torch.cuda.synchronize()
    return st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy(), it.cpu().numpy()


def generic_batch(seed, n_stores, **kw):
    gm = draw_generic_model(seed, **kw)
    m = pccp.Model.from_lists(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                              gm.objective, gm.branch)
    lbs, ubs = [], []
    for k in range(n_stores):
        lb, ub = draw_generic_store(gm, seed * 1000 + k)
        lbs.append(lb)
        ubs.append(ub)
    return gm, m, np.array(lbs), np.array(ubs)


CONFIGS = [None,
           pccp.launch_config(32, 1),
           pccp.launch_config(64, 4),
           pccp.launch_config(128, 8),
           pccp.launch_config(256, 2),
           pccp.launch_config(1024, 1),
           pccp.launch_config(96, 10, 1),
           pccp.launch_config(128, 4, skip_stable=True),
           pccp.launch_config(64, 8, skip_stable=True),
           pccp.launch_config(1024, 1, skip_stable=True)]


@pytest.mark.parametrize("cfg_i", range(len(CONFIGS)))
def test_generic_models_bit_exact(cfg_i):
    tot_x = tot_f = 0
    for seed in range(60):
        gm, m, lb, ub = generic_batch(seed, 24)
        st, glb, gub, _ = run(m, lb, ub, CONFIGS[cfg_i])
        x, f = compare_batch(oracle_model_from_lists(gm), lb, ub, st, glb, gub)
        tot_x += x
        tot_f += f
    assert tot_x > 100 and tot_f > 100


def test_long_linear_rows_and_wide_domains():
    """Rows longer than a warp (the reload path), large coefficients."""
    tot_x = 0
    for seed in range(40):
        gm, m, lb, ub = generic_batch(10_000 + seed, 16, n_int=40, n_bool=40, dom=300,
                                      n_temporal=4, n_linear=6, n_reified=8, max_len=100,
                                      coef=30)
        st, glb, gub, _ = run(m, lb, ub)
        x, _ = compare_batch(oracle_model_from_lists(gm), lb, ub, st, glb, gub)
        tot_x += x
    assert tot_x > 20


def test_j30_nodes_bit_exact():
    inst = config_instance("j30", 0)
    m = pccp.Model.from_rcpsp(inst)
    assert m.info.reordered == 0  # the caller's order has fewer bank conflicts here
    om = rcpsp_model(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 1500, seed=1)
    rows = pccp.rcpsp.build_rows(inst)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    olb = np.array([node_store(om, d)[0] for d in nodes])
    oub = np.array([node_store(om, d)[1] for d in nodes])
    assert np.array_equal(olb, lb) and np.array_equal(oub, ub)  # same inputs both sides
    st, glb, gub, it = run(m, lb, ub)
    x, f = compare_batch(om, lb, ub, st, glb, gub)
    assert x > 100 and f > 100
    assert (it[st == 0] >= 1).all()
    # work report: every row runs in the first iteration, stable rows are
    # skipped afterwards, never more than iterations x rows
    dlb = torch.from_numpy(lb).cuda()
    dub = torch.from_numpy(ub).cuda()
    work = torch.zeros((len(nodes), 2), dtype=torch.int32, device="cuda")
    st2, it2 = pccp.propagate(m, dlb, dub, work=work, config=pccp.launch_config(skip_stable=True))
    torch.cuda.synchronize()
    w, it2 = work.cpu().numpy(), it2.cpu().numpy()
    ok = st2.cpu().numpy() == 0
    assert (w[ok, 0] >= m.rows).all() and (w[ok, 0] <= it2[ok] * m.rows).all()
    assert w[ok, 0].sum() < it2[ok].sum() * m.rows  # something was skipped


def test_degenerate_temporal_rows_bit_exact():
    """Rows the generic generator no longer draws (it keeps self-rows
    x + d <= x at d <= 0 and backward rows mostly slack so that random
    models keep solutions): a self-row with d > 0 (fails whatever the
    store), precedence cycles of positive length (infeasible: bounds rise
    until an interval empties) and of non-positive length (feasible), mixed
    into generic models and compared with the oracle store by store."""
    tot_f = tot_x = 0
    for seed in range(40):
        gm = draw_generic_model(4000 + seed)
        g = SplitMix64.derive(seed, 77)
        extra = []
        kind = seed % 4
        x, y, z = 0, 1 + g.uniform_int(0, 2), 4 + g.uniform_int(0, 1)
        if kind == 0:
            extra = [(x, x, 1 + g.uniform_int(0, 3))]
        elif kind == 1:
            extra = [(x, y, 2), (y, z, 1), (z, x, g.uniform_int(-2, 0))]
        elif kind == 2:
            extra = [(x, y, 3), (y, x, -3 - g.uniform_int(0, 2))]
        else:
            extra = [(x, x, -g.uniform_int(0, 3)), (y, z, -1), (z, y, 1)]
        temporal = list(gm.temporal) + extra
        m = pccp.Model.from_lists(gm.lb0, gm.ub0, temporal, gm.linear, gm.reified,
                                  gm.objective, gm.branch)
        om = oracle.Model(gm.lb0, gm.ub0, temporal, gm.linear, gm.reified, gm.objective,
                          gm.branch)
        lbs, ubs = zip(*[draw_generic_store(gm, 100 * seed + k) for k in range(16)])
        lb, ub = np.array(lbs), np.array(ubs)
        st, glb, gub, _ = run(m, lb, ub)
        x_, f_ = compare_batch(om, lb, ub, st, glb, gub)
        tot_x += x_
        tot_f += f_
        if kind in (0, 1):  # a positive self-row or a positive cycle: nothing survives
            assert (st == pccp.PCCP_FAILED).all()
    assert tot_f > 0 and tot_x > 0


def test_uneven_models_bit_exact():
    for seed in range(6):
        inst = config_instance("mixed30_60", seed)
        m = pccp.Model.from_rcpsp(inst)
        om = rcpsp_model(inst)
        nodes = draw_partial_assignments(inst.n, inst.horizon, 150, seed=100 + seed)
        lb, ub = pccp.rcpsp.node_stores(pccp.rcpsp.build_rows(inst), nodes)
        st, glb, gub, _ = run(m, lb, ub)
        compare_batch(om, lb, ub, st, glb, gub)


def test_full_size_batch_every_store():
    """The 10,000-node j30 batch in the default launch shape: every store
    compared with the oracle, element by element (the oracle's batch split
    over the host cores), plus properties that hold at any size
    (re-propagating a fixed point changes nothing and takes one iteration;
    results lie inside the input box)."""
    inst = config_instance("j30", 0)
    m = pccp.Model.from_rcpsp(inst)
    om = rcpsp_model(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 10_000, seed=1)
    lb, ub = pccp.rcpsp.node_stores(pccp.rcpsp.build_rows(inst), nodes)
    st, glb, gub, it = run(m, lb, ub)
    nx, nf = compare_whole_batch(om, lb, ub, st, glb, gub)
    assert nx + nf == 10_000 and nx > 0 and nf > 0
    ok = st == pccp.PCCP_FIXPOINT
    assert set(np.unique(st)) <= {0, 1}
    assert (glb[ok] >= lb[ok]).all() and (gub[ok] <= ub[ok]).all()
    st2, glb2, gub2, it2 = run(m, glb[ok], gub[ok])
    assert (st2 == 0).all() and (it2 == 1).all()
    assert np.array_equal(glb2, glb[ok]) and np.array_equal(gub2, gub[ok])


def test_launch_shapes_agree():
    gm, m, lb, ub = generic_batch(77, 200, n_int=12, n_bool=12, n_temporal=12, n_linear=5,
                                  n_reified=12, max_len=8)
    ref = run(m, lb, ub)
    for cfg in CONFIGS[1:]:
        out = run(m, lb, ub, cfg)
        ok = ref[0] == 0
        assert np.array_equal(out[0], ref[0])
        assert np.array_equal(out[1][ok], ref[1][ok]) and np.array_equal(out[2][ok], ref[2][ok])


def test_edge_cases():
    # no rows at all: the result is the input joined with the root
    m = pccp.Model([0, -3], [9, 3])
    st, glb, gub, it = run(m, np.array([[2, -9], [5, 0]]), np.array([[20, 9], [4, 0]]))
    assert st.tolist() == [0, 1]
    assert glb[0].tolist() == [2, -3] and gub[0].tolist() == [9, 3]
    # zero stores queue nothing
    e = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    st0, _ = pccp.propagate(m, e, e.clone())
    assert st0.numel() == 0
    # an infeasible cycle x + 1 <= y, y + 1 <= x must end in failure
    cyc = pccp.Model.from_lists([0, 0], [1000, 1000], temporal=[(0, 1, 1), (1, 0, 1)])
    st, _, _, it = run(cyc, np.array([[0, 0]]), np.array([[1000, 1000]]))
    assert st.tolist() == [1] and it[0] >= 1
    # one store, one variable, a linear row fixing it
    one = pccp.Model.from_lists([0], [10], linear=[(7, [(2, 0)])])
    st, glb, gub, _ = run(one, np.array([[0]]), np.array([[10]]))
    assert st.tolist() == [0] and gub[0].tolist() == [3]
    # an iteration budget of 1 on a store that needs more reports PCCP_ERROR
    chain = pccp.Model.from_lists([0] * 6, [50] * 6, temporal=[(i, i + 1, 2) for i in range(5)])
    st, *_ = run(chain, np.zeros((1, 6)), np.full((1, 6), 50), pccp.launch_config(32, 1, 0, 1))
    assert st.tolist() == [pccp.PCCP_ERROR]


def test_store_size_limits():
    """A store larger than shared memory is refused on the host; a store near
    the limit (table read from global memory) is still bit-exact."""
    big = pccp.Model([0] * 40000, [1] * 40000, bool_store=-1)
    assert big.info.max_store_vars < 40000
    with pytest.raises(pccp.PccpError) as e:
        run(big, np.zeros((1, 40000)), np.ones((1, 40000)))
    assert e.value.code == pccp.PCCP_ERR_SMEM
    # the same 40,000 Booleans kept as bits (the default: intervals would not fit)
    bits = pccp.Model([0] * 40000, [1] * 40000)
    assert bits.info.bool_vars == 40000 and bits.info.store_bytes == 8 * 1250
    lb = np.zeros((2, 40000), dtype=np.int32)
    ub = np.ones((2, 40000), dtype=np.int32)
    lb[0, ::3] = 1
    ub[0, 1::3] = 0
    lb[1, 7], ub[1, 7] = 1, 0
    st, glb, gub, _ = run(bits, lb, ub)
    assert st.tolist() == [0, 1]
    assert np.array_equal(glb[0], lb[0]) and np.array_equal(gub[0], ub[0])
    n = int(0.9 * pccp.Model([0], [1]).info.max_store_vars)
    g = np.random.default_rng(4)
    lb0 = [0] * n
    ub0 = [int(v) for v in g.integers(100, 100000, n)]
    temporal = [(i, i + 1, int(g.integers(0, 3))) for i in range(0, n - 1, 2)]
    linear = [(int(g.integers(50, 500)), [(1, int(a)), (2, int(b)), (-1, int(c))])
              for a, b, c in g.integers(0, n, (2000, 3))]
    m = pccp.Model.from_lists(lb0, ub0, temporal, linear)
    om = oracle.Model(lb0, ub0, temporal, linear, [], -1, [])
    lb = np.tile(np.array(lb0, dtype=np.int32), (3, 1))
    ub = np.tile(np.array(ub0, dtype=np.int32), (3, 1))
    lb[1, ::7] = 40
    ub[2, 1::5] = 30
    st, glb, gub, _ = run(m, lb, ub)
    x, f = compare_batch(om, lb, ub, st, glb, gub)
    assert x >= 2


@pytest.mark.parametrize("pinned, chunk", [(True, 250), (True, 0), (False, 400), (False, 0),
                                           (True, pccp.PCCP_HOST_IN_PLACE)])
def test_host_memory_pipeline_bit_exact(pinned, chunk):
    """pccp_propagate_host: stores in host memory, copied in and out in chunks
    (ragged last chunk) while other chunks propagate, or read and written in
    place by the kernel (PCCP_HOST_IN_PLACE); results equal the oracle's and
    the device entry point's."""
    inst = config_instance("j30", 3)
    m = pccp.Model.from_rcpsp(inst)
    om = rcpsp_model(inst)
    rows = pccp.rcpsp.build_rows(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 600, seed=5)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    hlb, hub = torch.from_numpy(lb.copy()), torch.from_numpy(ub.copy())
    if pinned:
        hlb, hub = hlb.pin_memory(), hub.pin_memory()
    st, it = pccp.propagate_host(m, hlb, hub, chunk_stores=chunk)
    x, f = compare_batch(om, lb, ub, st.numpy(), hlb.numpy(), hub.numpy())
    assert x > 100 and f > 10
    dst, dlb, dub, dit = run(m, lb, ub)
    assert np.array_equal(st.numpy(), dst) and np.array_equal(hlb.numpy()[st.numpy() == 0],
                                                               dlb[dst == 0])


def test_host_in_place_needs_mapped_memory():
    inst = config_instance("j30", 3)
    m = pccp.Model.from_rcpsp(inst)
    lb = torch.tensor(m.lb0, dtype=torch.int32)[None].repeat(8, 1)
    ub = torch.tensor(m.ub0, dtype=torch.int32)[None].repeat(8, 1)
    for chunk in (pccp.PCCP_HOST_IN_PLACE, -2):
        with pytest.raises(pccp.PccpError) as e:
            pccp.propagate_host(m, lb.clone(), ub.clone(), chunk_stores=chunk)
        assert e.value.code == pccp.PCCP_ERR_INVALID
    # the chunked copies take any mix of pinned and pageable arrays
    plb, pub = lb.clone().pin_memory(), ub.clone().pin_memory()
    st = torch.empty(8, dtype=torch.int32)
    pccp.propagate_host(m, plb, pub, status=st)
    with pytest.raises(pccp.PccpError):
        pccp.propagate_host(m, lb.clone().pin_memory(), ub.clone().pin_memory(), status=st,
                            chunk_stores=pccp.PCCP_HOST_IN_PLACE)
    dst, dlb, dub, _ = run(m, lb.numpy(), ub.numpy())
    assert np.array_equal(st.numpy(), dst) and np.array_equal(plb.numpy()[dst == 0], dlb[dst == 0])


@pytest.mark.parametrize("family, n_nodes", [("tiny8", 300), ("j120", 48)])
def test_host_in_place_reordered_and_global_tables(family, n_nodes):
    """In place on a model kept in the library's own variable order (staging
    through the variable map) and on a 120-task model whose table is read
    from global memory: equal to the device entry point, and to the oracle
    on the stores it checks."""
    inst = config_instance(family, 0)
    m = pccp.Model.from_rcpsp(inst)
    if family == "tiny8":
        assert m.info.reordered == 1
    rows = pccp.rcpsp.build_rows(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, n_nodes, seed=11)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    hlb, hub = torch.from_numpy(lb.copy()).pin_memory(), torch.from_numpy(ub.copy()).pin_memory()
    st, it = pccp.propagate_host(m, hlb, hub, chunk_stores=pccp.PCCP_HOST_IN_PLACE)
    dst, dlb, dub, dit = run(m, lb, ub)
    # (iteration counts depend on the interleaving of the tells: not compared)
    assert np.array_equal(st.numpy(), dst) and (it.numpy()[dst == 0] >= 1).all()
    fx = dst == 0
    assert np.array_equal(hlb.numpy()[fx], dlb[fx]) and np.array_equal(hub.numpy()[fx], dub[fx])
    om = rcpsp_model(inst)
    sample = range(n_nodes) if family == "tiny8" else range(0, n_nodes, 12)
    x, f = compare_batch(om, lb, ub, st.numpy(), hlb.numpy(), hub.numpy(), rows=sample)
    assert x + f == len(sample)


def test_host_default_chunking_large_batch():
    """10,000 stores through the default chunking (a one-store-per-team first
    chunk, then chunks of two stores per team, four slots reused): equal to
    the device entry point everywhere and to the oracle on stores around
    every chunk boundary."""
    inst = config_instance("j30", 0)
    m = pccp.Model.from_rcpsp(inst)
    rows = pccp.rcpsp.build_rows(inst)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 10_000, seed=21)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    hlb, hub = torch.from_numpy(lb.copy()).pin_memory(), torch.from_numpy(ub.copy()).pin_memory()
    st, it = pccp.propagate_host(m, hlb, hub)
    dst, dlb, dub, _ = run(m, lb, ub)
    fx = dst == 0
    assert np.array_equal(st.numpy(), dst)
    assert np.array_equal(hlb.numpy()[fx], dlb[fx]) and np.array_equal(hub.numpy()[fx], dub[fx])
    assert (it.numpy()[fx] >= 1).all()
    sample = sorted({i for b in range(0, 10_001, 608) for i in (b - 1, b) if 0 <= i < 10_000})
    x, f = compare_batch(rcpsp_model(inst), lb, ub, st.numpy(), hlb.numpy(), hub.numpy(),
                         rows=sample)
    assert x + f == len(sample)


def test_host_pipeline_graph_replays():
    """With every array pinned, the chunked call is captured in a CUDA graph
    on its first use and replayed by later calls on the same arrays: fresh
    contents every call give the device entry point's results; other sizes,
    chunkings and arrays capture anew, and going back recaptures; a pageable
    status array takes the directly queued path on the same model."""
    inst = config_instance("j30", 2)
    m = pccp.Model.from_rcpsp(inst)
    rows = pccp.rcpsp.build_rows(inst)
    om = rcpsp_model(inst)
    n = 1500
    hlb = torch.empty((n, m.n_vars), dtype=torch.int32).pin_memory()
    hub = torch.empty((n, m.n_vars), dtype=torch.int32).pin_memory()
    st = torch.empty(n, dtype=torch.int32).pin_memory()
    it = torch.empty(n, dtype=torch.int32).pin_memory()

    def check(k, chunk, count, status=None):
        nodes = draw_partial_assignments(inst.n, inst.horizon, count, seed=100 + k)
        lb, ub = pccp.rcpsp.node_stores(rows, nodes)
        plb, pub = hlb[:count], hub[:count]
        plb.copy_(torch.from_numpy(lb))
        pub.copy_(torch.from_numpy(ub))
        s_ = st[:count] if status is None else status
        pccp.propagate_host(m, plb, pub, s_, it[:count], chunk_stores=chunk)
        dst, dlb, dub, _ = run(m, lb, ub)
        fx = dst == 0
        assert np.array_equal(s_.numpy(), dst), (k, chunk, count)
        assert np.array_equal(plb.numpy()[fx], dlb[fx]) and np.array_equal(pub.numpy()[fx], dub[fx])
        assert 0 < fx.sum() < count
        x, f = compare_batch(om, lb, ub, s_.numpy(), plb.numpy(), pub.numpy(),
                             rows=range(k, count, 97))
        assert x + f == len(range(k, count, 97))

    for k in range(3):
        check(k, 0, n)
    check(3, 400, n)
    check(4, 0, 700)
    check(5, 0, n)
    check(6, 0, 300, status=torch.empty(300, dtype=torch.int32))
    check(7, 0, n)


def test_models_of_different_sizes_interleaved_and_threaded():
    """A small model planned between two calls on a larger one (same kernel,
    less shared memory) leaves the larger one launchable, in sequence and
    from concurrent host threads on separate streams; results stay exact."""
    import threading
    big_inst, small_inst = config_instance("j30", 1), config_instance("tiny8", 3)
    big, small = pccp.Model.from_rcpsp(big_inst), pccp.Model.from_rcpsp(small_inst)
    assert big.info.table_bytes > 4 * small.info.table_bytes

    def batch(inst, n, seed):
        rows = pccp.rcpsp.build_rows(inst)
        return pccp.rcpsp.node_stores(rows, draw_partial_assignments(inst.n, inst.horizon, n,
                                                                     seed=seed))

    blb, bub = batch(big_inst, 300, 2)
    slb, sub = batch(small_inst, 300, 3)
    ref_big, ref_small = run(big, blb, bub), run(small, slb, sub)

    def same(ref, st, lb, ub):
        fx = ref[0] == 0
        return (np.array_equal(ref[0], st) and np.array_equal(ref[1][fx], lb[fx])
                and np.array_equal(ref[2][fx], ub[fx]))

    for _ in range(2):  # host entry point keeps its plan across the small model's calls
        h = [torch.from_numpy(blb.copy()).pin_memory(), torch.from_numpy(bub.copy()).pin_memory()]
        st, _ = pccp.propagate_host(big, h[0], h[1])
        assert same(ref_big, st.numpy(), h[0].numpy(), h[1].numpy())
        assert same(ref_small, *run(small, slb, sub)[:3])

    errors = []

    def worker(model, lb, ub, ref):
        try:
            stream = torch.cuda.Stream()
            for _ in range(20):
                with torch.cuda.stream(stream):
                    dlb = torch.from_numpy(lb).cuda()
                    dub = torch.from_numpy(ub).cuda()
                    st, _ = pccp.propagate(model, dlb, dub, stream=stream)
                stream.synchronize()
                if not same(ref, st.cpu().numpy(), dlb.cpu().numpy(), dub.cpu().numpy()):
                    errors.append("mismatch")
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))

    ts = [threading.Thread(target=worker, args=a) for a in
          ((big, blb, bub, ref_big), (small, slb, sub, ref_small),
           (big, blb, bub, ref_big), (small, slb, sub, ref_small))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors[:3]
