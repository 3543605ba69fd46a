"""Pins for the CPU oracle: each check compares it with something other than
itself (brute-force enumeration, a closed form, the paper's theorems as
executable invariants), chosen so a dropped term, a wrong sign, an off-by-one
or a swapped operand in any guarded command fails at least one test."""

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model, node_store, var_M
from synthetic import SplitMix64, config_instance, draw_generic_model, draw_generic_store
from synthetic.rcpsp import RcpspDistribution, draw_rcpsp


def hull(solutions, nv):
    a = np.asarray(solutions, dtype=np.int64).reshape(-1, nv)
    return a.min(axis=0), a.max(axis=0)


# ------------------------------------------------------------ single rows

@pytest.mark.parametrize("seed", range(300))
def test_single_linear_row_equals_projection_hull(seed):
    """One linear inequality over distinct variables: bounds propagation is
    exact, so the fixed point is the integer hull of its solution set
    (Sec. 2, [[sum r*b <= c]] generalised to any sign)."""
    g = SplitMix64.derive(seed, 11)
    nv = g.uniform_int(1, 4)
    lb = [g.uniform_int(-5, 3) for _ in range(nv)]
    ub = [l + g.uniform_int(0, 6) for l in lb]
    terms = []
    for v in range(nv):
        a = g.uniform_int(-4, 4) or 3
        terms.append((a, v))
    c = g.uniform_int(-15, 15)
    m = oracle.Model(lb, ub, linear=[(c, terms)])
    st, flb, fub, _ = oracle.propagate(m, lb, ub)
    sols = brute.generic_solutions([], [(c, terms)], [], lb, ub)
    if not sols:
        assert st == oracle.FAILED
    else:
        assert st == oracle.FIXPOINT
        hl, hu = hull(sols, nv)
        assert list(flb) == list(hl) and list(fub) == list(hu)


@pytest.mark.parametrize("seed", range(200))
def test_single_temporal_row_equals_projection_hull(seed):
    """x + d <= y ([[x + y <= c]] of Sec. 2 with y negated): exact hull,
    including x == y (fails iff d > 0)."""
    g = SplitMix64.derive(seed, 12)
    lb = [g.uniform_int(-6, 6) for _ in range(2)]
    ub = [l + g.uniform_int(0, 8) for l in lb]
    x = g.uniform_int(0, 1)
    y = g.uniform_int(0, 1)
    d = g.uniform_int(-4, 6)
    m = oracle.Model(lb, ub, temporal=[(x, y, d)])
    st, flb, fub, _ = oracle.propagate(m, lb, ub)
    sols = brute.generic_solutions([(x, y, d)], [], [], lb, ub)
    if not sols:
        assert st == oracle.FAILED
    else:
        assert st == oracle.FIXPOINT
        hl, hu = hull(sols, 2)
        assert list(flb) == list(hl) and list(fub) == list(hu)


@pytest.mark.parametrize("seed", range(400))
def test_single_reified_row_sound_and_decides_fixed_inputs(seed):
    """b <=> (x <= y and y < x + d): the four asks of [[phi <=> psi]] (Sec. 2)
    never remove a solution; with x, y fixed they decide b exactly; with all
    three fixed they fail iff the point is not a solution; and b is fixed to
    1 exactly when every point of the (x, y) box satisfies both conjuncts."""
    g = SplitMix64.derive(seed, 13)
    lb = [g.uniform_int(-4, 4), g.uniform_int(-4, 4), 0]
    ub = [lb[0] + g.uniform_int(0, 5), lb[1] + g.uniform_int(0, 5), 1]
    mode = g.uniform_int(0, 3)
    if mode == 1:  # fix b
        v = g.uniform_int(0, 1)
        lb[2] = ub[2] = v
    if mode == 2:  # fix x, y
        ub[0] = lb[0]
        ub[1] = lb[1]
    if mode == 3:  # fix all
        ub[0] = lb[0]
        ub[1] = lb[1]
        lb[2] = ub[2] = g.uniform_int(0, 1)
    d = g.uniform_int(1, 5)
    row = (2, 0, 1, d)
    m = oracle.Model([-20, -20, 0], [20, 20, 1], reified=[row])
    st, flb, fub, _ = oracle.propagate(m, lb, ub)
    sols = brute.generic_solutions([], [], [row], lb, ub)
    if st == oracle.FAILED:
        assert not sols
    else:
        for s in sols:
            assert all(flb[i] <= s[i] <= fub[i] for i in range(3))
    if mode in (2, 3):
        assert (st == oracle.FIXPOINT) == bool(sols)
        if sols:
            assert flb[2] == fub[2] == sols[0][2]
    if mode == 1 and st == oracle.FIXPOINT:
        ent_A = ub[0] <= lb[1]
        ent_B = ub[1] <= lb[0] + d - 1
        if lb[2] == 1 or ent_A or ent_B:
            # b fixed true gives x <= y <= x + d - 1; b fixed false with one
            # conjunct entailed gives the other's negation: difference
            # constraints, on which bounds propagation reaches the exact hull
            hl, hu = hull(sols, 3)
            assert list(flb) == list(hl) and list(fub) == list(hu)
        else:
            # b false and neither conjunct entailed: no command may fire
            assert list(flb) == lb and list(fub) == ub
    if mode == 1 and st == oracle.FAILED:
        assert not sols
    if mode == 0:
        all_true = all((x <= y and y < x + d)
                       for x in range(lb[0], ub[0] + 1) for y in range(lb[1], ub[1] + 1))
        assert (flb[2] == 1) == all_true


# ------------------------------------------------ Theorem 1 / Prop. 2 / Def. 4

def _generic_cases(count, base):
    for seed in range(count):
        gm = draw_generic_model(base + seed)
        m = oracle.Model(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified,
                         gm.objective, gm.branch)
        lb, ub = draw_generic_store(gm, base + seed)
        yield m, lb, ub


def _rcpsp_cases(count):
    for seed in range(count):
        inst = draw_rcpsp(RcpspDistribution(6, 9, 2, (1, 5), (0, 4), (4, 7), 0.25), seed)
        m = rcpsp_model(inst)
        g = SplitMix64.derive(seed, 14)
        dec = []
        for t in range(inst.n):
            if g.bernoulli(0.4):
                lo = g.uniform_int(0, inst.horizon)
                hi = g.uniform_int(lo, inst.horizon)
                dec.append((t, lo, hi))
        lb, ub = node_store(m, dec)
        yield m, lb, ub


def _all_cases():
    return list(_generic_cases(150, 1000)) + list(_rcpsp_cases(60))


def test_every_fair_order_reaches_the_same_fixed_point():
    """Sequential forward, reverse, Jacobi (parallel composition of Sec. 3)
    and random fair orders all reach the same fixed point or all fail
    (Prop. 2 and the fix D = fix O theorem)."""
    n_failed = n_fix = 0
    for m, lb, ub in _all_cases():
        ref = oracle.propagate(m, lb, ub, oracle.FORWARD)
        others = [oracle.propagate(m, lb, ub, oracle.REVERSE),
                  oracle.propagate(m, lb, ub, oracle.JACOBI)]
        others += [oracle.propagate(m, lb, ub, oracle.RANDOM, seed=s) for s in range(12)]
        for o in others:
            assert o[0] == ref[0]
            if ref[0] == oracle.FIXPOINT:
                assert np.array_equal(o[1], ref[1]) and np.array_equal(o[2], ref[2])
        n_failed += ref[0] == oracle.FAILED
        n_fix += ref[0] == oracle.FIXPOINT
    assert n_failed > 10 and n_fix > 10  # both outcomes exercised


def test_sequential_sweeps_never_need_more_than_jacobi():
    """A sequential pass is at least as strong as a parallel (Jacobi) pass
    (remark after Prop. 2), so it never needs more sweeps."""
    for m, lb, ub in _all_cases():
        f = oracle.propagate(m, lb, ub, oracle.FORWARD)
        j = oracle.propagate(m, lb, ub, oracle.JACOBI)
        if f[0] == oracle.FIXPOINT:
            assert f[3] <= j[3]


def test_fixed_point_is_a_closure():
    """fix D(P) is extensive, idempotent and monotone (Theorem 1), and every
    guarded command is stable on it."""
    for k, (m, lb, ub) in enumerate(_all_cases()):
        st, flb, fub, _ = oracle.propagate(m, lb, ub)
        if st != oracle.FIXPOINT:
            continue
        lbj = np.maximum(np.asarray(lb), m.lb0)
        ubj = np.minimum(np.asarray(ub), m.ub0)
        assert np.all(flb >= lbj) and np.all(fub <= ubj)  # extensive
        st2, lb2, ub2, sw2 = oracle.propagate(m, flb, fub)
        assert st2 == oracle.FIXPOINT and sw2 == 1  # idempotent
        assert np.array_equal(lb2, flb) and np.array_equal(ub2, fub)
        for gidx in range(m.command_count()):  # every command stable
            kind, var, val = oracle.command(m, flb, fub, gidx)
            if kind == oracle.TELL_LB:
                assert val <= flb[var]
            elif kind == oracle.TELL_UB:
                assert val >= fub[var]
        # monotone: a narrower input never gives a wider result
        g = SplitMix64.derive(k, 15)
        lbn, ubn = np.array(lbj), np.array(ubj)
        for v in range(m.n_vars):
            if g.bernoulli(0.3) and ubn[v] > lbn[v]:
                if g.bernoulli(0.5):
                    lbn[v] += 1
                else:
                    ubn[v] -= 1
        st3, lb3, ub3, _ = oracle.propagate(m, lbn, ubn)
        if st3 == oracle.FIXPOINT:
            assert np.all(lb3 >= flb) and np.all(ub3 <= fub)


def test_commands_are_monotone():
    """Lemma 1: every guarded command is a monotone function of the store:
    on s <= s' (s' narrower), the tell from s' is at least the tell from s
    whenever s's guard holds."""
    for k, (m, lb, ub) in enumerate(list(_generic_cases(60, 5000))):
        lbj = np.maximum(np.asarray(lb), m.lb0)
        ubj = np.minimum(np.asarray(ub), m.ub0)
        g = SplitMix64.derive(k, 16)
        lbn, ubn = lbj.copy(), ubj.copy()
        for v in range(m.n_vars):
            if ubn[v] > lbn[v] and g.bernoulli(0.5):
                lbn[v] = g.uniform_int(int(lbn[v]), int(ubn[v]))
            if ubn[v] > lbn[v] and g.bernoulli(0.5):
                ubn[v] = g.uniform_int(int(lbn[v]), int(ubn[v]))
        for gidx in range(m.command_count()):
            k1, v1, x1 = oracle.command(m, lbj, ubj, gidx)
            k2, v2, x2 = oracle.command(m, lbn, ubn, gidx)
            if k1 == oracle.TELL_NONE:
                continue
            assert k2 == k1 and v2 == v1
            if k1 == oracle.TELL_LB:
                assert x2 >= x1
            else:
                assert x2 <= x1


# ------------------------------------------------------------------ RCPSP

def _tiny_instances(count, n_lo=3, n_hi=5):
    dist = RcpspDistribution(n_lo, n_hi, 2, (1, 3), (0, 3), (3, 4), 0.3)
    return [draw_rcpsp(dist, 777 + s) for s in range(count)]


def test_rcpsp_fixed_starts_fail_iff_infeasible():
    """With every start fixed, the decomposition (Sec. 2) fails exactly on
    infeasible schedules: checked against the resource profile at every
    instant."""
    checked = feasible = 0
    for inst in _tiny_instances(40):
        m = rcpsp_model(inst)
        g = SplitMix64.derive(inst.seed, 17)
        for _ in range(25):
            s = [g.uniform_int(0, inst.horizon - inst.durations[i]) for i in range(inst.n)]
            dec = [(i, s[i], s[i]) for i in range(inst.n)]
            lb, ub = node_store(m, dec)
            st = oracle.propagate(m, lb, ub)[0]
            ok = brute.rcpsp_feasible(inst, s)
            assert (st == oracle.FIXPOINT) == ok
            checked += 1
            feasible += ok
    assert feasible > 20 and checked - feasible > 20


def test_rcpsp_optimum_and_solution_counts_match_enumeration():
    """Optimum = smallest makespan among all enumerated feasible schedules;
    count-all under makespan <= opt = number of such schedules; and every
    enumerated optimal schedule lies in the root fixed point."""
    for inst in _tiny_instances(25):
        m = rcpsp_model(inst)
        r = oracle.solve(m, oracle.OPTIMISE, oracle.INPUT_ORDER)
        sols_h = brute.rcpsp_enumerate(inst, inst.horizon)
        assert len(sols_h) > 0  # serial schedule always fits in h
        mk = (sols_h + np.asarray(inst.durations)[None, :]).max(axis=1)
        opt = int(mk.min())
        assert r["status"] == oracle.RES_OPTIMAL and r["objective"] == opt
        assert brute.rcpsp_feasible(inst, list(r["witness"][: inst.n]))
        c = oracle.solve(m, oracle.COUNT_ALL, oracle.INPUT_ORDER, obj_ub=opt)
        assert c["solutions"] == int((mk <= opt).sum())
        # first-fail finds the same optimum
        f = oracle.solve(m, oracle.OPTIMISE, oracle.FIRST_FAIL)
        assert f["objective"] == opt
        # soundness of the root fixed point w.r.t. all schedules within h
        st, flb, fub, _ = oracle.propagate(m, *m.root())
        assert st == oracle.FIXPOINT
        assert np.all(sols_h >= flb[: inst.n]) and np.all(sols_h <= fub[: inst.n])


def test_rcpsp_count_all_nodes_formula():
    """Reading of a node: every propagated store.  With no limit each
    branching adds two children, so nodes = 1 + 2 * (nodes - leaves)."""
    for inst in _tiny_instances(10):
        m = rcpsp_model(inst)
        c = oracle.solve(m, oracle.COUNT_ALL, oracle.INPUT_ORDER)
        leaves = c["fails"] + c["solutions"]
        branchings = c["nodes"] - leaves
        assert c["nodes"] == 1 + 2 * branchings


def test_precedence_only_root_is_critical_path():
    """Closed form: with no resource use, the root fixed point is the critical
    path method's earliest and latest starts (longest paths in the DAG)."""
    for s in range(40):
        inst = draw_rcpsp(RcpspDistribution(5, 14, 1, (1, 9), (0, 0), (5, 5), 0.3), 4000 + s)
        m = rcpsp_model(inst)
        st, flb, fub, _ = oracle.propagate(m, *m.root())
        assert st == oracle.FIXPOINT
        es, ls = brute.cpm_bounds(inst, inst.horizon)
        assert list(flb[: inst.n]) == es and list(fub[: inst.n]) == ls
        assert flb[var_M(inst.n)] == max(e + d for e, d in zip(es, inst.durations))
        # and the optimum (no resources) is the critical path length
        r = oracle.solve(m)
        assert r["objective"] == flb[var_M(inst.n)]


def test_tiny8_optima_match_stored_sgs_brute_force():
    """The 8-task family's optima against brute-force serial-SGS values
    stored by tests/golden/make_tiny8_optima.py (which calls oracle.brute)."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny8_sgs_optima.json")
    gold = json.load(open(path))
    assert len(gold["optima"]) == 100
    for seed in range(0, 100, 4):
        inst = config_instance("tiny8", seed)
        r = oracle.solve(rcpsp_model(inst))
        assert r["status"] == oracle.RES_OPTIMAL
        assert r["objective"] == gold["optima"][seed]
        assert brute.rcpsp_feasible(inst, list(r["witness"][: inst.n]))


def test_tiny8_sgs_recomputed_live():
    for seed in (1, 2):
        import json, os
        gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                           "tiny8_sgs_optima.json")))
        assert brute.rcpsp_optimum_sgs(config_instance("tiny8", seed)) == gold["optima"][seed]
