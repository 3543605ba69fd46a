"""Brute-force enumerators -- TEST INFRASTRUCTURE (pins for the oracle).

Nothing here propagates: every function enumerates candidate assignments and
checks the constraints' plain meaning, so it can pin the propagation-based
oracle against something other than itself.

  rcpsp_feasible      : precedences and the resource profile at every instant
  rcpsp_enumerate     : all feasible integer start vectors with makespan <= K
  rcpsp_optimum_sgs   : minimum makespan over the serial schedule generation
                        scheme applied to every precedence-feasible task list
                        (the active schedules contain an optimal one; Kolisch,
                        EJOR 90(2), 1996)
  cpm_bounds          : earliest / latest starts of a precedence-only model
                        (longest paths in the DAG, the critical path method)
  generic_solutions   : all integer points of a small box that satisfy every
                        row of a generic model
"""
import itertools

import numpy as np


def rcpsp_feasible(inst, s) -> bool:
    n = inst.n
    d = inst.durations
    if any(si < 0 for si in s):
        return False
    for (i, j) in inst.precedences:
        if s[i] + d[i] > s[j]:
            return False
    end = max(s[i] + d[i] for i in range(n)) if n else 0
    for k in range(inst.n_resources):
        for t in range(end):
            use = sum(inst.usage[k][i] for i in range(n) if s[i] <= t < s[i] + d[i])
            if use > inst.capacity[k]:
                return False
    return True


def rcpsp_enumerate(inst, K: int, max_points: int = 20_000_000):
    """All feasible start vectors s (s_i >= 0) with max_i s_i + d_i <= K, as an
    int64 array [count, n].  Vectorised over the full product of ranges."""
    n = inst.n
    d = np.asarray(inst.durations, dtype=np.int64)
    ranges = [np.arange(0, K - d[i] + 1, dtype=np.int64) for i in range(n)]
    if any(len(r) == 0 for r in ranges):
        return np.zeros((0, n), dtype=np.int64)
    total = 1
    for r in ranges:
        total *= len(r)
    if total > max_points:
        raise ValueError(f"brute force too large: {total}")
    grids = np.meshgrid(*ranges, indexing="ij")
    S = np.stack([g.reshape(-1) for g in grids], axis=1)
    ok = np.ones(len(S), dtype=bool)
    for (i, j) in inst.precedences:
        ok &= S[:, i] + d[i] <= S[:, j]
    S = S[ok]
    if len(S) == 0:
        return S
    for k in range(inst.n_resources):
        r = np.asarray(inst.usage[k], dtype=np.int64)
        for t in range(K):
            running = (S <= t) & (t < S + d[None, :])
            use = running.astype(np.int64) @ r
            S = S[use <= inst.capacity[k]]
            if len(S) == 0:
                return S
    return S


def rcpsp_optimum_sgs(inst) -> int:
    """Minimum makespan over serial-SGS schedules of all precedence-feasible
    task lists (depth-first over lists, sharing scheduled prefixes)."""
    n = inst.n
    d = inst.durations
    h = inst.horizon + max(d) + 1
    preds = [[] for _ in range(n)]
    for (i, j) in inst.precedences:
        preds[j].append(i)
    R = inst.n_resources
    best = [inst.horizon]

    def rec(done, start, prof, makespan):
        if makespan >= best[0] and len(done) < n:
            # lists extending this prefix can only end later or equal
            return
        if len(done) == n:
            best[0] = min(best[0], makespan)
            return
        for t in range(n):
            if t in done or any(p not in done for p in preds[t]):
                continue
            es = max([start[p] + d[p] for p in preds[t]], default=0)
            st = es
            while True:
                if all(prof[k][tau] + inst.usage[k][t] <= inst.capacity[k]
                       for k in range(R) for tau in range(st, st + d[t])):
                    break
                st += 1
            newprof = [list(p) for p in prof]
            for k in range(R):
                for tau in range(st, st + d[t]):
                    newprof[k][tau] += inst.usage[k][t]
            start2 = dict(start)
            start2[t] = st
            rec(done | {t}, start2, newprof, max(makespan, st + d[t]))

    rec(frozenset(), {}, [[0] * h for _ in range(R)], 0)
    return best[0]


def cpm_bounds(inst, horizon_M: int):
    """Earliest starts (longest path from the sources) and latest starts
    (horizon_M minus the longest path to the end, inclusive of own duration)
    for the precedence DAG; edges go from lower to higher index."""
    n = inst.n
    d = inst.durations
    es = [0] * n
    for j in range(n):  # indices are a topological order
        for (i, jj) in inst.precedences:
            if jj == j:
                es[j] = max(es[j], es[i] + d[i])
    tail = [d[i] for i in range(n)]  # longest path from start of i to the end
    for i in reversed(range(n)):
        for (ii, j) in inst.precedences:
            if ii == i:
                tail[i] = max(tail[i], d[i] + tail[j])
    ls = [horizon_M - tail[i] for i in range(n)]
    return es, ls


def generic_satisfied(temporal, linear, reified, x) -> bool:
    for (a, b, dd) in temporal:
        if not (x[a] + dd <= x[b]):
            return False
    for (c, terms) in linear:
        if sum(coef * x[v] for (coef, v) in terms) > c:
            return False
    for (b, a, y, dd) in reified:
        holds = (x[a] <= x[y]) and (x[y] < x[a] + dd)
        if x[b] not in (0, 1) or (x[b] == 1) != holds:
            return False
    return True


def generic_solutions(temporal, linear, reified, lb, ub, max_points: int = 2_000_000):
    """All integer points of [lb, ub] satisfying every row, as a list of tuples."""
    sizes = [max(0, u - l + 1) for l, u in zip(lb, ub)]
    total = 1
    for s in sizes:
        total *= s
    if total > max_points:
        raise ValueError(f"box too large: {total}")
    if total == 0:
        return []
    out = []
    for x in itertools.product(*[range(l, u + 1) for l, u in zip(lb, ub)]):
        if generic_satisfied(temporal, linear, reified, x):
            out.append(x)
    return out
