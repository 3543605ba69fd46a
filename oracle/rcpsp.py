"""The oracle's own expansion of an RCPSP instance into constraints.

Follows the PCCP model of the scheduling problem in Sec. 2 of the paper:
  s_i in [0, h]  (h = sum of durations),  b_{i,j} in [0, 1],
  s_i + d_i <= s_j for every precedence i << j,
  b_{i,j} <=> (s_i <= s_j and s_j < s_i + d_i)  for every ordered pair,
  sum_i r_{k,i} * b_{i,j} <= c_k  for every resource k and task j.
Readings where the paper is silent:
  - b_{j,j}: x - x arithmetic on intervals cannot entail s_j <= s_j, so the
    diagonal Boolean is created fixed to 1 (true for d_j >= 1) with no reified
    constraint; it keeps its slot in the n x n block.
  - objective: a makespan variable M in [0, h] with s_i + d_i <= M for every
    task; minimise M; branch on the start variables in index order.
Variable layout: s_i at i, b_{i,j} at n + i*n + j, M at n + n*n.
"""
from . import Model


def var_s(n, i):
    return i


def var_b(n, i, j):
    return n + i * n + j


def var_M(n):
    return n + n * n


def rcpsp_model(inst, horizon=None) -> Model:
    n = inst.n
    h = inst.horizon if horizon is None else horizon
    nv = n + n * n + 1
    lb0 = [0] * nv
    ub0 = [0] * nv
    for i in range(n):
        ub0[var_s(n, i)] = h
    for i in range(n):
        for j in range(n):
            lb0[var_b(n, i, j)] = 1 if i == j else 0
            ub0[var_b(n, i, j)] = 1
    ub0[var_M(n)] = h
    temporal = [(var_s(n, i), var_s(n, j), inst.durations[i]) for (i, j) in inst.precedences]
    temporal += [(var_s(n, i), var_M(n), inst.durations[i]) for i in range(n)]
    reified = []
    for j in range(n):
        for i in range(n):
            if i != j:
                reified.append((var_b(n, i, j), var_s(n, i), var_s(n, j), inst.durations[i]))
    linear = []
    for k in range(inst.n_resources):
        for j in range(n):
            terms = [(inst.usage[k][i], var_b(n, i, j)) for i in range(n) if inst.usage[k][i] != 0]
            linear.append((inst.capacity[k], terms))
    return Model(lb0, ub0, temporal, linear, reified, objective=var_M(n),
                 branch=[var_s(n, i) for i in range(n)])


def node_store(model: Model, decisions):
    """Root store with each (task, lo, hi) restriction intersected in."""
    lb, ub = model.root()
    for (t, lo, hi) in decisions:
        lb[t] = max(lb[t], lo)
        ub[t] = min(ub[t], hi)
    return lb, ub
