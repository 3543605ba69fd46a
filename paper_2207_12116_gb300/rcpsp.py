"""Scheduling model builder: an RCPSP instance <T, P, R> -> pccp_model_desc rows.

The PCCP model of Sec. 2 of the paper:
  s_i in [0, h] (h = sum of durations)         start of task i
  b_{i,j} in [0, 1]                            task i runs when task j starts
  s_i + d_i <= s_j            for i << j        temporal rows
  b_{i,j} <=> (s_i <= s_j and s_j < s_i + d_i)  reified rows, i != j
  sum_i r_{k,i} * b_{i,j} <= c_k                linear rows, per resource k, task j
Where the paper is silent: b_{j,j} is fixed to 1 with no reified row (interval
arithmetic cannot entail s_j <= s_j, and d_j >= 1 makes it true); the
objective is a makespan variable M in [0, h] with s_i + d_i <= M, minimised;
search branches on s_0 .. s_{n-1} in index order.
Variable layout: s_i at i, b_{i,j} at n + i*n + j, M at n + n*n.
"""
import numpy as np


def layout(n):
    return {"s": 0, "b": n, "M": n + n * n, "n_vars": n + n * n + 1}


def build_rows(inst):
    """Row arrays for one instance (all int32 numpy arrays)."""
    n = inst.n
    d = list(inst.durations)
    h = int(sum(d))
    nv = n + n * n + 1
    M = n + n * n
    lb0 = np.zeros(nv, dtype=np.int32)
    ub0 = np.zeros(nv, dtype=np.int32)
    ub0[:n] = h
    bidx = n + np.arange(n * n)
    ub0[bidx] = 1
    diag = n + np.arange(n) * n + np.arange(n)
    lb0[diag] = 1
    ub0[M] = h
    temporal = [(i, j, d[i]) for (i, j) in inst.precedences] + [(i, M, d[i]) for i in range(n)]
    reified = [(n + i * n + j, i, j, d[i]) for j in range(n) for i in range(n) if i != j]
    lin_c, lin_off, coef, var = [], [0], [], []
    for k in range(len(inst.capacity)):
        for j in range(n):
            for i in range(n):
                r = inst.usage[k][i]
                if r:
                    coef.append(r)
                    var.append(n + i * n + j)
            lin_c.append(inst.capacity[k])
            lin_off.append(len(coef))
    a32 = lambda x, shape=None: np.ascontiguousarray(np.asarray(x, dtype=np.int32).reshape(shape if shape else -1))
    return {
        "lb0": lb0, "ub0": ub0,
        "temporal": a32(temporal, (-1, 3)) if temporal else np.zeros((0, 3), np.int32),
        "reified": a32(reified, (-1, 4)) if reified else np.zeros((0, 4), np.int32),
        "linear_c": a32(lin_c), "linear_off": a32(lin_off),
        "term_coef": a32(coef), "term_var": a32(var),
        "objective": M, "branch": a32(list(range(n))),
    }


def root_store(rows):
    return rows["lb0"].copy(), rows["ub0"].copy()


def node_stores(rows, nodes):
    """Stores (lb, ub) [len(nodes), n_vars] for search nodes given as lists of
    (task, lo, hi) restrictions of the start variables."""
    nv = len(rows["lb0"])
    lb = np.tile(rows["lb0"], (len(nodes), 1))
    ub = np.tile(rows["ub0"], (len(nodes), 1))
    for r, dec in enumerate(nodes):
        for (t, lo, hi) in dec:
            lb[r, t] = max(lb[r, t], lo)
            ub[r, t] = min(ub[r, t], hi)
    return np.ascontiguousarray(lb, dtype=np.int32), np.ascontiguousarray(ub, dtype=np.int32)
