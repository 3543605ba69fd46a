"""Random search-tree nodes over an RCPSP instance.

A node is a list of bound restrictions on start variables s_i (the variables
a search branches on).  Each restriction is (task, lo, hi): the node's store
is the root store with s_task's interval intersected with [lo, hi].  Tasks are
restricted in input order (lowest index first, moving on once a task's
interval is a single value), each restriction keeps a random side of a random
cut of the current interval.  No propagation is involved: the restrictions
are drawn on the unpropagated intervals.
"""
from typing import List, Tuple

from .rng import SplitMix64


def draw_partial_assignments(n_tasks: int, horizon: int, count: int, seed: int,
                             max_decisions: int = 15) -> List[List[Tuple[int, int, int]]]:
    g = SplitMix64.derive(seed, 0xD0DE5)
    nodes = []
    for _ in range(count):
        k = g.uniform_int(0, max_decisions)
        lo = [0] * n_tasks
        hi = [horizon] * n_tasks
        task = 0
        dec = []
        for _ in range(k):
            while task < n_tasks and lo[task] == hi[task]:
                task += 1
            if task >= n_tasks:
                break
            cut = g.uniform_int(lo[task], hi[task] - 1)
            if g.bernoulli(0.5):
                hi[task] = cut
            else:
                lo[task] = cut + 1
            dec.append((task, lo[task], hi[task]))
        nodes.append(dec)
    return nodes
