"""Seeded resource-constrained project scheduling (RCPSP) instances.

An instance is the tuple <T, P, R> of the paper's scheduling example (Sec. 2):
task durations d_i, resource usages r_{k,i}, capacities c_k and a precedence
DAG given as edges (i, j) meaning task i ends before task j starts.  Edges
only go from a lower to a higher task index, so the DAG is acyclic.

The distributions mirror the shape of PSPLIB j30 (30 tasks, 4 resources), the
data set the paper evaluates on; that data set itself is not reproduced.
"""
from dataclasses import dataclass
from typing import List, Tuple

from .rng import SplitMix64


@dataclass(frozen=True)
class RcpspInstance:
    n: int                              # tasks
    durations: Tuple[int, ...]          # d_i >= 1
    usage: Tuple[Tuple[int, ...], ...]  # usage[k][i] = r_{k,i} >= 0
    capacity: Tuple[int, ...]           # c_k
    precedences: Tuple[Tuple[int, int], ...]  # (i, j): i << j
    seed: int = 0
    name: str = ""

    @property
    def n_resources(self) -> int:
        return len(self.capacity)

    @property
    def horizon(self) -> int:
        """h = sum of durations (the horizon the paper suggests)."""
        return int(sum(self.durations))


@dataclass(frozen=True)
class RcpspDistribution:
    n_lo: int
    n_hi: int
    n_resources: int
    dur: Tuple[int, int]
    usage: Tuple[int, int]
    cap: Tuple[int, int]
    edge_p: float


# Instance families (all ranges inclusive).
CONFIGS = {
    # tiny plain solve: 8 tasks, 1 resource of capacity 4
    "tiny8": RcpspDistribution(8, 8, 1, (1, 5), (1, 3), (4, 4), 0.2),
    # propagation batch model: 30 tasks, 4 resources (j30 shape)
    "j30": RcpspDistribution(30, 30, 4, (1, 10), (0, 5), (5, 10), 0.1),
    # uneven batched solves: 30-60 tasks, same distributions
    "mixed30_60": RcpspDistribution(30, 60, 4, (1, 10), (0, 5), (5, 10), 0.1),
    # uneven batched complete solves: 6-10 tasks, same distributions (the
    # largest sizes whose first-fail proofs all end within a few hundred
    # thousand nodes of the plain sequential search)
    "mixed6_10": RcpspDistribution(6, 10, 4, (1, 10), (0, 5), (5, 10), 0.1),
    # learned-branching family: 60 tasks
    "j60": RcpspDistribution(60, 60, 4, (1, 10), (0, 5), (5, 10), 0.1),
    # large family: 120 tasks
    "j120": RcpspDistribution(120, 120, 4, (1, 10), (0, 5), (5, 10), 0.1),
}


def draw_rcpsp(dist: RcpspDistribution, seed: int, name: str = "") -> RcpspInstance:
    g = SplitMix64.derive(seed, 0x5C4ED)
    n = g.uniform_int(dist.n_lo, dist.n_hi)
    R = dist.n_resources
    durations = tuple(g.uniform_int(*dist.dur) for _ in range(n))
    capacity = tuple(g.uniform_int(*dist.cap) for _ in range(R))
    usage = []
    for k in range(R):
        # a task never needs more than a resource's capacity on its own
        hi = min(dist.usage[1], capacity[k])
        usage.append(tuple(g.uniform_int(dist.usage[0], hi) for _ in range(n)))
    prec: List[Tuple[int, int]] = []
    for i in range(n):
        for j in range(i + 1, n):
            if g.bernoulli(dist.edge_p):
                prec.append((i, j))
    return RcpspInstance(n, durations, tuple(usage), capacity, tuple(prec), seed, name)


def config_instance(family: str, seed: int) -> RcpspInstance:
    return draw_rcpsp(CONFIGS[family], seed, f"{family}/{seed}")
