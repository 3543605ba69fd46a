"""Random generic constraint models (not RCPSP) for property tests.

A generic model is plain data: variable domains, temporal rows (x, y, d)
meaning x + d <= y, linear rows (c, [(coef, var)...]) meaning
sum coef*var <= c, reified rows (b, x, y, d) meaning b <=> (x <= y and
y < x + d), an objective variable and branching variables.
"""
from dataclasses import dataclass
from typing import List, Tuple

from .rng import SplitMix64


@dataclass
class GenericModel:
    lb0: List[int]
    ub0: List[int]
    temporal: List[Tuple[int, int, int]]
    linear: List[Tuple[int, List[Tuple[int, int]]]]
    reified: List[Tuple[int, int, int, int]]
    objective: int
    branch: List[int]

    @property
    def n_vars(self) -> int:
        return len(self.lb0)


def draw_generic_model(seed: int, n_int: int = 6, n_bool: int = 4, dom: int = 12,
                       n_temporal: int = 5, n_linear: int = 3, n_reified: int = 4,
                       max_len: int = 4, coef: int = 4, allow_negative: bool = True) -> GenericModel:
    g = SplitMix64.derive(seed, 0x6E0E7)
    nv = n_int + n_bool
    lb0, ub0 = [], []
    for _ in range(n_int):
        a = g.uniform_int(-dom, dom // 2)
        lb0.append(a)
        ub0.append(a + g.uniform_int(0, 2 * dom))
    for _ in range(n_bool):
        lb0.append(0)
        ub0.append(1)
    temporal = []
    for _ in range(n_temporal):
        x = g.uniform_int(0, n_int - 1)
        y = g.uniform_int(0, n_int - 1)
        if n_int > 1 and g.uniform_int(0, 7) != 0:  # mostly distinct variables
            while y == x:
                y = g.uniform_int(0, n_int - 1)
        if x > y and g.uniform_int(0, 3) != 0:  # mostly lower -> higher index
            x, y = y, x
        d = g.uniform_int(-4 if allow_negative else 0, 4)
        if x > y and allow_negative:  # backward rows mostly slack: feasible cycles
            d = -g.uniform_int(0, 2 * dom)
        if x == y:  # x + d <= x holds iff d <= 0; keep the degenerate row satisfiable
            d = -g.uniform_int(0, 3)
        temporal.append((x, y, d))
    linear = []
    for _ in range(n_linear):
        ln = g.uniform_int(1, max_len)
        vs = []
        for _ in range(ln):
            v = g.uniform_int(0, nv - 1)
            a = g.uniform_int(-coef if allow_negative else 1, coef)
            if a == 0:
                a = 1
            vs.append((a, v))
        c = g.uniform_int(-dom, 3 * dom * coef)
        linear.append((c, vs))
    reified = []
    for _ in range(n_reified if n_bool > 0 else 0):
        b = n_int + g.uniform_int(0, n_bool - 1)
        x = g.uniform_int(0, n_int - 1)
        y = g.uniform_int(0, n_int - 1)
        d = g.uniform_int(1, 6)
        reified.append((b, x, y, d))
    return GenericModel(lb0, ub0, temporal, linear, reified, objective=0,
                        branch=list(range(n_int)))


def draw_generic_store(model: GenericModel, seed: int, p_narrow: float = 0.3):
    """A random store inside the model's domains (each bound narrowed with
    probability p_narrow); may be empty nowhere."""
    g = SplitMix64.derive(seed, 0x570E)
    lb, ub = [], []
    for l0, u0 in zip(model.lb0, model.ub0):
        lo, hi = l0, u0
        if g.bernoulli(p_narrow) and hi > lo:
            lo = g.uniform_int(lo, hi)
        if g.bernoulli(p_narrow) and hi > lo:
            hi = g.uniform_int(lo, hi)
        lb.append(lo)
        ub.append(hi)
    return lb, ub
