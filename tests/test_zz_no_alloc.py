"""The allocation-free batched solve (pccp_solve_batch_noalloc).

Callers that may not allocate device memory (hosts that reserve all memory at
start-up, plug-ins whose application owns the allocator, work issued during
stream capture) use this entry point; its scratch is a fixed array inside the
library.  It must give exactly the results of pccp_solve_batch, call after
call, although every call reuses the same scratch.  This file is collected
last so that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

import paper_2207_12116_gb300 as pccp
from synthetic import config_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same(a, b):
    # every deterministic output; fixed-point iteration counts depend on the
    # interleaving of the lock-free loop and are not compared
    keys = ("status", "has_solution", "objective", "nodes", "fails", "solutions", "max_depth")
    for k in keys:
        assert a[k] == b[k], (k, a[k], b[k])
    if a["has_solution"]:
        assert np.array_equal(a["witness"], b["witness"])


def test_noalloc_matches_batch_on_two_calls_in_a_row():
    first = [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(40)]
    second = [pccp.Model.from_rcpsp(config_instance("mixed30_60", s)) for s in range(10)] + \
             [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(40, 60)]
    for models, kw in ((first, {}), (second, {"node_limit": 300})):
        ref = pccp.solve_batch(models, **kw)
        got = pccp.solve_batch(models, noalloc=True, **kw)
        assert len(ref) == len(got)
        for a, b in zip(ref, got):
            _same(a, b)
    # and the first request again, after the scratch held the second one
    again = pccp.solve_batch(first, noalloc=True)
    for a, b in zip(pccp.solve_batch(first), again):
        _same(a, b)


def test_noalloc_rejects_requests_beyond_its_scratch():
    m = pccp.Model.from_rcpsp(config_instance("tiny8", 0))
    per_model = 40 + 64 + 4 * m.n_vars
    n = (8 << 20) // per_model + 16
    with pytest.raises(pccp.PccpError) as e:
        pccp.solve_batch([m] * n, noalloc=True)
    assert e.value.code == pccp.PCCP_ERR_SCRATCH
