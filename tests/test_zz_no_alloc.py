"""The allocation-free batched solve (pccp_solve_batch_noalloc).

Callers that may not allocate device memory use this entry point: hosts that
reserve all their memory at start-up and allocate nothing after a
no-allocation point, and plug-ins whose application owns the device
allocator.  Its scratch is a fixed array inside the library.  It must give
exactly the results of pccp_solve_batch, call after call, although every call
reuses the same scratch, and it must leave device memory as it found it.
This file is collected last so that a stop-at-first-failure run has already
run every other test."""
import ctypes

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


def test_noalloc_global_tables_and_learned_strategy():
    """Tables too large for shared memory (read from global memory, with the
    same default team size as pccp_solve_batch) and the learned strategy."""
    big = [pccp.Model.from_rcpsp(config_instance("j120", s)) for s in range(3)]
    for a, b in zip(pccp.solve_batch(big, node_limit=12),
                    pccp.solve_batch(big, node_limit=12, noalloc=True)):
        _same(a, b)
    pol = pccp.Policy.random(3)
    small = [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(12)]
    kw = {"strategy": pccp.PCCP_LEARNED, "policy": pol}
    for a, b in zip(pccp.solve_batch(small, **kw), pccp.solve_batch(small, noalloc=True, **kw)):
        _same(a, b)


def test_noalloc_rejects_requests_beyond_its_scratch():
    m = pccp.Model.from_rcpsp(config_instance("tiny8", 0))
    per_model = 40 + 64 + 4 * m.n_vars
    n = (8 << 20) // per_model + 16
    with pytest.raises(pccp.PccpError) as e:
        pccp.solve_batch([m] * n, noalloc=True)
    assert e.value.code == pccp.PCCP_ERR_SCRATCH


def _pool_used_high():
    """High-water mark of the current device's default stream-ordered memory
    pool (driver API), or None when the driver library cannot be reached."""
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    dev = ctypes.c_int(0)
    pool = ctypes.c_void_p()
    val = ctypes.c_uint64(0)
    used_mem_high = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH
    if cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) != 0:
        return None
    if cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) != 0:
        return None
    if cu.cuMemPoolGetAttribute(pool, used_mem_high, ctypes.byref(val)) != 0:
        return None
    return cu, pool, val.value


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which loads the module and reserves the scratch),
    repeated calls change neither the device's free memory, nor torch's
    allocations, nor the stream-ordered pool's high-water mark (reset to its
    current use before the calls)."""
    models = [pccp.Model.from_rcpsp(config_instance("mixed30_60", s)) for s in range(6)] + \
             [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(20)]
    pccp.solve_batch(models, node_limit=100, noalloc=True)
    torch.cuda.synchronize()
    pool = _pool_used_high()
    if pool is not None:
        cu, handle, _ = pool
        zero = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(handle, 8, ctypes.byref(zero)) == 0
        high0 = _pool_used_high()[2]
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for k in range(5):
        pccp.solve_batch(models, node_limit=100 + 50 * k, noalloc=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    if pool is not None:
        assert _pool_used_high()[2] == high0
