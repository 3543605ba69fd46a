"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle


def oracle_model_from_lists(gm):
    return oracle.Model(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified, gm.objective, gm.branch)


def oracle_batch(om, lb_in, ub_in, threads=None):
    """The oracle's fixed points of a whole batch (forward sweeps), split over
    host threads (the C oracle releases the GIL): (status, lb, ub)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    lb_in = np.asarray(lb_in, dtype=np.int64)
    ub_in = np.asarray(ub_in, dtype=np.int64)
    threads = threads or os.cpu_count() or 1
    parts = np.array_split(np.arange(len(lb_in)), threads)
    with ThreadPoolExecutor(threads) as ex:
        outs = list(ex.map(lambda ix: oracle.propagate_batch(om, lb_in[ix], ub_in[ix]), parts))
    st = np.concatenate([o[0] for o in outs])
    lb = np.concatenate([o[1] for o in outs])
    ub = np.concatenate([o[2] for o in outs])
    return st, lb, ub


def compare_whole_batch(om, lb_in, ub_in, st_gpu, lb_gpu, ub_gpu):
    """Every store of a batch against the oracle: equal status everywhere,
    equal lb/ub on every fixed point (failed stores' contents are
    unspecified).  Returns (n_fixpoint, n_failed)."""
    st, flb, fub = oracle_batch(om, lb_in, ub_in)
    st_gpu = np.asarray(st_gpu)
    assert set(np.unique(st).tolist()) <= {oracle.FIXPOINT, oracle.FAILED}
    bad = np.nonzero(st_gpu != st)[0]
    assert len(bad) == 0, f"status differs on stores {bad[:10].tolist()}"
    ok = st == oracle.FIXPOINT
    diff = ok[:, None] & ((np.asarray(lb_gpu) != flb) | (np.asarray(ub_gpu) != fub))
    rows = np.nonzero(diff.any(axis=1))[0]
    assert len(rows) == 0, f"fixed points differ on stores {rows[:10].tolist()}"
    return int(ok.sum()), int((~ok).sum())


def compare_batch(om, lb_in, ub_in, st_gpu, lb_gpu, ub_gpu, rows=None):
    """Element-by-element comparison of GPU results with the oracle on the
    given input stores (int arrays [n, n_vars]).  Failed stores compare by
    status only.  Returns (n_fixpoint, n_failed)."""
    idx = range(len(lb_in)) if rows is None else rows
    nf = nx = 0
    for i in idx:
        s, flb, fub, _ = oracle.propagate(om, lb_in[i], ub_in[i])
        assert s in (oracle.FIXPOINT, oracle.FAILED)
        assert int(st_gpu[i]) == s, f"store {i}: gpu status {int(st_gpu[i])} oracle {s}"
        if s == oracle.FIXPOINT:
            nx += 1
            if not (np.array_equal(lb_gpu[i], flb) and np.array_equal(ub_gpu[i], fub)):
                bad = np.nonzero((lb_gpu[i] != flb) | (ub_gpu[i] != fub))[0][:10]
                raise AssertionError(
                    f"store {i} differs at vars {bad.tolist()}: gpu "
                    f"{[(int(lb_gpu[i][v]), int(ub_gpu[i][v])) for v in bad]} oracle "
                    f"{[(int(flb[v]), int(fub[v])) for v in bad]}")
        else:
            nf += 1
    return nx, nf
