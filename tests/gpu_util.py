"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle


def oracle_model_from_lists(gm):
    return oracle.Model(gm.lb0, gm.ub0, gm.temporal, gm.linear, gm.reified, gm.objective, gm.branch)


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
