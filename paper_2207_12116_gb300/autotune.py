"""Autotuner for the launch shapes of the propagation and search kernels.

The result of every launch shape is the same fixed point (any fair order
reaches it, Sec. 3 of the paper), so the shape is a pure performance choice:
threads per team (which sets the rows each thread evaluates per iteration),
teams per CTA (how many stores share one copy of the table in shared
memory) and, for the batched search, threads per model.  The tuner times
each candidate on a sample with CUDA events on the current stream, restoring
the sample's stores before every trial, and caches the fastest per model
shape.  Every trial runs the library's own kernels through the C ABI.
"""
import statistics

from . import Model, launch_config, propagate, solve_batch, PccpError

PROPAGATE_CANDIDATES = [(64, 4), (64, 8), (64, 15), (96, 5), (96, 10), (128, 2), (128, 4),
                        (128, 8), (160, 3), (192, 5), (256, 2), (256, 4), (512, 1)]
SEARCH_THREADS = [64, 128, 256, 512]

_cache = {}


def _shape_key(model: Model):
    i = model.info
    return (int(i.n_vars), int(i.n_temporal), int(i.n_reified), int(i.n_linear), int(i.n_terms))


def tune_propagate(model: Model, lb, ub, candidates=None, trials=3, use_cache=True):
    """Pick the fastest (team_threads, teams_per_cta) for propagating batches
    like (lb, ub) (int32 CUDA tensors [n, n_vars], left unchanged).
    Returns (pccp_launch_config, report) where report lists every candidate's
    best time in ms (None when it does not fit shared memory)."""
    import torch
    key = ("propagate", _shape_key(model), int(lb.shape[0]))
    if use_cache and key in _cache:
        return _cache[key]
    stream = torch.cuda.current_stream()
    wlb, wub = lb.clone(), ub.clone()
    st = torch.empty(lb.shape[0], dtype=torch.int32, device=lb.device)
    it = torch.empty_like(st)
    report = {}
    best = None
    for team, teams in (candidates or PROPAGATE_CANDIDATES):
        cfg = launch_config(team, teams)
        times = []
        try:
            for _ in range(trials + 1):  # the first run warms up
                wlb.copy_(lb)
                wub.copy_(ub)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                propagate(model, wlb, wub, st, it, config=cfg)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
        except PccpError:
            report[(team, teams)] = None
            continue
        t = min(times[1:])
        report[(team, teams)] = t
        if best is None or t < best[0]:
            best = (t, team, teams)
    if best is None:
        raise PccpError(-3, "no launch shape fits shared memory")
    out = (launch_config(best[1], best[2]), report)
    _cache[key] = out
    return out


def tune_search_threads(models, node_limit=200, candidates=None, use_cache=True):
    """Pick the threads per model (one team per CTA) for a batched search of
    models like these: each candidate solves the batch with a small node
    limit and the fastest kernel time wins.  Returns (threads, report)."""
    key = ("search", tuple(sorted(_shape_key(m) for m in models)), node_limit)
    if use_cache and key in _cache:
        return _cache[key]
    report = {}
    best = None
    for threads in (candidates or SEARCH_THREADS):
        try:
            solve_batch(models, node_limit=max(1, node_limit // 8), threads=threads)
            r = solve_batch(models, node_limit=node_limit, threads=threads)
        except PccpError:
            report[threads] = None
            continue
        ms = statistics.mean(x["elapsed_ms"] for x in r)
        nodes = sum(x["nodes"] for x in r)
        rate = nodes / (ms / 1000.0)
        report[threads] = rate
        if best is None or rate > best[0]:
            best = (rate, threads)
    if best is None:
        raise PccpError(-3, "no team size fits shared memory")
    out = (best[1], report)
    _cache[key] = out
    return out
