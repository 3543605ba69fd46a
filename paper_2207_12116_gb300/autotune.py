"""Autotuner for the launch shapes of the propagation and search kernels.

The result of every launch shape is the same fixed point (any fair order
reaches it, Sec. 3 of the paper), so the shape is a pure performance choice:
threads per team (which sets the propagator rows each thread evaluates per
iteration), teams per CTA (how many stores share one copy of the table in
shared memory, or, for the batched search, how many models are searched
side by side in one CTA), and, for the parallel search of one model, the
queue granularity (frontier subproblems per team) and the node budget after
which a team hands work to idle teams.  The tuner times each candidate on a
sample with CUDA events on the current stream (or the search's own device
time), restoring the sample's stores before every trial, and caches the
fastest per model shape.  Every trial runs the library's own kernels through
the C ABI.
"""
import statistics

from . import Model, launch_config, propagate, solve, solve_batch, PccpError

PROPAGATE_CANDIDATES = [(64, 4), (64, 8), (64, 15), (96, 5), (96, 10), (128, 2), (128, 4),
                        (128, 8), (160, 3), (192, 5), (256, 2), (256, 4), (512, 1)]
SEARCH_THREADS = [64, 128, 256, 512, 1024]
# batched search: (teams per CTA, threads per team); 0 threads = rows-based
SEARCH_SHAPES = [(1, 256), (1, 512), (1, 1024), (2, 256), (2, 512), (3, 256), (4, 128), (4, 256),
                 (6, 128), (8, 128), (8, 64), (12, 64), (15, 64), (15, 32)]
# parallel search of one model: (frontier subproblems per team, donation node budget)
EPS_CANDIDATES = [(2, 0), (4, 0), (8, 0), (4, -1), (16, -1)]

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


def tune_search_shape(models, node_limit=300, candidates=None, strategy=None, use_cache=True,
                      deterministic=True):
    """Pick (teams_per_cta, threads) for a batched search of models like these:
    each candidate solves the batch with a node limit per model (in the
    sequential order every candidate does the same work; in the parallel
    form about the same; node_limit=0: complete solves, for batches that
    finish quickly) and the highest nodes/s of device time (complete solves:
    the shortest time, reported as proofs of the whole batch per second) wins.
    Returns ((teams_per_cta, threads), report)."""
    from . import PCCP_FIRST_FAIL
    strategy = PCCP_FIRST_FAIL if strategy is None else strategy
    key = ("shape", tuple(sorted(_shape_key(m) for m in models)), node_limit, strategy,
           deterministic)
    if use_cache and key in _cache:
        return _cache[key]
    report = {}
    best = None
    for teams, threads in (candidates or SEARCH_SHAPES):
        try:
            solve_batch(models, node_limit=max(1, node_limit // 8) if node_limit else 0,
                        threads=threads, teams_per_cta=teams, strategy=strategy,
                        deterministic=deterministic)
            r = solve_batch(models, node_limit=node_limit, threads=threads, teams_per_cta=teams,
                            strategy=strategy, deterministic=deterministic)
        except PccpError:
            report[(teams, threads)] = None
            continue
        ms = r[0]["elapsed_ms"]
        # node-limited runs: nodes/s; complete runs: 1 / time to the last proof
        rate = sum(x["nodes"] for x in r) / (ms / 1000.0) if node_limit else 1000.0 / ms
        report[(teams, threads)] = rate
        if best is None or rate > best[0]:
            best = (rate, (teams, threads))
    if best is None:
        raise PccpError(-3, "no batched launch shape fits shared memory")
    out = (best[1], report)
    _cache[key] = out
    return out


def tune_parallel(model, node_limit=200_000, candidates=None, use_cache=True):
    """Pick (queue_granularity, donate_nodes) for the parallel search of one
    model: each candidate runs a node-limited search and the highest nodes/s
    wins.  Returns ((queue_granularity, donate_nodes), report)."""
    key = ("eps", _shape_key(model), node_limit)
    if use_cache and key in _cache:
        return _cache[key]
    report = {}
    best = None
    for gran, donate in (candidates or EPS_CANDIDATES):
        try:
            r = solve(model, deterministic=False, node_limit=node_limit, queue_granularity=gran,
                      donate_nodes=donate)
        except PccpError:
            report[(gran, donate)] = None
            continue
        rate = r["nodes"] / (r["elapsed_ms"] / 1000.0)
        report[(gran, donate)] = rate
        if best is None or rate > best[0]:
            best = (rate, (gran, donate))
    if best is None:
        raise PccpError(-3, "no parallel search shape ran")
    out = (best[1], report)
    _cache[key] = out
    return out
