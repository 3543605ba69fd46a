"""Benchmark: propagation of a batch of search-tree nodes to their fixed points.

Workload (the propagation-batch configuration): one seeded 30-task, 4-resource
scheduling model (931 variables, ~1,060 propagator rows) and 10,000 search
nodes, each the root store narrowed by 0-15 random branching decisions.  One
step propagates all 10,000 stores through the C ABI (pccp_propagate), in
place, from pristine copies restored before every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank propagates its own
10,000-node batch (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import config_instance, draw_partial_assignments  # noqa: E402

N_NODES = 10_000
NODE_SEED = 1
FAMILY, INSTANCE = "j30", 0
METRIC = "search nodes/s"
UNIT = "nodes/s"
L2_FLUSH_BYTES = 256 << 20


TASKS = {"tiny8": 8, "j30": 30, "j60": 60, "j120": 120}


def workload_config(n_vars, rows, extra=None):
    what = f"{TASKS[FAMILY]}-task" if FAMILY in TASKS else FAMILY
    cfg = {"workload": f"propagation batch: {N_NODES} search nodes (0-15 decisions each) of a "
                       f"seeded {what} 4-resource scheduling model ({n_vars} vars, {rows} rows)",
           "model": f"{FAMILY}/{INSTANCE}", "nodes_per_step": N_NODES, "node_seed": NODE_SEED,
           "l2": "flushed between steps (256 MB write); stores restored from pristine copies"}
    if extra:
        cfg.update(extra)
    return cfg


def build_inputs(rank=0):
    """The model and this rank's 10,000 nodes.  Ranks are independent
    replicas: rank r draws its nodes with seed NODE_SEED + r (rank 0 is the
    single-GPU workload)."""
    inst = config_instance(FAMILY, INSTANCE)
    nodes = draw_partial_assignments(inst.n, inst.horizon, N_NODES, seed=NODE_SEED + rank)
    return inst, nodes


def max_over_ranks(x, world, device):
    """Largest value of x over all ranks (the slowest rank sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_max):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1000.0)


# ------------------------------------------------------------ CPU oracle leg

def oracle_rate(inst, nodes, n_sample, threads):
    """Time the CPU oracle (as it stands) on the first n_sample nodes, split
    over `threads` Python threads (the C oracle releases the GIL)."""
    import oracle
    from oracle.rcpsp import rcpsp_model, node_store
    from concurrent.futures import ThreadPoolExecutor
    om = rcpsp_model(inst)
    sample = nodes[:n_sample]
    lb = np.array([node_store(om, d)[0] for d in sample])
    ub = np.array([node_store(om, d)[1] for d in sample])
    chunks = np.array_split(np.arange(len(sample)), threads)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda ix: oracle.propagate_batch(om, lb[ix], ub[ix]), chunks))
    dt = time.perf_counter() - t0
    return len(sample) / dt, dt


def cpu_baseline(inst, nodes, target_s=12.0):
    """The oracle on the host cores: a 1-thread rate on 1,500 nodes, then the
    whole 10,000-node batch repeated until about target_s of wall time over
    all cores."""
    cores = os.cpu_count() or 1
    r1, t1 = oracle_rate(inst, nodes, 1500, 1)
    passes = max(1, int(round(target_s * r1 * cores / N_NODES)))
    rN, tN = oracle_rate(inst, nodes * passes, N_NODES * passes, cores)
    return {"value": rN, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the {N_NODES}-node batch x {passes} over {cores} threads ({tN:.1f} s); "
                      f"1 thread: {r1:.1f} nodes/s on the first 1500 nodes ({t1:.1f} s)",
            "value_1core": r1}


def run_reference(args):
    """The oracle as the reference arm: each step propagates a bounded
    sample of the same workload on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst, nodes = build_inputs()
    import oracle
    from oracle.rcpsp import rcpsp_model, node_store
    from concurrent.futures import ThreadPoolExecutor
    om = rcpsp_model(inst)
    cores = os.cpu_count() or 1
    per_step = 64 * cores
    lb = np.array([node_store(om, d)[0] for d in nodes[:per_step]])
    ub = np.array([node_store(om, d)[1] for d in nodes[:per_step]])
    chunks = np.array_split(np.arange(per_step), cores)

    def step():
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda ix: oracle.propagate_batch(om, lb[ix], ub[ix]), chunks))

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = per_step / (ms / 1000)
    rows = om.temporal and (len(om.temporal) + len(om.reified) + len(om.linear))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": workload_config(om.n_vars, rows, {"sample_nodes_per_step": per_step}),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"first {per_step} of the {N_NODES} nodes per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def snapshot(self):
        """One query, for a timed region shorter than the sampling period."""
        try:
            out = subprocess.run(["nvidia-smi", f"--id={self.device_index}",
                                  f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=20).stdout
            self.lines += [ln.strip() for ln in out.splitlines() if ln.strip()]
            self.note = "one query at the end of a timed region shorter than the 100 ms period"
        except (OSError, subprocess.TimeoutExpired):
            pass

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.lines:
            self.snapshot()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None,
               "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
               "samples": len(sm)}
        if getattr(self, "note", None):
            out["note"] = self.note
        return out


def explicit_launch(args):
    return bool(args.team or args.teams or args.ctas_per_sm or args.skip_stable
                or args.stream_table)


def launch_desc(args):
    if not explicit_launch(args):
        return "library default"
    return {"team_threads": args.team, "teams_per_cta": args.teams,
            "ctas_per_sm": args.ctas_per_sm, "skip_stable": bool(args.skip_stable),
            "stream_table": bool(args.stream_table)}


KERNEL_SOURCES = ("paper_2207_12116_gb300/csrc/k_propagate.cuh",
                  "paper_2207_12116_gb300/csrc/pccp_device.cuh")
def profile_path():
    """The committed ncu summary of the propagation workload being run."""
    return f"profiles/k_propagate_{FAMILY}_batch.md"


def kernel_hash():
    """Hash of the propagation kernel's sources with comments and blank lines
    left out (a comment edit does not make a capture stale)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        for line in open(os.path.join(ROOT, p)).read().splitlines():
            code = re.sub(r"//.*$", "", line).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of k_propagate from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    try:
        text = open(os.path.join(ROOT, profile_path())).read()
    except OSError:
        return None, None
    rec = {}
    for line in text.splitlines():
        if line.startswith("<!-- ") and ":" in line:
            k, v = line[5:].rstrip(" ->").split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_sha") != kernel_hash():
        return None, "kernel changed since the committed ncu capture"
    if rec.get("nodes", str(N_NODES)) != str(N_NODES):
        return None, "the committed ncu capture is of another batch size"
    try:
        return int(rec["dram_bytes_per_launch"]), profile_path()
    except (KeyError, ValueError):
        return None, None


SEARCH_MODELS = 256
SEARCH_NODE_LIMIT = 4000
EPS_TIME_MS = 2000
EPS_NODE_LIMIT = 0  # > 0: the parallel runs stop on nodes instead of time


COMPLETE_FAMILY, COMPLETE_MODELS = "mixed6_10", 256
COMPLETE_BATCH = True
COMPLETE_SEQUENTIAL = True  # the one-team-per-model form too (about a minute)
LEARNED_IN_BENCH = True     # train a policy (~20 s) and time the learned form
SCALE_LEGS = True           # 60- and 120-task models, first-fail and learned (~30 s)


def _graph_solve(pccp, batch, **kw):
    """One search of a reusable batch captured in a CUDA graph and replayed;
    returns (device ms of the replay, results)."""
    import torch
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            batch.solve_async(stream=stream, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):  # replay on the stream the events are recorded on
        e0.record(stream)
        graph.replay()
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), batch.results(stream=stream)


def _proof_summary(pccp, ms, res):
    nodes = sum(r["nodes"] for r in res)
    per = sorted(r["model_ms"] for r in res)
    return {"ms_to_last_proof": ms, "nodes": nodes, "nodes_per_s": nodes / (ms / 1000),
            "proven": sum(r["status"] == pccp.PCCP_RES_OPTIMAL for r in res),
            "complete": all(r["status"] == pccp.PCCP_RES_OPTIMAL for r in res),
            "model_ms_to_proof": {"p50": per[len(per) // 2], "p99": per[int(0.99 * len(per)) - 1],
                                  "max": per[-1]}}


def complete_batch_bench(pccp, policy=None, training=None):
    """Batched complete solves (the uneven-batch configuration): 256 seeded
    6-10-task models proved optimal, each search one CUDA graph replay of a
    reusable batch in the launch shape the autotuner picks.  Two forms:
    parallel (every team over one shared queue of subproblems of all models,
    work donation, per-model incumbents) for the plain strategies and the
    learned policy, and the sequential order (one team per model, node
    counts equal to the oracle's) for first-fail."""
    from synthetic import config_instance
    from paper_2207_12116_gb300 import autotune
    models = [pccp.Model.from_rcpsp(config_instance(COMPLETE_FAMILY, s))
              for s in range(COMPLETE_MODELS)]
    t0 = time.perf_counter()
    # the shapes are timed on the workload itself: complete parallel solves
    # take a fraction of a second each
    (teams, threads), report = autotune.tune_search_shape(models, node_limit=0,
                                                          deterministic=False)
    tune_s = time.perf_counter() - t0
    b = pccp.Batch(models, threads=threads, teams_per_cta=teams)
    out = {"workload": f"{COMPLETE_MODELS} seeded models of "
                       f"{COMPLETE_FAMILY.replace('mixed', '').replace('_', '-')} tasks, 4 resources "
                       "(config-2 distributions), complete branch and bound to proven optima",
           "graph": True,
           "shape": {"teams_per_cta": teams, "threads": threads, "autotune_s": tune_s,
                     "autotune_batches_per_s": {f"{k[0]}x{k[1]}": v for k, v in report.items()}}}
    forms = [("first_fail", {"strategy": pccp.PCCP_FIRST_FAIL}),
             ("input_order", {"strategy": pccp.PCCP_INPUT_ORDER})]
    if policy is not None:
        forms.append(("learned", {"strategy": pccp.PCCP_LEARNED, "policy": policy}))
    optima = None
    for name, kw in forms:
        _graph_solve(pccp, b, deterministic=False, **kw)  # first replay pays the warm-up
        ms, res = _graph_solve(pccp, b, deterministic=False, **kw)
        out[name] = _proof_summary(pccp, ms, res)
        obj = [r["objective"] for r in res]
        assert optima is None or obj == optima, "optima differ between strategies"
        optima = obj
    out["optima_sum"] = sum(optima)
    if policy is not None:
        # a second sample of the same family (seeds 7000-7255, disjoint from
        # the training seeds too): first-fail's proof sizes have a heavy tail,
        # so the two samples differ
        held = [pccp.Model.from_rcpsp(config_instance(COMPLETE_FAMILY, s))
                for s in range(7000, 7000 + COMPLETE_MODELS)]
        hk = dict(deterministic=False, teams_per_cta=teams, threads=threads)
        h_ff = pccp.solve_batch(held, strategy=pccp.PCCP_FIRST_FAIL, **hk)
        h_ln = pccp.solve_batch(held, strategy=pccp.PCCP_LEARNED, policy=policy, **hk)
        assert [r["objective"] for r in h_ff] == [r["objective"] for r in h_ln]
        out["held_out_seeds_7000_7255"] = {
            name: {"ms_to_last_proof": r[0]["elapsed_ms"], "nodes": sum(x["nodes"] for x in r),
                   "proven": sum(x["status"] == pccp.PCCP_RES_OPTIMAL for x in r)}
            for name, r in (("first_fail", h_ff), ("learned", h_ln))}
        out["learned_vs_first_fail"] = {
            "time_ratio": out["learned"]["ms_to_last_proof"] / out["first_fail"]["ms_to_last_proof"],
            "node_ratio": out["learned"]["nodes"] / out["first_fail"]["nodes"],
            "training": training}
    # the plain form without batching: one parallel search per model, one
    # after another (device time summed; host wall time of the loop)
    t0 = time.perf_counter()
    one = [pccp.solve(m, strategy=pccp.PCCP_FIRST_FAIL, deterministic=False) for m in models]
    wall = time.perf_counter() - t0
    assert [r["objective"] for r in one] == optima
    out["first_fail_one_model_at_a_time"] = {
        "device_ms_sum": sum(r["elapsed_ms"] for r in one), "wall_ms": 1000 * wall,
        "nodes": sum(r["nodes"] for r in one),
        "proven": sum(r["status"] == pccp.PCCP_RES_OPTIMAL for r in one)}
    if COMPLETE_SEQUENTIAL:
        ms, res = _graph_solve(pccp, b, deterministic=True, strategy=pccp.PCCP_FIRST_FAIL)
        out["first_fail_sequential_order"] = _proof_summary(pccp, ms, res)
        assert [r["objective"] for r in res] == optima
    return out


def scale_legs(pccp):
    """Short forms of the 60-task learned-branching comparison and of the
    120-task batch: a policy trained as in --learned (probe labels on 8- and
    30-task nodes, 8 epochs); 64 seeded 60-task models (seeds 1000-1063),
    5,000 nodes each, and 152 seeded 120-task models (seeds 2000-2151, tables
    read from global memory), 1 s each; first-fail and learned, one launch
    per strategy.  Per strategy: nodes/s, models with a schedule, their mean
    best makespan; and model by model, whether the learned policy's best
    makespan is lower, equal or higher.  No model of these sizes is proved
    within such limits, so these are best-makespan-under-a-limit figures."""
    pol, training = train_policy(argparse.Namespace(learned_epochs=8))
    out = {}
    for key, fam, seeds, limit, what in (
            ("learned_60", "j60", range(1000, 1064), {"node_limit": 5000}, "5,000 nodes each"),
            ("large_120", "j120", range(2000, 2152), {"time_limit_ms": 1000},
             "1 s each, tables read from global memory")):
        models = [pccp.Model.from_rcpsp(config_instance(fam, s)) for s in seeds]
        leg = {"workload": f"{len(models)} seeded {fam[1:]}-task 4-resource models, one launch "
                           f"per strategy, {what}"}
        best = {}
        for name, kw in (("first_fail", {"strategy": pccp.PCCP_FIRST_FAIL}),
                         ("learned", {"strategy": pccp.PCCP_LEARNED, "policy": pol})):
            res = pccp.solve_batch(models, **limit, **kw)
            ms = res[0]["elapsed_ms"]
            nodes = sum(r["nodes"] for r in res)
            found = [r["objective"] for r in res if r["has_solution"]]
            best[name] = [r["objective"] if r["has_solution"] else None for r in res]
            leg[name] = {"kernel_ms": ms, "nodes": nodes, "nodes_per_s": nodes / (ms / 1000),
                         "propagator_evals_per_s": sum(r["rows_evaluated"] for r in res)
                         / (ms / 1000),
                         "models_with_schedule": len(found),
                         "mean_best_makespan": float(np.mean(found)) if found else None,
                         "proven": sum(r["status"] != pccp.PCCP_RES_LIMIT for r in res)}
        both = [(a, b) for a, b in zip(best["first_fail"], best["learned"])
                if a is not None and b is not None]
        leg["learned_better_equal_worse"] = [sum(b < a for a, b in both),
                                             sum(b == a for a, b in both),
                                             sum(b > a for a, b in both)]
        leg["training"] = training
        out[key] = leg
    return out


def search_bench(pccp, cpu=True):
    """Search throughput: (a) one persistent launch solving 256 seeded
    30-60-task models depth first, one team per model, each stopped after
    4,000 nodes; (a') the batched complete solves of complete_batch_bench;
    (b) every team of the GPU on one 30-task model (subproblems from
    breadth-first growth, shared incumbent) for 2 s, and on one 120-task
    model; (c) the oracle on a bounded sample of (a)."""
    from synthetic import config_instance
    insts = [config_instance("mixed30_60", s) for s in range(SEARCH_MODELS)]
    models = [pccp.Model.from_rcpsp(i) for i in insts]
    pccp.solve_batch(models[:8], node_limit=50)  # warm-up
    res = pccp.solve_batch(models, node_limit=SEARCH_NODE_LIMIT)
    ms = res[0]["elapsed_ms"]
    nodes = sum(r["nodes"] for r in res)
    rows = sum(r["rows_evaluated"] for r in res)
    out = {"batched": {
        "workload": f"{SEARCH_MODELS} models, 30-60 tasks, 4 resources, depth-first "
                    f"input-order search, {SEARCH_NODE_LIMIT} nodes each, one launch",
        "nodes_per_s": nodes / (ms / 1000), "propagator_evals_per_s": rows / (ms / 1000),
        "ms": ms, "nodes": nodes,
        "solutions_found": sum(r["solutions"] for r in res),
        "iterations_per_node": sum(r["iterations"] for r in res) / max(nodes, 1)}}
    if COMPLETE_BATCH:
        pol = training = None
        if LEARNED_IN_BENCH:
            pol, training = train_policy_rollouts()
        out["batched_complete"] = complete_batch_bench(pccp, pol, training)
    if SCALE_LEGS:
        out.update(scale_legs(pccp))
    for key, fam, what in (("parallel", "j30", "30-task"), ("parallel_large", "j120", "120-task")):
        m = pccp.Model.from_rcpsp(config_instance(fam, 0))
        if EPS_NODE_LIMIT:
            r = pccp.solve(m, deterministic=False, node_limit=EPS_NODE_LIMIT)
        else:
            r = pccp.solve(m, deterministic=False, time_limit_ms=EPS_TIME_MS)
        limit = f"{EPS_NODE_LIMIT} node limit" if EPS_NODE_LIMIT else f"{EPS_TIME_MS} ms limit"
        out[key] = {
            "workload": f"one {what} model ({fam}/0), all teams, {limit}"
                        + (", table read from global memory" if fam == "j120" else ""),
            "nodes_per_s": r["nodes"] / (r["elapsed_ms"] / 1000),
            "propagator_evals_per_s": r["rows_evaluated"] / (r["elapsed_ms"] / 1000),
            "ms": r["elapsed_ms"], "nodes": r["nodes"], "status": r["status"],
            "best_makespan": r["objective"]}
    if cpu:
        import oracle
        from oracle.rcpsp import rcpsp_model
        from concurrent.futures import ThreadPoolExecutor
        cores = os.cpu_count() or 1
        sample = insts[:cores]
        lim = 400
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            rs = list(ex.map(lambda i: oracle.solve(rcpsp_model(i), node_limit=lim), sample))
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"kind": "oracle", "cores": cores,
                               "nodes_per_s": sum(x["nodes"] for x in rs) / dt,
                               "sample": f"first {len(sample)} of the {SEARCH_MODELS} models, "
                                         f"{lim} nodes each, one thread per model ({dt:.1f} s)"}
    return out


def link_probe(nbytes, reps=5):
    """The CPU-GPU link as the host pipeline uses it: copy-engine copies of
    nbytes between pinned host memory and the device, host to device, device
    to host, and both at once on two streams (best of reps, CUDA events)."""
    import torch
    n = nbytes // 4
    h_in = torch.ones(n, dtype=torch.int32).pin_memory()
    h_out = torch.empty(n, dtype=torch.int32).pin_memory()
    d_in = torch.empty(n, dtype=torch.int32, device="cuda")
    d_out = torch.ones(n, dtype=torch.int32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = {"h2d": 1e9, "d2h": 1e9, "both": 1e9}
    for _ in range(reps):
        for kind in best:
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s1)
            s2.wait_event(a)
            if kind in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    d_in.copy_(h_in, non_blocking=True)
            if kind in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    h_out.copy_(d_out, non_blocking=True)
            c = torch.cuda.Event()
            c.record(s2)
            s1.wait_event(c)
            b.record(s1)
            b.synchronize()
            best[kind] = min(best[kind], a.elapsed_time(b))
    return {"h2d_gbs": 4 * n / best["h2d"] / 1e6, "d2h_gbs": 4 * n / best["d2h"] / 1e6,
            "both_gbs": 8 * n / best["both"] / 1e6, "bytes_each_way": 4 * n}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2207_12116_gb300 as pccp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    inst, nodes = build_inputs(rank)
    rows = pccp.rcpsp.build_rows(inst)
    model = pccp.Model.from_rows(rows)
    lb_h, ub_h = pccp.rcpsp.node_stores(rows, nodes)
    nv = model.n_vars
    pristine_lb = torch.from_numpy(lb_h).to(dev)
    pristine_ub = torch.from_numpy(ub_h).to(dev)
    lb = pristine_lb.clone()
    ub = pristine_ub.clone()
    status = torch.empty(N_NODES, dtype=torch.int32, device=dev)
    iters = torch.empty(N_NODES, dtype=torch.int32, device=dev)
    work = torch.empty((N_NODES, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    cfg = None
    if explicit_launch(args):
        cfg = pccp.launch_config(args.team, args.teams, args.ctas_per_sm, 0,
                                 True if args.skip_stable else None, args.stream_table)

    def prepare():
        lb.copy_(pristine_lb)
        ub.copy_(pristine_ub)
        flush.fill_(1)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        prepare()
        pccp.propagate(model, lb, ub, status, iters, config=cfg)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        prepare()
        ev[k][0].record(stream)
        pccp.propagate(model, lb, ub, status, iters, config=cfg, work=work)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(kernel_ms)
    ms_max = max_over_ranks(ms, world, dev)

    st = status.cpu().numpy()
    it = iters.cpu().numpy().astype(np.int64)
    wk = work.cpu().numpy().astype(np.int64)
    rows_per_sweep = model.rows
    evals = int(wk[:, 0].sum())          # rows actually evaluated (stable rows skipped)
    bytes_smem = int(wk[:, 1].sum())     # algorithmic bytes they read
    io_bytes = 4 * nv * N_NODES * 4 + 8 * N_NODES  # read+write lb, ub; status, iterations

    e2e = None
    if not args.no_e2e:
        if cfg is not None:
            raise SystemExit("--no-e2e is required with an explicit launch shape")
        # end to end through the public API (pccp_propagate_host): pinned host
        # stores in, fixed points out, copied in chunks that overlap the
        # propagation of other chunks (--e2e-chunk -1: read and written in
        # place by the kernel); wall time of each synchronous call
        src_lb = torch.from_numpy(lb_h)
        src_ub = torch.from_numpy(ub_h)
        lb_pin = torch.empty_like(src_lb).pin_memory()
        ub_pin = torch.empty_like(src_ub).pin_memory()
        out_st = torch.empty(N_NODES, dtype=torch.int32).pin_memory()
        out_it = torch.empty(N_NODES, dtype=torch.int32).pin_memory()
        e2e_ms = []
        n_e2e = min(args.steps, 100)
        for k in range(max(args.warmup, 0) + n_e2e):
            lb_pin.copy_(src_lb)  # this step's inputs (outside the timed call)
            ub_pin.copy_(src_ub)
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pccp.propagate_host(model, lb_pin, ub_pin, out_st, out_it, chunk_stores=args.e2e_chunk)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                e2e_ms.append(dt * 1000.0)
        e2e_v = whole_job_rate(world, N_NODES, max_over_ranks(statistics.mean(e2e_ms), world, dev))
        assert np.array_equal(out_st.numpy(), st), "end-to-end results differ from device-timed run"
        fx = st == 0  # fixed points are unique; failed stores' contents are unspecified
        assert np.array_equal(lb_pin.numpy()[fx], lb.cpu().numpy()[fx]), "end-to-end stores differ"
        e2e = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * nv * N_NODES,
               "d2h_bytes_per_step": 2 * 4 * nv * N_NODES + 8 * N_NODES,
               "api": ("pccp_propagate_host (pinned host stores read and written in place by "
                       "the kernel over the CPU-GPU link)" if args.e2e_chunk < 0 else
                       "pccp_propagate_host (pinned host stores, copied in chunks of "
                       + (f"{args.e2e_chunk}" if args.e2e_chunk else "the library's size")
                       + " overlapping the propagation; the call's copies and launches "
                         "captured in a CUDA graph on the first warm-up call and replayed)"),
               "timing": "host wall clock around each synchronous call"}
        if not args.no_probes:
            # the roof of this path: every store crosses the CPU-GPU link twice
            lk = link_probe(8 * nv * N_NODES)  # lb and ub, each way
            step_bytes = e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]
            link_gbs = step_bytes / (statistics.mean(e2e_ms) / 1000) / 1e9
            e2e["link"] = {"bound": "cpu-gpu link", "achieved": link_gbs, "peak": lk["both_gbs"],
                           "unit": "GB/s", "frac": link_gbs / lk["both_gbs"],
                           "peak_source": "measured in this run: copy-engine copies of "
                                          f"{lk['bytes_each_way']} B each way at once, pinned",
                           "h2d_gbs": lk["h2d_gbs"], "d2h_gbs": lk["d2h_gbs"]}

    if rank == 0:
        peaks = load_peaks()
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        sm_mhz = clk.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median")
        smem_peak = sms * 128 * (sm_mhz or 0) * 1e6 / 1e9  # GB/s: 128 B/clk/SM
        achieved = bytes_smem / (ms / 1000) / 1e9
        hbm_peak = peaks.get("hbm_gbs")
        traffic, traffic_src = recorded_traffic()
        line = {
            "metric": METRIC, "value": whole_job_rate(world, N_NODES, ms_max), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": workload_config(nv, rows_per_sweep, {"parallelism": f"replicas{world}",
                                                           "launch": launch_desc(args)}),
            "propagator_evals_per_s": world * evals / (ms_max / 1000),
            "fixpoint_iterations_per_node": float(it.mean()),
            "rows_evaluated_per_node": evals / N_NODES,
            "rows_skipped_fraction": 1.0 - evals / float(it.sum() * rows_per_sweep),
            "failed_nodes": int((st == 1).sum()),
            "roofline": {"bound": "smem", "achieved": achieved, "peak": smem_peak,
                         "unit": "GB/s", "frac": achieved / smem_peak if smem_peak else None,
                         "traffic": traffic, "traffic_source": traffic_src,
                         "peak_source": f"derived: {sms} SMs x 128 B/clk x {sm_mhz} MHz "
                                        f"(median SM clock sampled during the run)",
                         "algorithmic_bytes_per_launch": bytes_smem,
                         "hbm": {"io_bytes_per_launch": io_bytes,
                                 "achieved": io_bytes / (ms / 1000) / 1e9,
                                 "peak": hbm_peak, "peak_source": "of measured (MEASURED_PEAKS.json)"}},
            "cpu_baseline": None,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk,
            "wall_s_timed_loop": wall,
            "kernel_ms_min": min(kernel_ms), "kernel_ms_max": max(kernel_ms),
        }
        if not args.no_probes:
            # measured roofs (after the timed region): the nominal 128 B/clk/SM
            # cross-checked by a conflict-free shared-load probe
            probes = pccp.roofline_probes()
            line["roofline"]["probes"] = probes
            meas = probes["smem_load"]["per_clk_per_sm"] * sms * (sm_mhz or 0) * 1e6 / 1e9
            line["roofline"]["frac_of_probe"] = achieved / meas if meas else None
            # the second roof: the kernels' own access pattern, 8-byte interval
            # loads at random indices (random banks halve the conflict-free rate)
            gather = probes["smem_scattered_v2"]["per_clk_per_sm"] * sms * (sm_mhz or 0) * 1e6 / 1e9
            line["roofline"]["gather_roof"] = {
                "peak": gather, "unit": "GB/s", "frac": achieved / gather if gather else None,
                "source": "measured: 8-byte shared loads at random indices "
                          f"({probes['smem_scattered_v2']['per_clk_per_sm']:.1f} B/clk/SM)"}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst, nodes)
        if not args.no_search:
            line["search"] = search_bench(pccp, cpu=not args.no_cpu_baseline)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_profile_leg(args):
    """One warm-up launch and one launch of a search kernel, for ncu captures
    (skip 1 launch of the kernel, capture 1):
      batched : k_solve_slots, 256 seeded 30-60-task models, input order,
                500 nodes each, the library's launch shape;
      complete: k_search_queue, the 256 6-10-task models proved optimal in
                the parallel form, first-fail, 8 teams of 64 threads per CTA."""
    import torch
    import paper_2207_12116_gb300 as pccp
    from synthetic import config_instance
    torch.cuda.set_device(0)
    if args.profile_leg == "batched":
        models = [pccp.Model.from_rcpsp(config_instance("mixed30_60", s)) for s in range(256)]
        pccp.solve_batch(models[:8], node_limit=50)
        r = pccp.solve_batch(models, node_limit=500)
    else:
        models = [pccp.Model.from_rcpsp(config_instance(COMPLETE_FAMILY, s))
                  for s in range(COMPLETE_MODELS)]
        kw = dict(strategy=pccp.PCCP_FIRST_FAIL, deterministic=False, teams_per_cta=8, threads=64)
        pccp.solve_batch(models[:4], **kw)
        r = pccp.solve_batch(models, **kw)
    print(json.dumps({"leg": args.profile_leg, "ms": r[0]["elapsed_ms"],
                      "nodes": sum(x["nodes"] for x in r),
                      "rows": sum(x["rows_evaluated"] for x in r)}), flush=True)


def run_search_only(args):
    """Only the search leg (used for ncu captures of the search kernels)."""
    import torch
    import paper_2207_12116_gb300 as pccp
    torch.cuda.set_device(0)
    global SEARCH_MODELS, SEARCH_NODE_LIMIT, EPS_NODE_LIMIT, COMPLETE_BATCH
    SEARCH_MODELS, SEARCH_NODE_LIMIT, EPS_NODE_LIMIT, COMPLETE_BATCH = 64, 500, 2_000_000, False
    print(json.dumps(search_bench(pccp, cpu=False)), flush=True)


ROLLOUT_TRAIN_SEEDS = range(5000, 5096)  # disjoint from the complete batch's seeds 0..255


def train_policy_rollouts():
    """A learned-branching policy for the complete-solve family, trained on
    96 other seeded 6-10-task models: proof-phase nodes labelled by the
    measured first-fail proof sizes below each candidate's split, with
    first-fail's width preference as a prior (soft targets, T = 0.5, width
    weight 0.5), 30 epochs.  Returns (policy, training summary)."""
    import paper_2207_12116_gb300 as pccp
    from paper_2207_12116_gb300 import learn
    t0 = time.perf_counter()
    insts = [config_instance(COMPLETE_FAMILY, s) for s in ROLLOUT_TRAIN_SEEDS]
    data, stats = learn.collect_rollouts(insts, nodes_per_model=32, seed=1)
    t1 = time.perf_counter()
    learn.rollout_targets(data, "soft_ff", 0.5, 0.5)
    pol = pccp.Policy.random(0)
    losses = learn.train(pol, data, epochs=30, groups_per_batch=64, lr=2e-3)
    return pol, {"labels": "first-fail proof sizes below each candidate's split (rollouts), "
                           "soft targets with a first-fail width prior",
                 "train_models": f"{COMPLETE_FAMILY} seeds {ROLLOUT_TRAIN_SEEDS.start}-"
                                 f"{ROLLOUT_TRAIN_SEEDS.stop - 1}",
                 **stats, "epochs": 30, "loss_first_last": [losses[0], losses[-1]],
                 "top1_accuracy": learn.ranking_accuracy(pol, data),
                 "collect_s": t1 - t0, "seconds": time.perf_counter() - t0}


def train_policy(args):
    """A learned-branching policy trained on nodes of the 8-task and 30-task
    families (strong-branching probes blended with first-fail); returns
    (policy, training summary)."""
    import paper_2207_12116_gb300 as pccp
    from paper_2207_12116_gb300 import learn
    t0 = time.perf_counter()
    train_insts = [config_instance("tiny8", s) for s in range(64)] + \
                  [config_instance("j30", s) for s in range(16)]
    data = learn.collect(train_insts, nodes_per_model=256, seed=7)
    pol = pccp.Policy.random(0)
    losses = learn.train(pol, data, epochs=args.learned_epochs, groups_per_batch=256, lr=2e-3)
    acc = learn.ranking_accuracy(pol, data)
    return pol, {"groups": int(data["group_off"].numel() - 1),
                 "rows": int(data["features"].shape[0]), "epochs": args.learned_epochs,
                 "loss_first_last": [losses[0], losses[-1]], "probe_top1_accuracy": acc,
                 "seconds": time.perf_counter() - t0}


def run_learned(args):
    """Learned branching against plain first-fail on 64 seeded 60-task models
    (one persistent launch each, same limits, same GPU).  The policy is
    trained first on nodes of the 8-task and 30-task families."""
    import torch
    import paper_2207_12116_gb300 as pccp
    torch.cuda.set_device(0)
    pol, training = train_policy(args)
    models = [pccp.Model.from_rcpsp(config_instance("j60", 1000 + s)) for s in range(64)]
    out = {}
    for name, kw in (("first_fail", {"strategy": pccp.PCCP_FIRST_FAIL}),
                     ("learned", {"strategy": pccp.PCCP_LEARNED, "policy": pol})):
        res = pccp.solve_batch(models, node_limit=args.learned_nodes,
                               time_limit_ms=args.learned_ms, **kw)
        proven = [r for r in res if r["status"] != pccp.PCCP_RES_LIMIT]
        out[name] = {
            "kernel_ms": res[0]["elapsed_ms"], "nodes": sum(r["nodes"] for r in res),
            "proven_optimal_or_infeasible": len(proven),
            "nodes_to_proof_mean": (float(np.mean([r["nodes"] for r in proven]))
                                    if proven else None),
            "with_solution": sum(r["has_solution"] for r in res),
            "mean_best_makespan": float(np.mean([r["objective"] for r in res
                                                 if r["has_solution"]] or [float("nan")])),
            "best_makespans": [r["objective"] for r in res]}
    both = [(a, b) for a, b in zip(out["first_fail"]["best_makespans"],
                                   out["learned"]["best_makespans"])
            if a is not None and b is not None]
    # 8-task models: complete searches, so nodes and time to proven optimum
    tiny = [pccp.Model.from_rcpsp(config_instance("tiny8", s)) for s in range(100)]
    proofs = {}
    for name, kw in (("first_fail", {"strategy": pccp.PCCP_FIRST_FAIL}),
                     ("learned", {"strategy": pccp.PCCP_LEARNED, "policy": pol})):
        res = pccp.solve_batch(tiny, **kw)
        proofs[name] = {"kernel_ms": res[0]["elapsed_ms"],
                        "nodes_total": sum(r["nodes"] for r in res),
                        "proven": sum(r["status"] == pccp.PCCP_RES_OPTIMAL for r in res),
                        "optima": [r["objective"] for r in res]}
    assert proofs["first_fail"]["optima"] == proofs["learned"]["optima"], "optima must agree"
    line = {"metric": "time and nodes to proven optimum, learned vs first-fail",
            "proofs_tiny8": {k: {kk: vv for kk, vv in v.items() if kk != "optima"}
                             for k, v in proofs.items()},
            "workload": f"64 seeded 60-task 4-resource models, one launch per strategy, "
                        f"{args.learned_nodes} nodes and {args.learned_ms} ms per model",
            "training": training,
            "first_fail": {k: v for k, v in out["first_fail"].items() if k != "best_makespans"},
            "learned": {k: v for k, v in out["learned"].items() if k != "best_makespans"},
            "learned_better_equal_worse": [sum(b < a for a, b in both), sum(b == a for a, b in both),
                                           sum(b > a for a, b in both)]}
    print(json.dumps(line), flush=True)


def run_large(args):
    """120-task models (14,521 variables, ~570 KB table read from global
    memory) solved in one persistent launch, one 1024-thread team per model,
    each model stopped after a time limit.  For every strategy asked for
    (first-fail, and the learned policy trained as in --learned) and every
    limit in --large-limits: nodes/s, the bytes the row evaluations read per
    second and the best makespans found (best makespan against time)."""
    import torch
    import paper_2207_12116_gb300 as pccp
    torch.cuda.set_device(0)
    models = [pccp.Model.from_rcpsp(config_instance("j120", 2000 + s))
              for s in range(args.large_models)]
    info = models[0].info
    bytes_per_row = info.bytes_per_sweep / models[0].rows
    # the table's share of those bytes (rows and terms, read from global
    # memory through L1/L2 at this size): T 12 B, Rf 16 B, L 12 B + 8 B/term
    table_per_row = (12 * info.n_temporal + 16 * info.n_reified + 12 * info.n_linear
                     + 8 * info.n_terms) / models[0].rows
    limits = [int(x) for x in args.large_limits.split(",")] if args.large_limits else [args.large_ms]
    strategies = [("first_fail", {"strategy": pccp.PCCP_FIRST_FAIL})]
    training = None
    if args.large_learned:
        pol, training = train_policy(args)
        strategies.append(("learned", {"strategy": pccp.PCCP_LEARNED, "policy": pol}))
    runs = []
    for name, kw in strategies:
        for lim in limits:
            t0 = time.perf_counter()
            res = pccp.solve_batch(models, time_limit_ms=lim, stream_table=args.stream_table,
                                   **kw)
            wall = time.perf_counter() - t0
            ms = res[0]["elapsed_ms"]
            nodes = sum(r["nodes"] for r in res)
            rows = sum(r["rows_evaluated"] for r in res)
            found = [r["objective"] for r in res if r["has_solution"]]
            runs.append({"strategy": name, "limit_ms": lim, "kernel_ms": ms, "wall_s": wall,
                         "nodes": nodes, "nodes_per_s": nodes / (ms / 1000),
                         "propagator_evals_per_s": rows / (ms / 1000),
                         "row_bytes_per_s": rows * bytes_per_row / (ms / 1000),
                         "table_gbs": rows * table_per_row / (ms / 1000) / 1e9,
                         "models_with_solution": len(found),
                         "mean_best_makespan": float(np.mean(found)) if found else None})
    first = runs[0]
    line = {"metric": "search nodes/s, best makespan under a time limit (120-task models)",
            "workload": f"{args.large_models} seeded 120-task 4-resource models, one launch per "
                        f"strategy and limit, one 1024-thread team per model",
            **{k: first[k] for k in ("nodes_per_s", "propagator_evals_per_s", "row_bytes_per_s",
                                     "kernel_ms", "wall_s", "nodes", "models_with_solution",
                                     "mean_best_makespan")},
            "runs": runs, "training": training, "stream_table": bool(args.stream_table)}
    line["table_stream"] = {"achieved_gbs": first["table_gbs"], "table_bytes": info.table_bytes}
    if not args.no_probes:
        l2 = pccp.roofline_probes()["l2_read"]
        line["table_stream"].update({"l2_probe_gbs": l2["gbs"],
                                     "frac_of_l2_probe": first["table_gbs"] / l2["gbs"]})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="stores per chunk of the end-to-end call (0: the library's choice; "
                         "-1: no copies, the kernel reads and writes the host stores)")
    ap.add_argument("--no-search", action="store_true")
    ap.add_argument("--learned", action="store_true",
                    help="learned branching vs first-fail on 64 60-task models (own JSON line)")
    ap.add_argument("--learned-epochs", type=int, default=8)
    ap.add_argument("--learned-nodes", type=int, default=20000)
    ap.add_argument("--learned-ms", type=int, default=20000)
    ap.add_argument("--family", default="",
                    help="propagation workload's model family (default j30: the headline)")
    ap.add_argument("--nodes", type=int, default=0,
                    help="stores per propagation step (default 10,000)")
    ap.add_argument("--no-probes", action="store_true",
                    help="skip the roofline microbenchmarks after the timed region")
    ap.add_argument("--large", action="store_true",
                    help="120-task models in one launch (own JSON line)")
    ap.add_argument("--large-models", type=int, default=1024)
    ap.add_argument("--stream-table", action="store_true",
                    help="stream tables too large for shared memory through TMA bulk-copy "
                         "rings (default: read in place)")
    ap.add_argument("--large-ms", type=int, default=7000)
    ap.add_argument("--large-limits", default="",
                    help="comma-separated time limits (ms) for a best-makespan-vs-time curve")
    ap.add_argument("--large-learned", action="store_true",
                    help="also run the learned policy (trained first, as in --learned)")
    ap.add_argument("--search-only", action="store_true",
                    help="small search leg only (64 models x 500 nodes; parallel runs "
                         "stopped after 2,000,000 nodes)")
    ap.add_argument("--profile-leg", choices=["batched", "complete"], default="",
                    help="one warm-up and one measured launch of a search kernel (ncu captures)")
    ap.add_argument("--team", type=int, default=0, help="threads per team (0: library default)")
    ap.add_argument("--teams", type=int, default=0, help="teams per CTA (0: library default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--skip-stable", action="store_true",
                    help="re-run a row only after one of its variables changed")
    args = ap.parse_args()
    global FAMILY, N_NODES
    if args.family:  # another propagation workload (profiling and parity of other sizes)
        FAMILY = args.family
    if args.nodes > 0:
        N_NODES = args.nodes
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_leg:
        run_profile_leg(args)
    elif args.search_only:
        run_search_only(args)
    elif args.learned:
        run_learned(args)
    elif args.large:
        run_large(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
