"""GB300 (sm_103a) PCCP propagate-and-search: Python binding of libpccp.so.

The names mirror the C ABI of include/pccp.h.  This module only marshals
arguments (numpy arrays for model rows, torch CUDA tensors for stores); every
step of propagation and search runs in the CUDA library, and loading fails
loudly when the library is missing.

    m = Model.from_arrays(...) or Model.from_rcpsp(instance)
    propagate(m, lb, ub)          # torch int32 CUDA tensors [n, n_vars], in place
    solve(m) / solve_batch([m1, m2, ...])
"""
import ctypes

import numpy as np

from . import _abi
from ._abi import (PCCP_OK, PCCP_ERR_INVALID, PCCP_ERR_OVERFLOW, PCCP_ERR_SMEM,  # noqa: F401
                   PCCP_ERR_TIMEOUT, PCCP_ERR_CUDA, PCCP_ERR_UNSUPPORTED, PCCP_ERR_SCRATCH,
                   PCCP_FIXPOINT,
                   PCCP_FAILED, PCCP_ERROR, PCCP_INPUT_ORDER, PCCP_FIRST_FAIL, PCCP_LEARNED,
                   PCCP_OPTIMISE,
                   PCCP_COUNT_ALL, PCCP_RES_OPTIMAL, PCCP_RES_INFEASIBLE, PCCP_RES_LIMIT,
                   PCCP_HOST_IN_PLACE, INT32_MAX, PccpError, check, load, library_path)
from . import rcpsp  # noqa: F401

__all__ = ["Model", "pccp_model_create", "pccp_model_destroy", "pccp_model_get_info",
           "pccp_propagate", "pccp_propagate_ex", "pccp_solve", "pccp_solve_batch",
           "pccp_solve_batch_noalloc", "pccp_batch_create", "pccp_batch_solve_async",
           "pccp_batch_results", "pccp_batch_destroy", "pccp_batch_get_shape", "Batch", "Policy",
           "pccp_policy_create", "pccp_policy_destroy", "pccp_policy_get_weights",
           "pccp_policy_get_gradients",
           "pccp_policy_features", "pccp_policy_score", "pccp_policy_train_step",
           "pccp_error_string", "propagate", "propagate_host", "pccp_propagate_host", "solve",
           "solve_batch",
           "PccpError", "load", "library_path", "pccp_probe", "roofline_probes"]


def _i32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    if a.size and (a.min() < -(1 << 31) or a.max() >= (1 << 31)):
        raise PccpError(PCCP_ERR_OVERFLOW, "value outside int32")
    a = a.astype(np.int32)
    return a.reshape(shape) if shape is not None else a.reshape(-1)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


# ------------------------------------------------------------- raw C names

def pccp_model_create(desc):
    h = ctypes.c_void_p()
    rc = load().pccp_model_create(ctypes.byref(desc), ctypes.byref(h))
    return rc, h


def pccp_model_destroy(handle):
    load().pccp_model_destroy(handle)


def pccp_model_get_info(handle):
    info = _abi.pccp_model_info()
    rc = load().pccp_model_get_info(handle, ctypes.byref(info))
    return rc, info


def pccp_propagate(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr, stream):
    return load().pccp_propagate(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr, stream)


def pccp_propagate_ex(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr, work_ptr, cfg,
                      stream):
    return load().pccp_propagate_ex(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr,
                                    work_ptr, ctypes.byref(cfg) if cfg is not None else None,
                                    stream)


def pccp_solve(handle, opts, result, stream):
    return load().pccp_solve(handle, ctypes.byref(opts), ctypes.byref(result), stream)


def pccp_solve_batch(handles, opts, results, stream):
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.value for h in handles])
    return load().pccp_solve_batch(arr, n, ctypes.byref(opts), results, stream)


def pccp_solve_batch_noalloc(handles, opts, results, stream):
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.value for h in handles])
    return load().pccp_solve_batch_noalloc(arr, n, ctypes.byref(opts), results, stream)


def pccp_batch_create(handles, threads, teams_per_cta=0):
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.value for h in handles])
    h = ctypes.c_void_p()
    rc = load().pccp_batch_create(arr, n, threads, teams_per_cta, ctypes.byref(h))
    return rc, h


def pccp_batch_get_shape(handle):
    t, k, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = load().pccp_batch_get_shape(handle, ctypes.byref(t), ctypes.byref(k), ctypes.byref(g))
    return rc, (t.value, k.value, g.value)


def pccp_batch_solve_async(handle, opts, stream):
    return load().pccp_batch_solve_async(handle, ctypes.byref(opts), stream)


def pccp_batch_results(handle, results, stream):
    return load().pccp_batch_results(handle, results, stream)


def pccp_batch_destroy(handle):
    load().pccp_batch_destroy(handle)


def pccp_error_string(code):
    return _abi.error_string(code)


def pccp_probe(kind, iters=0):
    """One roofline microbenchmark (include/pccp_probe.h) on the current
    device: {"work", "ms", "sm_cycles", "n_sms", "ctas"}."""
    r = _abi.pccp_probe_result()
    check(_abi.load_probe().pccp_probe(kind, iters, ctypes.byref(r)), "pccp_probe")
    return {"work": r.work, "ms": r.ms, "sm_cycles": r.sm_cycles, "n_sms": r.n_sms,
            "ctas": r.ctas}


def roofline_probes():
    """The measured roofs: shared-memory load bytes and relaxed shared atomics
    per clock per SM, scattered 8-byte interval loads per clock per SM, and L2
    read GB/s; each with the SM clock the probe ran at."""
    out = {}
    for name, kind, unit in (("smem_load", _abi.PCCP_PROBE_SMEM_LOAD, "B/clk/SM"),
                             ("smem_atomic", _abi.PCCP_PROBE_SMEM_ATOM, "ops/clk/SM"),
                             ("smem_scattered_v2", _abi.PCCP_PROBE_SMEM_DOM, "B/clk/SM")):
        r = pccp_probe(kind)
        out[name] = {"per_clk_per_sm": r["work"] / (r["sm_cycles"] * r["n_sms"]), "unit": unit,
                     "sm_mhz": r["sm_cycles"] / (r["ms"] * 1e3)}
    r = pccp_probe(_abi.PCCP_PROBE_L2_READ)
    out["l2_read"] = {"gbs": r["work"] / (r["ms"] * 1e6), "sm_mhz": r["sm_cycles"] / (r["ms"] * 1e3)}
    return out


# ------------------------------------------------------------------- model

class Model:
    """A created pccp_model (device copy of the packed propagator table)."""

    def __init__(self, lb0, ub0, temporal=None, linear_c=None, linear_off=None, term_coef=None,
                 term_var=None, reified=None, objective=-1, branch=None, bool_store=0):
        """bool_store: 1 keep the Booleans that allow it as bits, -1 as
        intervals, 0 the library's choice (pccp_model_desc.bool_store)."""
        self.lb0 = _i32(lb0)
        self.ub0 = _i32(ub0)
        self.n_vars = len(self.lb0)
        self.temporal = _i32(temporal if temporal is not None else np.zeros((0, 3)), (-1, 3))
        self.reified = _i32(reified if reified is not None else np.zeros((0, 4)), (-1, 4))
        self.linear_c = _i32(linear_c if linear_c is not None else [])
        self.linear_off = _i32(linear_off if linear_off is not None else [0])
        self.term_coef = _i32(term_coef if term_coef is not None else [])
        self.term_var = _i32(term_var if term_var is not None else [])
        self.objective = int(objective)
        self.branch = _i32(branch if branch is not None else [])
        desc = _abi.pccp_model_desc(
            self.n_vars, _ptr(self.lb0), _ptr(self.ub0),
            len(self.temporal), _ptr(self.temporal),
            len(self.linear_c), _ptr(self.linear_c), _ptr(self.linear_off),
            _ptr(self.term_coef), _ptr(self.term_var),
            len(self.reified), _ptr(self.reified),
            self.objective, len(self.branch), _ptr(self.branch), int(bool_store))
        rc, h = pccp_model_create(desc)
        check(rc, "pccp_model_create")
        self.handle = h
        rc, info = pccp_model_get_info(h)
        check(rc, "pccp_model_get_info")
        self.info = info

    @classmethod
    def from_rows(cls, rows, bool_store=0):
        return cls(rows["lb0"], rows["ub0"], rows["temporal"], rows["linear_c"],
                   rows["linear_off"], rows["term_coef"], rows["term_var"], rows["reified"],
                   rows["objective"], rows["branch"], bool_store)

    @classmethod
    def from_rcpsp(cls, inst, bool_store=0):
        return cls.from_rows(rcpsp.build_rows(inst), bool_store)

    @classmethod
    def from_lists(cls, lb0, ub0, temporal=(), linear=(), reified=(), objective=-1, branch=(),
                   bool_store=0):
        """temporal [(x, y, d)], linear [(c, [(coef, var), ...])], reified [(b, x, y, d)]."""
        off = [0]
        coef, var = [], []
        for _, terms in linear:
            for a, v in terms:
                coef.append(a)
                var.append(v)
            off.append(len(coef))
        return cls(lb0, ub0, list(temporal) or np.zeros((0, 3)), [c for c, _ in linear], off,
                   coef, var, list(reified) or np.zeros((0, 4)), objective, list(branch),
                   bool_store)

    @property
    def rows(self) -> int:
        return int(self.info.n_temporal + self.info.n_reified + self.info.n_linear)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            pccp_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------- torch front end

def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _skip(skip_stable):
    """None: the library's choice (0); True: 1; False: -1."""
    return 0 if skip_stable is None else (1 if skip_stable else -1)


def launch_config(team_threads=0, teams_per_cta=0, ctas_per_sm=0, max_iterations=0,
                  skip_stable=None, stream_table=False, temporal_levels=None):
    """stream_table=True streams a table too large for shared memory through
    shared-memory buffers (TMA bulk copies) instead of reading it in place.
    temporal_levels: None the library's choice, True walk the temporal rows
    level by level, False a thread per row."""
    return _abi.pccp_launch_config(team_threads, teams_per_cta, ctas_per_sm, max_iterations,
                                   _skip(skip_stable), int(bool(stream_table)),
                                   _skip(temporal_levels))


def propagate(model: Model, lb, ub, status=None, iterations=None, config=None, stream=None,
              work=None):
    """Propagate the stores in place.  lb/ub: int32 CUDA tensors [n, n_vars]
    (contiguous).  Returns (status, iterations) int32 CUDA tensors [n].
    work: optional int32 CUDA tensor [n, 2] receiving, per store, the rows
    evaluated and the algorithmic bytes they read."""
    import torch
    if lb.dtype != torch.int32 or ub.dtype != torch.int32 or not lb.is_cuda or not ub.is_cuda:
        raise PccpError(PCCP_ERR_INVALID, "lb/ub must be int32 CUDA tensors")
    if not lb.is_contiguous() or not ub.is_contiguous() or lb.shape != ub.shape:
        raise PccpError(PCCP_ERR_INVALID, "lb/ub must be contiguous and of the same shape")
    n = lb.shape[0] if lb.dim() == 2 else 1
    if lb.numel() != n * model.n_vars:
        raise PccpError(PCCP_ERR_INVALID, "store width differs from the model's variables")
    if status is None:
        status = torch.empty(n, dtype=torch.int32, device=lb.device)
    if iterations is None:
        iterations = torch.empty(n, dtype=torch.int32, device=lb.device)
    sp = _stream_ptr(stream)
    wp = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    rc = pccp_propagate_ex(model.handle, n, ctypes.c_void_p(lb.data_ptr()),
                           ctypes.c_void_p(ub.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                           ctypes.c_void_p(iterations.data_ptr()), wp, config, sp)
    check(rc, "pccp_propagate")
    return status, iterations


def pccp_propagate_host(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr, chunk_stores,
                        stream):
    return load().pccp_propagate_host(handle, n_stores, lb_ptr, ub_ptr, status_ptr, iters_ptr,
                                      chunk_stores, stream)


def propagate_host(model: Model, lb, ub, status=None, iterations=None, chunk_stores=0,
                   stream=None):
    """End-to-end form (pccp_propagate_host): HOST int32 tensors [n, n_vars],
    updated in place with the fixed points.  chunk_stores 0 (the library's
    chunking) or > 0 copies them through device slots in chunks that overlap
    the propagation (pin them, e.g. torch.empty(..., pin_memory=True), for
    the overlap); PCCP_HOST_IN_PLACE has the kernel read and write pinned
    tensors where they lie.  Returns (status, iterations), host int32
    tensors [n]."""
    import torch
    if lb.dtype != torch.int32 or ub.dtype != torch.int32 or lb.is_cuda or ub.is_cuda:
        raise PccpError(PCCP_ERR_INVALID, "lb/ub must be int32 host tensors")
    if not lb.is_contiguous() or not ub.is_contiguous() or lb.shape != ub.shape:
        raise PccpError(PCCP_ERR_INVALID, "lb/ub must be contiguous and of the same shape")
    n = lb.shape[0] if lb.dim() == 2 else 1
    if lb.numel() != n * model.n_vars:
        raise PccpError(PCCP_ERR_INVALID, "store width differs from the model's variables")
    pinned = lb.is_pinned()
    if status is None:
        status = torch.empty(n, dtype=torch.int32, pin_memory=pinned)
    if iterations is None:
        iterations = torch.empty(n, dtype=torch.int32, pin_memory=pinned)
    rc = pccp_propagate_host(model.handle, n, ctypes.c_void_p(lb.data_ptr()),
                             ctypes.c_void_p(ub.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                             ctypes.c_void_p(iterations.data_ptr()), chunk_stores,
                             _stream_ptr(stream))
    check(rc, "pccp_propagate_host")
    return status, iterations


def _opts(strategy, mode, deterministic, obj_ub, node_limit, time_limit_ms, threads, blocks,
          skip_stable=None, policy=None, stream_table=False, teams_per_cta=0,
          props_per_thread=0, queue_granularity=0, donate_nodes=0, temporal_levels=None):
    return _abi.pccp_solve_opts(strategy, mode, int(bool(deterministic)), obj_ub, node_limit,
                                time_limit_ms, threads, blocks, _skip(skip_stable),
                                int(bool(stream_table)),
                                policy.handle if policy is not None else None,
                                teams_per_cta, props_per_thread, queue_granularity, donate_nodes,
                                _skip(temporal_levels))


def _result_dict(r, w):
    return {"status": r.status, "has_solution": bool(r.has_solution),
            "objective": int(r.objective) if r.has_solution else None,
            "witness": w.copy() if r.has_solution else None,
            "nodes": int(r.nodes), "fails": int(r.fails), "solutions": int(r.solutions),
            "iterations": int(r.iterations), "rows_evaluated": int(r.rows_evaluated),
            "max_depth": int(r.max_depth), "elapsed_ms": float(r.elapsed_ms),
            "model_ms": float(r.model_ms)}


def solve(model: Model, strategy=PCCP_INPUT_ORDER, mode=PCCP_OPTIMISE, deterministic=True,
          obj_ub=INT32_MAX, node_limit=0, time_limit_ms=0, threads=0, blocks=0, stream=None,
          skip_stable=None, policy=None, stream_table=False, props_per_thread=0,
          queue_granularity=0, donate_nodes=0, temporal_levels=None):
    o = _opts(strategy, mode, deterministic, obj_ub, node_limit, time_limit_ms, threads, blocks,
              skip_stable, policy, stream_table, 0, props_per_thread, queue_granularity,
              donate_nodes, temporal_levels)
    w = np.zeros(model.n_vars, dtype=np.int32)
    r = _abi.pccp_result()
    r.witness = w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    rc = pccp_solve(model.handle, o, r, _stream_ptr(stream))
    check(rc, "pccp_solve")
    return _result_dict(r, w)


def solve_batch(models, strategy=PCCP_INPUT_ORDER, mode=PCCP_OPTIMISE, obj_ub=INT32_MAX,
                node_limit=0, time_limit_ms=0, threads=0, blocks=0, stream=None, noalloc=False,
                skip_stable=None, policy=None, stream_table=False, teams_per_cta=0,
                props_per_thread=0, deterministic=True, queue_granularity=0, donate_nodes=0,
                temporal_levels=None):
    """Solve many models in one launch.  deterministic=True: one team per
    model in the sequential order; False: every team over one shared queue of
    subproblems of all models, with work donation.  noalloc=True uses the
    allocation-free entry point (fixed device scratch; see include/pccp.h)."""
    o = _opts(strategy, mode, deterministic, obj_ub, node_limit, time_limit_ms, threads, blocks,
              skip_stable, policy, stream_table, teams_per_cta, props_per_thread,
              queue_granularity, donate_nodes, temporal_levels)
    n = len(models)
    ws = [np.zeros(m.n_vars, dtype=np.int32) for m in models]
    res = (_abi.pccp_result * n)()
    for i in range(n):
        res[i].witness = ws[i].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    call = pccp_solve_batch_noalloc if noalloc else pccp_solve_batch
    rc = call([m.handle for m in models], o, res, _stream_ptr(stream))
    check(rc, call.__name__)
    return [_result_dict(res[i], ws[i]) for i in range(n)]


class Batch:
    """Models prepared for repeated batched searches; solve_async() only
    queues work on the stream (capturable in a CUDA graph)."""

    def __init__(self, models, threads=0, teams_per_cta=0):
        self.models = list(models)  # keep the models alive
        rc, h = pccp_batch_create([m.handle for m in self.models], threads, teams_per_cta)
        check(rc, "pccp_batch_create")
        self.handle = h
        self._ws = [np.zeros(m.n_vars, dtype=np.int32) for m in self.models]

    @property
    def shape(self):
        """(threads per team, teams per CTA, CTAs) of the planned launch."""
        rc, shp = pccp_batch_get_shape(self.handle)
        check(rc, "pccp_batch_get_shape")
        return shp

    def solve_async(self, strategy=PCCP_INPUT_ORDER, mode=PCCP_OPTIMISE, obj_ub=INT32_MAX,
                    node_limit=0, time_limit_ms=0, stream=None, skip_stable=None, policy=None,
                    deterministic=True, queue_granularity=0, donate_nodes=0,
                    temporal_levels=None):
        o = _opts(strategy, mode, deterministic, obj_ub, node_limit, time_limit_ms, 0, 0,
                  skip_stable, policy, False, 0, 0, queue_granularity, donate_nodes,
                  temporal_levels)
        check(pccp_batch_solve_async(self.handle, o, _stream_ptr(stream)), "pccp_batch_solve_async")

    def results(self, stream=None):
        n = len(self.models)
        res = (_abi.pccp_result * n)()
        for i in range(n):
            res[i].witness = self._ws[i].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        check(pccp_batch_results(self.handle, res, _stream_ptr(stream)), "pccp_batch_results")
        return [_result_dict(res[i], self._ws[i]) for i in range(n)]

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            pccp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- learned branching

def pccp_policy_create(weights):
    h = ctypes.c_void_p()
    rc = load().pccp_policy_create(ctypes.byref(weights), ctypes.byref(h))
    return rc, h


def pccp_policy_destroy(handle):
    load().pccp_policy_destroy(handle)


def pccp_policy_get_weights(handle, w1, b1, w2, b2, w3, b3):
    return load().pccp_policy_get_weights(handle, w1, b1, w2, b2, w3, b3)


def pccp_policy_get_gradients(handle, w1, b1, w2, b2, w3, b3):
    return load().pccp_policy_get_gradients(handle, w1, b1, w2, b2, w3, b3)


def pccp_policy_features(model_handle, n, lb, ub, depth, out, stream):
    return load().pccp_policy_features(model_handle, n, lb, ub, depth, out, stream)


def pccp_policy_score(handle, n, features, scores, stream):
    return load().pccp_policy_score(handle, n, features, scores, stream)


def pccp_policy_train_step(handle, n_rows, features, group_off, n_groups, target, lr, loss, stream):
    return load().pccp_policy_train_step(handle, n_rows, features, group_off, n_groups, target,
                                         lr, loss, stream)


POLICY_SHAPES = {"w1": (128, 12), "b1": (128,), "w2": (128, 128), "b2": (128,), "w3": (128,)}


class Policy:
    """A learned branching policy on the device (MLP 12 -> 128 -> 128 -> 1)."""

    def __init__(self, weights):
        arr = {k: np.ascontiguousarray(np.asarray(weights[k], dtype=np.float32).reshape(shape))
               for k, shape in POLICY_SHAPES.items()}
        self._host = arr
        w = _abi.pccp_policy_weights(*[ctypes.c_void_p(arr[k].ctypes.data)
                                       for k in ("w1", "b1", "w2", "b2", "w3")],
                                     float(weights["b3"]))
        rc, h = pccp_policy_create(w)
        check(rc, "pccp_policy_create")
        self.handle = h

    @classmethod
    def random(cls, seed=0, scale=1.0):
        """He-initialised weights from a seeded generator."""
        g = np.random.default_rng(seed)
        return cls({"w1": g.normal(0, scale * np.sqrt(2 / 12), (128, 12)),
                    "b1": np.zeros(128), "w2": g.normal(0, scale * np.sqrt(2 / 128), (128, 128)),
                    "b2": np.zeros(128), "w3": g.normal(0, scale * np.sqrt(1 / 128), 128),
                    "b3": 0.0})

    def _params(self, call, name):
        out = {k: np.zeros(shape, dtype=np.float32) for k, shape in POLICY_SHAPES.items()}
        b3 = np.zeros(1, dtype=np.float32)
        rc = call(self.handle, *[ctypes.c_void_p(out[k].ctypes.data)
                                 for k in ("w1", "b1", "w2", "b2", "w3")],
                  ctypes.c_void_p(b3.ctypes.data))
        check(rc, name)
        out["b3"] = float(b3[0])
        return out

    def weights(self):
        return self._params(pccp_policy_get_weights, "pccp_policy_get_weights")

    def gradients(self):
        """Gradient of the last training step's mean loss (weight shapes)."""
        return self._params(pccp_policy_get_gradients, "pccp_policy_get_gradients")

    def score(self, features, stream=None):
        """Scores of feature rows (float32 CUDA tensor [n, 12]) -> CUDA tensor [n]."""
        import torch
        f = features.contiguous()
        s = torch.empty(f.shape[0], dtype=torch.float32, device=f.device)
        check(pccp_policy_score(self.handle, f.shape[0], ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(s.data_ptr()), _stream_ptr(stream)),
              "pccp_policy_score")
        return s

    def train_step(self, features, group_off, target, lr=1e-3, stream=None):
        """One Adam step on the mean listwise cross-entropy; returns the loss."""
        loss = ctypes.c_float(0.0)
        f = features.contiguous()
        go = group_off.contiguous()
        t = target.contiguous()
        check(pccp_policy_train_step(self.handle, f.shape[0], ctypes.c_void_p(f.data_ptr()),
                                     ctypes.c_void_p(go.data_ptr()), go.shape[0] - 1,
                                     ctypes.c_void_p(t.data_ptr()), lr, ctypes.byref(loss),
                                     _stream_ptr(stream)), "pccp_policy_train_step")
        return loss.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            pccp_policy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def policy_features(model: Model, lb, ub, depth=None, stream=None):
    """Features [n, n_branch, 12] (float32 CUDA) of stores lb/ub [n, n_vars]."""
    import torch
    n = lb.shape[0]
    out = torch.empty((n, len(model.branch), 12), dtype=torch.float32, device=lb.device)
    dp = ctypes.c_void_p(depth.data_ptr()) if depth is not None else ctypes.c_void_p(0)
    check(pccp_policy_features(model.handle, n, ctypes.c_void_p(lb.data_ptr()),
                               ctypes.c_void_p(ub.data_ptr()), dp, ctypes.c_void_p(out.data_ptr()),
                               _stream_ptr(stream)), "pccp_policy_features")
    return out
