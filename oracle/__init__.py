"""CPU oracle for the PCCP propagate-and-search method -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package.  The CUDA product path never imports
it and shares no code with it.

The arithmetic lives in pccp_oracle.c (plain sequential C, int64); this module
only marshals numpy arrays through ctypes.  See pccp_oracle.c for the passages
of the paper each function follows.  rcpsp.py is the oracle's own expansion of
a scheduling instance into constraints; brute.py holds brute-force
enumerators that pin the oracle without using propagation at all.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pccp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FORWARD, REVERSE, RANDOM, JACOBI = 0, 1, 2, 3
FIXPOINT, FAILED, NONTERMINATING = 0, 1, 2
OPTIMISE, COUNT_ALL = 0, 1
INPUT_ORDER, FIRST_FAIL = 0, 1
RES_OPTIMAL, RES_INFEASIBLE, RES_LIMIT = 0, 1, 2
TELL_NONE, TELL_LB, TELL_UB = 0, 1, 2
INT64_MAX = (1 << 63) - 1


def build(force: bool = False) -> str:
    """Compile pccp_oracle.c with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("n_vars", ctypes.c_int32), ("lb0", ctypes.c_void_p), ("ub0", ctypes.c_void_p),
        ("n_temporal", ctypes.c_int32), ("t_x", ctypes.c_void_p), ("t_y", ctypes.c_void_p),
        ("t_d", ctypes.c_void_p),
        ("n_reified", ctypes.c_int32), ("r_b", ctypes.c_void_p), ("r_x", ctypes.c_void_p),
        ("r_y", ctypes.c_void_p), ("r_d", ctypes.c_void_p),
        ("n_linear", ctypes.c_int32), ("l_c", ctypes.c_void_p), ("l_off", ctypes.c_void_p),
        ("l_var", ctypes.c_void_p), ("l_coef", ctypes.c_void_p),
        ("objective", ctypes.c_int32), ("n_branch", ctypes.c_int32), ("branch", ctypes.c_void_p),
    ]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("strategy", ctypes.c_int32),
                ("node_limit", ctypes.c_int64), ("obj_ub", ctypes.c_int64)]


class _SolveResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("has_solution", ctypes.c_int32),
                ("objective", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("fails", ctypes.c_int64), ("solutions", ctypes.c_int64),
                ("sweeps", ctypes.c_int64), ("max_depth", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point the wrapper at a deliberately broken build of the
            # oracle to check that the pins catch it
            override = os.environ.get("PCCP_ORACLE_LIB")
            lib = ctypes.CDLL(override if override else build())
            P = ctypes.c_void_p
            lib.om_propagate.argtypes = [P, P, P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, P]
            lib.om_propagate.restype = ctypes.c_int
            lib.om_propagate_batch.argtypes = [P, ctypes.c_int64, P, P, P, P]
            lib.om_propagate_batch.restype = None
            lib.om_command_count.argtypes = [P]
            lib.om_command_count.restype = ctypes.c_int64
            lib.om_command.argtypes = [P, P, P, ctypes.c_int64, P, P]
            lib.om_command.restype = ctypes.c_int
            lib.om_solve.argtypes = [P, P, P, P]
            lib.om_solve.restype = ctypes.c_int
            lib.om_solve_traced.argtypes = [P, P, P, P, P, ctypes.c_int64, P]
            lib.om_solve_traced.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


class Model:
    """A constraint model as the oracle sees it (plain arrays, int64 values).

    temporal: (x, y, d) meaning x + d <= y
    linear:   (c, [(coef, var), ...]) meaning sum coef*var <= c
    reified:  (b, x, y, d) meaning b <=> (x <= y and y < x + d)
    """

    def __init__(self, lb0, ub0, temporal=(), linear=(), reified=(), objective=-1, branch=()):
        self.lb0 = _i64(lb0)
        self.ub0 = _i64(ub0)
        self.n_vars = len(self.lb0)
        temporal = list(temporal)
        reified = list(reified)
        linear = [(c, [(a, v) for (a, v) in terms if a != 0]) for (c, terms) in linear]
        self.temporal = temporal
        self.reified = reified
        self.linear = linear
        self.t_x = _i32([t[0] for t in temporal])
        self.t_y = _i32([t[1] for t in temporal])
        self.t_d = _i64([t[2] for t in temporal])
        self.r_b = _i32([r[0] for r in reified])
        self.r_x = _i32([r[1] for r in reified])
        self.r_y = _i32([r[2] for r in reified])
        self.r_d = _i64([r[3] for r in reified])
        off = [0]
        for _, terms in linear:
            off.append(off[-1] + len(terms))
        self.l_c = _i64([c for c, _ in linear])
        self.l_off = _i32(off)
        self.l_var = _i32([v for _, terms in linear for (_, v) in terms])
        self.l_coef = _i64([a for _, terms in linear for (a, _) in terms])
        self.objective = int(objective)
        self.branch = _i32(list(branch))
        p = lambda a: a.ctypes.data if a.size else None
        self._c = _Model(self.n_vars, p(self.lb0), p(self.ub0),
                         len(temporal), p(self.t_x), p(self.t_y), p(self.t_d),
                         len(reified), p(self.r_b), p(self.r_x), p(self.r_y), p(self.r_d),
                         len(linear), p(self.l_c), self.l_off.ctypes.data, p(self.l_var),
                         p(self.l_coef), self.objective, len(self.branch), p(self.branch))

    @property
    def cptr(self):
        return ctypes.addressof(self._c)

    def root(self):
        return self.lb0.copy(), self.ub0.copy()

    def command_count(self) -> int:
        return int(_load().om_command_count(self.cptr))


def sweep_bound(model: Model) -> int:
    """Every sweep that changes the store narrows some bound by at least one
    and a failure is caught at the tell that empties a domain, so a run needs
    at most (total width of the root box) + 2 sweeps."""
    return int(np.sum(model.ub0 - model.lb0 + 1)) + 2


def propagate(model: Model, lb, ub, order: int = FORWARD, seed: int = 0,
              max_sweeps: int = None):
    """Least fixed point above (lb, ub) join root.  Returns
    (status, lb, ub, sweeps); lb/ub are new int64 arrays."""
    lib = _load()
    if max_sweeps is None:
        max_sweeps = sweep_bound(model)
    lb = _i64(lb).copy()
    ub = _i64(ub).copy()
    sw = ctypes.c_int64(0)
    st = lib.om_propagate(model.cptr, lb.ctypes.data, ub.ctypes.data, order,
                          seed & ((1 << 64) - 1), max_sweeps, ctypes.addressof(sw))
    return st, lb, ub, sw.value


def propagate_batch(model: Model, lb, ub):
    """Forward-order fixed points of a batch; lb/ub are [n, n_vars] arrays.
    Returns (status int32[n], lb, ub, sweeps int64[n]).  Releases the GIL."""
    lib = _load()
    lb = np.ascontiguousarray(np.asarray(lb, dtype=np.int64)).copy()
    ub = np.ascontiguousarray(np.asarray(ub, dtype=np.int64)).copy()
    n = lb.shape[0]
    status = np.zeros(n, dtype=np.int32)
    sweeps = np.zeros(n, dtype=np.int64)
    lib.om_propagate_batch(model.cptr, n, lb.ctypes.data, ub.ctypes.data,
                           status.ctypes.data, sweeps.ctypes.data)
    return status, lb, ub, sweeps


def command(model: Model, lb, ub, g: int):
    """Evaluate guarded command g once on (lb, ub): (kind, var, value)."""
    lib = _load()
    lb = _i64(lb)
    ub = _i64(ub)
    var = ctypes.c_int32(0)
    val = ctypes.c_int64(0)
    kind = lib.om_command(model.cptr, lb.ctypes.data, ub.ctypes.data, g,
                          ctypes.addressof(var), ctypes.addressof(val))
    return kind, var.value, val.value


NODE_FAILED, NODE_SOLUTION, NODE_BRANCH = 0, 1, 2
TRACE_FIELDS = 6


def solve(model: Model, mode: int = OPTIMISE, strategy: int = INPUT_ORDER,
          node_limit: int = 0, obj_ub: int = INT64_MAX, trace_cap: int = 0):
    """Depth-first branch and bound.  Returns a dict with status, objective,
    witness (lb of the recorded solution), nodes, fails, solutions, sweeps.
    With trace_cap > 0 it also returns "trace": the first trace_cap nodes in
    depth-first preorder, each (depth, decision var, side, value, outcome,
    chosen var): the decision that created the node (var -1 for the root;
    side 0 = left, ub <= value; 1 = right, lb >= value), the node's outcome
    (NODE_FAILED / NODE_SOLUTION / NODE_BRANCH) and the variable it
    branches on (-1 unless it branches)."""
    lib = _load()
    o = _SolveOpts(mode, strategy, node_limit, obj_ub)
    r = _SolveResult()
    w = np.zeros(max(model.n_vars, 1), dtype=np.int64)
    tr = np.zeros((max(trace_cap, 1), TRACE_FIELDS), dtype=np.int64)
    tn = ctypes.c_int64(0)
    if trace_cap > 0:
        rc = lib.om_solve_traced(model.cptr, ctypes.addressof(o), ctypes.addressof(r),
                                 w.ctypes.data, tr.ctypes.data, trace_cap, ctypes.addressof(tn))
    else:
        rc = lib.om_solve(model.cptr, ctypes.addressof(o), ctypes.addressof(r), w.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle search aborted (code {rc})")
    out = {
        "status": r.status, "has_solution": bool(r.has_solution),
        "objective": int(r.objective) if r.has_solution else None,
        "witness": w[: model.n_vars].copy() if r.has_solution else None,
        "nodes": int(r.nodes), "fails": int(r.fails), "solutions": int(r.solutions),
        "sweeps": int(r.sweeps), "max_depth": int(r.max_depth),
    }
    if trace_cap > 0:
        out["trace"] = [tuple(int(x) for x in row) for row in tr[: min(tn.value, trace_cap)]]
        out["trace_nodes"] = int(tn.value)
    return out
