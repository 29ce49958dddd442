"""CPU oracle for the Louvain method -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded statement of GVE-Louvain's Algorithms 1-3 with Eqs. 1-2
(see louvain_oracle.cpp for the readings of every point the paper leaves open).  Only tests/,
`__graft_entry__.smoke()` and the benchmark's CPU-baseline / reference leg may import this
package; the GPU library never does, and the two share no code.

Parity status of each function (what pins it lives in tests/test_oracle_pins.py):
  modularity ........ pinned (brute-force pair sum, networkx, closed forms of clique families)
  move_score ........ pinned (exact Delta Q from Eq. 1 before/after every single-vertex move)
  colour ............ pinned (properness; complete graphs; brute-force greedy on tiny graphs)
  aggregate ......... pinned (numpy scatter-add of community pairs; Q invariance; 2m invariance)
  local_move/louvain  pinned (brute-force optimum on <= 9 vertices; clique rings; planted SBM;
                      hand-traced two-vertex/triangle cases; the karate club's published optimum;
                      tolerance limits and the single-move optimum at tolerance 0; hand-traced
                      ties, zero-gain moves and same-iteration eligibility)
  update_graph ...... pinned (an edge dictionary rebuilt independently in Python)
  louvain_from ...... pinned (singleton start = the cold run; clique partitions of clique rings are
                      fixed points; one community cannot split; the sequential schedule never ends
                      below the modularity it started from; a warm start after a small update of
                      a planted partition keeps the cold run's quality)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "louvain_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
# A test that plants a mistake in a copy of the oracle points this variable at the copy's build.
_SO_OVERRIDE = os.environ.get("LOUVAIN_ORACLE_SO")

SCHEDULE_COLOUR_SYNC = 0
SCHEDULE_SEQUENTIAL = 1


def build(force: bool = False) -> str:
    """Compile louvain_oracle.cpp into _build/liboracle.so (g++ -O2, no OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("max_passes", ctypes.c_int32), ("max_iterations", ctypes.c_int32),
                ("tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("pruning", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class PassStats(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int32), ("iterations", ctypes.c_int32), ("moves", ctypes.c_int64),
                ("n_vertices", ctypes.c_int64), ("n_arcs", ctypes.c_int64),
                ("n_communities", ctypes.c_int64), ("modularity", ctypes.c_double)]


def default_params(**kw) -> Params:
    """The paper's settings (Section 4.1): 20 iterations per pass, tolerance 0.01 dropped 10x per
    pass, aggregation tolerance 0.8, pruning on; MAX_PASSES (unstated) read as 10."""
    p = Params(max_passes=10, max_iterations=20, tolerance=1e-2, tolerance_drop=10.0,
               aggregation_tolerance=0.8, pruning=1, schedule=SCHEDULE_COLOUR_SYNC, seed=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_SO_OVERRIDE or build())
        lib.oracle_hash3.restype = ctypes.c_uint64
        lib.oracle_hash3.argtypes = [ctypes.c_uint64] * 3
        lib.oracle_modularity.restype = ctypes.c_double
        lib.oracle_modularity.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, _P]
        lib.oracle_move_score_int.restype = ctypes.c_int64
        lib.oracle_move_score_int.argtypes = [ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_colour.restype = ctypes.c_int
        lib.oracle_colour.argtypes = [ctypes.c_int64, _P, _P, ctypes.c_uint64, ctypes.c_int32, _P, _P]
        lib.oracle_aggregate.restype = ctypes.c_int64
        lib.oracle_aggregate.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int64, _P, _P, _P,
                                         ctypes.c_int64]
        lib.oracle_local_move.restype = ctypes.c_int
        lib.oracle_local_move.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, ctypes.POINTER(Params),
                                          ctypes.c_int32, ctypes.c_double, _P, _P, _P]
        lib.oracle_louvain.restype = ctypes.c_int
        lib.oracle_louvain.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, ctypes.POINTER(Params), _P, _P, _P,
                                       ctypes.POINTER(PassStats), ctypes.c_int32]
        lib.oracle_update_graph.restype = ctypes.c_int64
        lib.oracle_update_graph.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                            _P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_int64]
        lib.oracle_louvain_from.restype = ctypes.c_int
        lib.oracle_louvain_from.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_int, ctypes.POINTER(Params), _P, _P,
                                            _P, _P, ctypes.POINTER(PassStats), ctypes.c_int32]
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _graph_args(offsets, targets, weights):
    offs = _c(offsets, np.int64)
    tg = _c(targets, np.int32)
    fp = np.asarray(weights).dtype.kind == "f"
    w = _c(weights, np.float32 if fp else np.int32)
    return offs, tg, w, int(fp)


def hash3(a: int, b: int, c: int) -> int:
    return int(_load().oracle_hash3(a, b, c))


def modularity(offsets, targets, weights, membership) -> float:
    """Eq. 1 with membership ids in [0, n); exact integer arithmetic for int32 weights."""
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    m = _c(membership, np.int32)
    q = _load().oracle_modularity(len(offs) - 1, _ptr(offs), _ptr(tg), _ptr(w), fp, _ptr(m))
    if q == -2.0:
        raise ValueError("invalid graph or membership")
    return float(q)


def move_score(offsets, targets, weights, membership, i: int, c: int) -> int:
    """Eq. 2 numerator N (Delta Q = 2N / (2m)^2) for moving i from its community to c."""
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    assert not fp
    m = _c(membership, np.int32)
    return int(_load().oracle_move_score_int(len(offs) - 1, _ptr(offs), _ptr(tg), _ptr(w), _ptr(m), i, c))


def colour(offsets, targets, seed: int, pass_index: int):
    offs = _c(offsets, np.int64)
    tg = _c(targets, np.int32)
    n = len(offs) - 1
    col = np.empty(n, dtype=np.int32)
    nc = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_colour(n, _ptr(offs), _ptr(tg), seed, pass_index, _ptr(col), _ptr(nc))
    if rc:
        raise ValueError("invalid graph")
    return col, int(nc[0])


def aggregate(offsets, targets, weights, membership, n_comm: int):
    """Super-vertex graph for a dense membership; rows sorted by target.  Weights int64 / float64."""
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    m = _c(membership, np.int32)
    cap = max(len(tg), 1)
    oo = np.empty(n_comm + 1, dtype=np.int64)
    ot = np.empty(cap, dtype=np.int32)
    ow = np.empty(cap, dtype=np.float64 if fp else np.int64)
    a = _load().oracle_aggregate(len(offs) - 1, _ptr(offs), _ptr(tg), _ptr(w), fp, _ptr(m), n_comm, _ptr(oo),
                                 _ptr(ot), _ptr(ow), cap)
    if a < 0:
        raise ValueError("invalid aggregation input")
    return oo, ot[:a].copy(), ow[:a].copy()


def local_move(offsets, targets, weights, params: Params | None = None, pass_index: int = 0,
               tau: float | None = None):
    """One local-moving phase from singletons: (C' not renumbered, iterations, moves)."""
    p = params or default_params()
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    n = len(offs) - 1
    cp = np.empty(n, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    mv = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_local_move(n, _ptr(offs), _ptr(tg), _ptr(w), fp, ctypes.byref(p), pass_index,
                                   p.tolerance if tau is None else tau, _ptr(cp), _ptr(it), _ptr(mv))
    if rc:
        raise ValueError(f"oracle_local_move failed ({rc})")
    return cp, int(it[0]), int(mv[0])


def update_graph(offsets, targets, weights, n_new: int, deletions, insertions, insert_weights):
    """Batch update of a symmetric CSR: deleted edges {u, v} lose every arc between u and v, then each
    inserted edge (u, v) adds u->v and v->u (one arc for a self-loop) with its weight; rows may grow
    to n_new.  Row r: surviving arcs in their old order, then inserted arcs in list order."""
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    d = np.asarray(deletions, dtype=np.int32).reshape(-1, 2)
    ins = np.asarray(insertions, dtype=np.int32).reshape(-1, 2)
    du, dv = _c(d[:, 0], np.int32), _c(d[:, 1], np.int32)
    iu, iv = _c(ins[:, 0], np.int32), _c(ins[:, 1], np.int32)
    iw = _c(insert_weights, np.float32 if fp else np.int32)
    cap = len(tg) + 2 * len(iu) + 1
    oo = np.empty(n_new + 1, dtype=np.int64)
    ot = np.empty(cap, dtype=np.int32)
    ow = np.empty(cap, dtype=np.float32 if fp else np.int32)
    a = _load().oracle_update_graph(len(offs) - 1, _ptr(offs), _ptr(tg), _ptr(w), fp, n_new, len(du), _ptr(du),
                                    _ptr(dv), len(iu), _ptr(iu), _ptr(iv), _ptr(iw), _ptr(oo), _ptr(ot), _ptr(ow), cap)
    if a < 0:
        raise ValueError("invalid update")
    return oo, ot[:a].copy(), ow[:a].copy()


def louvain_from(offsets, targets, weights, initial, params: Params | None = None, stats_cap: int = 128):
    """Algorithm 1 with the first pass starting from the membership `initial` (a warm start)."""
    p = params or default_params()
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    n = len(offs) - 1
    init = _c(initial, np.int32)
    mem = np.empty(n, dtype=np.int32)
    q = np.zeros(1, dtype=np.float64)
    np_ = np.zeros(1, dtype=np.int32)
    st = (PassStats * stats_cap)()
    rc = _load().oracle_louvain_from(n, _ptr(offs), _ptr(tg), _ptr(w), fp, ctypes.byref(p), _ptr(init), _ptr(mem),
                                     _ptr(q), _ptr(np_), st, stats_cap)
    if rc == 3:
        raise OverflowError("integer 2m >= 2^31")
    if rc:
        raise ValueError(f"oracle_louvain_from failed ({rc})")
    passes = int(np_[0])
    stats = [dict(pass_=s.pass_, iterations=s.iterations, moves=s.moves, n_vertices=s.n_vertices, n_arcs=s.n_arcs,
                  n_communities=s.n_communities, modularity=s.modularity) for s in st[:min(passes, stats_cap)]]
    return mem, float(q[0]), passes, stats


def louvain(offsets, targets, weights, params: Params | None = None, stats_cap: int = 128):
    """Algorithm 1: (membership, modularity, passes, [per-pass stats dicts])."""
    p = params or default_params()
    offs, tg, w, fp = _graph_args(offsets, targets, weights)
    n = len(offs) - 1
    mem = np.empty(n, dtype=np.int32)
    q = np.zeros(1, dtype=np.float64)
    np_ = np.zeros(1, dtype=np.int32)
    st = (PassStats * stats_cap)()
    rc = _load().oracle_louvain(n, _ptr(offs), _ptr(tg), _ptr(w), fp, ctypes.byref(p), _ptr(mem), _ptr(q), _ptr(np_),
                                st, stats_cap)
    if rc == 3:
        raise OverflowError("integer 2m >= 2^31")
    if rc:
        raise ValueError(f"oracle_louvain failed ({rc})")
    passes = int(np_[0])
    stats = [dict(pass_=s.pass_, iterations=s.iterations, moves=s.moves, n_vertices=s.n_vertices, n_arcs=s.n_arcs,
                  n_communities=s.n_communities, modularity=s.modularity) for s in st[:min(passes, stats_cap)]]
    return mem, float(q[0]), passes, stats
