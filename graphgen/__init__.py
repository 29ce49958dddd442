"""Seeded synthetic graph generators (symmetric CSR), shared by the oracle tests and the GPU
path's tests and benchmark.  Holds none of the Louvain method's arithmetic.

The generators stand in for the paper's SuiteSparse graphs (Table 2), which are not shipped:
  * planted-partition SBM (`sbm`), the batched SBM family (`batch_sbm_params` + `sbm`),
  * R-MAT without noise or scrambling (`rmat`), int weights 1..8 or fp32 weights in (0, 1],
  * a road-like perturbed grid (`grid`).
All randomness is the counter hash `hash3(seed, stream, index)` (SplitMix64 output function),
computed in C without libm so that x86-64 and aarch64 hosts produce identical graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libgraphgen.so")

W_UNIT, W_INT8, W_FP32 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile graphgen.c into _build/libgraphgen.so (gcc, -ffp-contract=off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_arcs", ctypes.c_int64),
                ("offsets", ctypes.POINTER(ctypes.c_int64)),
                ("targets", ctypes.POINTER(ctypes.c_int32)),
                ("wi", ctypes.POINTER(ctypes.c_int32)),
                ("wf", ctypes.POINTER(ctypes.c_float)),
                ("n_edges_drawn", ctypes.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_CSR)
        lib.gg_sbm.restype = P
        lib.gg_sbm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_int]
        lib.gg_rmat.restype = P
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.gg_grid.restype = P
        lib.gg_grid.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64]
        lib.gg_free.argtypes = [P]
        lib.gg_free.restype = None
        lib.gg_hash3.restype = ctypes.c_uint64
        lib.gg_hash3.argtypes = [ctypes.c_uint64] * 3
        lib.gg_splitmix64_nth.restype = ctypes.c_uint64
        lib.gg_splitmix64_nth.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_log.restype = ctypes.c_double
        lib.gg_log.argtypes = [ctypes.c_double]
        lib.gg_exp.restype = ctypes.c_double
        lib.gg_exp.argtypes = [ctypes.c_double]
        lib.gg_batch_params.restype = None
        lib.gg_batch_params.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint64)]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Symmetric CSR: offsets int64 [n+1], targets int32 [A], weights int32 or float32 [A]."""
    n: int
    offsets: np.ndarray
    targets: np.ndarray
    weights: np.ndarray
    name: str = ""
    edges_drawn: int = 0

    @property
    def n_arcs(self) -> int:
        return int(self.targets.shape[0])

    @property
    def is_fp(self) -> bool:
        return self.weights.dtype == np.float32

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


def _take(ptr, name: str) -> Graph:
    if not ptr:
        raise MemoryError(f"graph generator {name} failed (bad parameters or out of host memory)")
    lib = _load()
    try:
        c = ptr.contents
        n, a = int(c.n), int(c.n_arcs)
        offs = np.ctypeslib.as_array(c.offsets, shape=(n + 1,)).copy()
        tg = np.ctypeslib.as_array(c.targets, shape=(max(a, 1),))[:a].copy()
        if c.wf:
            w = np.ctypeslib.as_array(c.wf, shape=(max(a, 1),))[:a].copy()
        else:
            w = np.ctypeslib.as_array(c.wi, shape=(max(a, 1),))[:a].copy()
        return Graph(n, offs, tg, w, name, int(c.n_edges_drawn))
    finally:
        lib.gg_free(ptr)


def hash3(a: int, b: int, c: int) -> int:
    return int(_load().gg_hash3(a, b, c))


def splitmix64_nth(seed: int, i: int) -> int:
    return int(_load().gg_splitmix64_nth(seed, i))


def sbm(n: int, k: int, p_in: float, p_out: float, seed: int, weights: int = W_UNIT) -> Graph:
    """Planted-partition SBM; block b = [floor(b n / k), floor((b+1) n / k))."""
    return _take(_load().gg_sbm(n, k, p_in, p_out, seed, weights), f"sbm(n={n},k={k})")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 22, weights: int = W_INT8) -> Graph:
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed, weights), f"rmat(scale={scale})")


def grid(rows: int, cols: int, p_del: float = 0.10, p_long: float = 0.01, seed: int = 3) -> Graph:
    return _take(_load().gg_grid(rows, cols, p_del, p_long, seed), f"grid({rows}x{cols})")


def planted_blocks(n: int, k: int) -> np.ndarray:
    """Block id of every vertex of `sbm(n, k, ...)`."""
    v = np.arange(n, dtype=np.int64)
    # block b holds [floor(b n / k), floor((b+1) n / k)); invert with a search over the bounds
    bounds = (np.arange(k + 1, dtype=np.int64) * n) // k
    return (np.searchsorted(bounds, v, side="right") - 1).astype(np.int32)


def batch_sbm_params(base_seed: int, g: int, n_lo: float = 1e3, n_hi: float = 2e5, k_lo: int = 2,
                     k_hi: int = 64, d_lo: float = 4.0, d_hi: float = 64.0, ratio: float = 0.02):
    """(n, k, p_in, p_out, seed) of member g of the batched SBM family."""
    out = (ctypes.c_double * 4)()
    sd = ctypes.c_uint64()
    _load().gg_batch_params(base_seed, g, n_lo, n_hi, k_lo, k_hi, d_lo, d_hi, ratio, out, ctypes.byref(sd))
    return int(out[0]), int(out[1]), float(out[2]), float(out[3]), int(sd.value)


def batch_sbm(base_seed: int, g: int, **kw) -> Graph:
    n, k, p_in, p_out, seed = batch_sbm_params(base_seed, g, **kw)
    gr = sbm(n, k, p_in, p_out, seed, W_UNIT)
    gr.name = f"batch_sbm[{g}](n={n},k={k})"
    return gr


def from_edges(n: int, edges, weights=None, fp: bool = False) -> Graph:
    """Symmetric CSR from an undirected edge list [(u, v), ...] (self-loops allowed, stored once;
    duplicates must not occur).  Small hand-made test graphs only."""
    arcs = []
    for idx, (u, v) in enumerate(edges):
        w = 1 if weights is None else weights[idx]
        arcs.append((u, v, w))
        if u != v:
            arcs.append((v, u, w))
    arcs.sort()
    offs = np.zeros(n + 1, dtype=np.int64)
    for u, _, _ in arcs:
        offs[u + 1] += 1
    offs = np.cumsum(offs).astype(np.int64)
    tg = np.array([v for _, v, _ in arcs], dtype=np.int32)
    w = np.array([w for _, _, w in arcs], dtype=np.float32 if fp else np.int32)
    return Graph(n, offs, tg, w, "edges")


def concat(graphs):
    """Segmented CSR of a list of graphs: (vo [G + 1] vertex ranges, union row offsets [n + 1],
    graph-LOCAL targets, weights), the input layout of a batched run."""
    G = len(graphs)
    vo = np.zeros(G + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        vo[k + 1] = vo[k] + g.n
    n = int(vo[-1])
    offs = np.zeros(n + 1, dtype=np.int64)
    abase = 0
    for k, g in enumerate(graphs):
        offs[vo[k]:vo[k + 1] + 1] = g.offsets + abase
        abase += g.n_arcs
    tg = np.concatenate([g.targets for g in graphs]) if G else np.zeros(0, np.int32)
    wt = np.concatenate([g.weights for g in graphs]) if G else np.zeros(0, np.int32)
    return vo, offs, tg.astype(np.int32, copy=False), wt


def drop_isolated(g: Graph) -> Graph:
    """The same graph without its isolated vertices (rows with no arc): the others keep their
    order and are renumbered 0..n'-1, so every remaining arc and weight is unchanged."""
    deg = np.diff(g.offsets)
    keep = deg > 0
    newid = (np.cumsum(keep) - 1).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(deg[keep])]).astype(np.int64)
    tg = newid[g.targets].astype(np.int32)
    return Graph(int(keep.sum()), offs, tg, g.weights.copy(), g.name + " (isolated vertices dropped)",
                 g.edges_drawn)


def serving_request(base_seed: int, r: int) -> Graph:
    """Request r of the mixed serving stream: target edge count E log-uniform in [1e4, 2e7]; even
    r: a planted-partition SBM (average degree log-uniform in [4, 64], 2-64 blocks, p_out/p_in =
    0.02, unit weights); odd r: R-MAT (0.57, 0.19, 0.19, 0.05) at scale ceil(log2(E / 16)) with the
    edge factor that makes the draws closest to E, int32 weights 1..8."""
    import math
    u = lambda k: ((hash3(base_seed, r, k) >> 11) + 1) / 9007199254740992.0  # (0, 1]
    E = math.exp(math.log(1e4) + u(1) * (math.log(2e7) - math.log(1e4)))
    seed = hash3(base_seed, r, 0) & 0x7FFFFFFFFFFFFFFF
    if r % 2 == 0:
        d = math.exp(math.log(4.0) + u(2) * (math.log(64.0) - math.log(4.0)))
        n = max(16, int(2.0 * E / d))
        k = 2 + int(hash3(base_seed, r, 3) % 63)
        k = min(k, n)
        s = n / k
        p_in = min(1.0, d / ((s - 1.0) + 0.02 * (n - s)))
        g = sbm(n, k, p_in, 0.02 * p_in, seed, W_UNIT)
        g.name = f"serve_sbm[{r}](n={n},k={k})"
        return g
    scale = max(1, math.ceil(math.log2(E / 16.0)))
    ef = max(1, round(E / (1 << scale)))
    g = rmat(scale, ef, 0.57, 0.19, 0.19, seed, W_INT8)
    g.name = f"serve_rmat[{r}](scale={scale},ef={ef})"
    return g
