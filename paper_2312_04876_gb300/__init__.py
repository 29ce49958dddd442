"""GB300-native Louvain community detection (GVE-Louvain, arXiv 2312.04876).

Python binding of liblouvain.so (include/louvain.h).  Every step of the method runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch supplies device memory
and streams.  If the library is missing the calls raise -- there is no CPU fallback.

    import torch, paper_2312_04876_gb300 as lv
    L = lv.Louvain(device=0)
    membership, result = L.run(offsets, targets, weights, mode="fast")
    result.modularity, result.passes, result.stats   # per-pass statistics in result.stats
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

from . import _native
from ._native import MODE_DETERMINISTIC, MODE_FAST, W_FP32, W_INT32, Params, PassStats, Result

__all__ = ["Louvain", "LouvainError", "Server", "default_params", "MODE_DETERMINISTIC", "MODE_FAST"]


class LouvainError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


def _status_name(s: int) -> str:
    lib = _native.load()
    return lib.louvain_status_string(s).decode()


def default_params(**overrides) -> Params:
    """Defaults of Section 4.1 (louvain_default_params); keyword overrides, mode by name allowed."""
    lib = _native.load()
    p = Params()
    lib.louvain_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "mode" and isinstance(v, str):
            v = {"deterministic": MODE_DETERMINISTIC, "fast": MODE_FAST}[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


STATIC_SCAN_MAX = 1 << 26


def _check_scan_args(values, out):
    """The scan kernels read values[0, n) and write out[0, n]: both must be contiguous int64 CUDA
    tensors on one device, out holding at least n + 1 elements."""
    import torch
    if not isinstance(values, torch.Tensor) or values.dtype != torch.int64 or not values.is_cuda \
            or not values.is_contiguous():
        raise ValueError("values must be a contiguous int64 CUDA tensor")
    if out is not None:
        if not isinstance(out, torch.Tensor) or out.dtype != torch.int64 or not out.is_cuda \
                or not out.is_contiguous() or out.device != values.device:
            raise ValueError("out must be a contiguous int64 CUDA tensor on the device of values")
        if out.numel() < values.numel() + 1:
            raise ValueError(f"out holds {out.numel()} elements; the scan writes {values.numel() + 1}")


def exclusive_scan_static(values, out=None, stream=None):
    """Exclusive scan through louvain_exclusive_scan_static, the entry point that allocates
    nothing (scratch in a fixed device array; at most 2^26 elements; no handle).  For callers that
    cannot call cudaMalloc.  Runs on the device of `values`.  Returns (out int64 tensor of at least
    numel + 1 elements, total)."""
    import torch
    _check_scan_args(values, out)
    lib = _native.load()
    n = values.numel()
    with torch.cuda.device(values.device):
        if out is None:
            out = torch.empty(n + 1, dtype=torch.int64, device=values.device)
        tot = ctypes.c_int64()
        st = lib.louvain_exclusive_scan_static(values.data_ptr(), out.data_ptr(), n, _stream_ptr(stream),
                                               ctypes.byref(tot))
    if st != _native.OK:
        raise LouvainError(st, f"louvain_exclusive_scan_static(count={n}) failed")
    return out, int(tot.value)


class Server:
    """Continuous-batching request loop (louvain_serve_*): host CSRs in, memberships out.

        srv = Server(device=0, hbm_budget_bytes=40 << 30, lanes=4, mode="deterministic")
        t = srv.submit(offsets, targets, weights)        # numpy arrays, kept alive by the server object
        membership, info = srv.result(t)                 # waits; info: modularity, latency_ms, ...

    info also carries where the request's batch spent its time (prep_ms on the host; upload_ms,
    run_ms and download_ms on the device, shared by the batch's graphs).
    """

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 40 << 30, lanes: int = 4,
                 max_batch_graphs: int = 256, max_batch_arcs: int = 0, params: Params | None = None, **overrides):
        self._lib = _native.load()
        self._s = ctypes.c_void_p()
        p = params if params is not None else default_params(**overrides)
        st = self._lib.louvain_serve_create(ctypes.byref(self._s), device, hbm_budget_bytes, lanes, max_batch_graphs,
                                            max_batch_arcs, ctypes.byref(p))
        if st != _native.OK:
            raise LouvainError(st, "louvain_serve_create failed")
        self._keep = {}

    def submit(self, offsets, targets, weights) -> int:
        import numpy as np
        o = np.ascontiguousarray(offsets, dtype=np.int64)
        t = np.ascontiguousarray(targets, dtype=np.int32)
        fp = np.asarray(weights).dtype == np.float32
        w = np.ascontiguousarray(weights, dtype=np.float32 if fp else np.int32)
        n = len(o) - 1
        out = np.empty(max(n, 0), dtype=np.int32)
        tk = ctypes.c_uint64()
        st = self._lib.louvain_serve_submit(self._s, n, len(t), o.ctypes.data, t.ctypes.data, w.ctypes.data,
                                            W_FP32 if fp else W_INT32, out.ctypes.data, ctypes.byref(tk))
        if st != _native.OK:
            raise LouvainError(st, "louvain_serve_submit failed")
        self._keep[tk.value] = (o, t, w, out)
        return tk.value

    def poll(self, ticket: int, wait_ms: int = 0):
        """(membership, info) once finished, else None."""
        r = _native.ServeResult()
        st = self._lib.louvain_serve_poll(self._s, ticket, wait_ms, ctypes.byref(r))
        if st != _native.OK:
            raise LouvainError(st, f"louvain_serve_poll({ticket}) failed")
        if not r.ready:
            return None
        _, _, _, out = self._keep.pop(ticket)
        if r.status != _native.OK:
            raise LouvainError(r.status, f"request {ticket} failed")
        info = dict(modularity=r.result.modularity, passes=r.result.passes,
                    total_iterations=r.result.total_iterations, n_communities=r.result.n_communities,
                    latency_ms=r.latency_ms, queue_ms=r.queue_ms, batch_graphs=r.batch_graphs,
                    prep_ms=r.prep_ms, upload_ms=r.upload_ms, run_ms=r.run_ms, download_ms=r.download_ms)
        return out, info

    def result(self, ticket: int, timeout_s: float = 600.0):
        import time
        t_end = time.monotonic() + timeout_s
        while True:
            got = self.poll(ticket, 200)
            if got is not None:
                return got
            if time.monotonic() > t_end:
                raise TimeoutError(f"request {ticket} not finished after {timeout_s} s")

    def close(self):
        if self._s:
            self._lib.louvain_serve_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class RunResult:
    modularity: float
    passes: int
    total_iterations: int
    n_communities: int
    ms_total: float
    kernel_launches: int
    stats: list = field(default_factory=list)


def _wtype(t) -> int:
    import torch
    if t.dtype == torch.int32:
        return W_INT32
    if t.dtype == torch.float32:
        return W_FP32
    raise TypeError("weights must be int32 or float32")


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _stats_list(st, n) -> list:
    return [dict(pass_=s.pass_, iterations=s.iterations, moves=s.moves, n_vertices=s.n_vertices, n_arcs=s.n_arcs,
                 n_communities=s.n_communities, modularity=s.modularity, ms_colour=s.ms_colour, ms_move=s.ms_move,
                 ms_aggregate=s.ms_aggregate, ms_other=s.ms_other, colours=s.colours,
                 colour_rounds=s.colour_rounds, ms_graph=s.ms_graph,
                 graphs_instantiated=s.graphs_instantiated) for s in st[:n]]


class Louvain:
    """A library handle on one CUDA device (owns the reusable workspace)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._lib = _native.load()
        self._h = ctypes.c_void_p()
        st = self._lib.louvain_create(ctypes.byref(self._h), device, hbm_budget_bytes)
        if st != _native.OK:
            raise LouvainError(st, f"louvain_create(device={device}) failed")
        self.device = device

    def close(self):
        if self._h:
            self._lib.louvain_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        """Device bytes the handle's workspace holds now (louvain_workspace_bytes)."""
        b = ctypes.c_size_t()
        self._check(self._lib.louvain_workspace_bytes(self._h, ctypes.byref(b)))
        return int(b.value)

    def inject_alloc_failure(self, k: int) -> None:
        """Make the k-th device allocation from now fail once (testing the out-of-memory path)."""
        self._check(self._lib.louvain_inject_alloc_failure(self._h, k))

    def _check(self, st: int):
        if st != _native.OK:
            raise LouvainError(st, self._lib.louvain_last_error(self._h).decode())

    # ---------------------------------------------------------------- full method
    def run(self, offsets, targets, weights, params: Params | None = None, membership=None, stream=None,
            stats_cap: int = 64, **overrides):
        """louvain_run on device tensors (int64 offsets, int32 targets, int32/float32 weights).
        Returns (membership int32 tensor, RunResult)."""
        import torch
        p = params if params is not None else default_params(**overrides)
        n = offsets.numel() - 1
        if membership is None:
            membership = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        res = Result()
        st = (PassStats * max(stats_cap, 1))()
        nst = ctypes.c_int32(0)
        rc = self._lib.louvain_run(self._h, n, targets.numel(), offsets.data_ptr(), targets.data_ptr(),
                                   weights.data_ptr(), _wtype(weights), ctypes.byref(p), _stream_ptr(stream),
                                   membership.data_ptr(), ctypes.byref(res), st, stats_cap, ctypes.byref(nst))
        self._check(rc)
        return membership, RunResult(res.modularity, res.passes, res.total_iterations, res.n_communities,
                                     res.ms_total, res.kernel_launches, _stats_list(st, nst.value))

    def run_from(self, offsets, targets, weights, initial, params: Params | None = None, membership=None,
                 stream=None, stats_cap: int = 64, **overrides):
        """louvain_run_from: Algorithm 1 whose first pass starts from the device int32 membership
        `initial` (a warm start after a batch update).  Returns (membership, RunResult)."""
        import torch
        p = params if params is not None else default_params(**overrides)
        n = offsets.numel() - 1
        if initial.dtype != torch.int32 or not initial.is_cuda or not initial.is_contiguous() or initial.numel() != n:
            raise ValueError("initial must be a contiguous int32 CUDA tensor of n entries")
        if membership is None:
            membership = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        res = Result()
        st = (PassStats * stats_cap)()
        ns = ctypes.c_int32()
        rc = self._lib.louvain_run_from(self._h, n, targets.numel(), offsets.data_ptr(), targets.data_ptr(),
                                        weights.data_ptr(), _wtype(weights), ctypes.byref(p), _stream_ptr(stream),
                                        initial.data_ptr(), membership.data_ptr(), ctypes.byref(res), st, stats_cap,
                                        ctypes.byref(ns))
        self._check(rc)
        return membership, RunResult(res.modularity, res.passes, res.total_iterations, res.n_communities,
                                     res.ms_total, res.kernel_launches, _stats_list(st, ns.value))

    def update_graph(self, offsets, targets, weights, n_new: int, deletions, insertions, insert_weights,
                     stream=None):
        """louvain_update_graph: the CSR after deleting the edges `deletions` (int32 [k, 2]) and
        inserting `insertions` (int32 [k, 2]) with `insert_weights`, rows grown to n_new; all device
        tensors.  Returns (offsets, targets, weights) of the updated graph."""
        import torch
        dev = offsets.device
        dl = deletions.reshape(-1, 2).to(dev, torch.int32)
        il = insertions.reshape(-1, 2).to(dev, torch.int32)
        du, dv = dl[:, 0].contiguous(), dl[:, 1].contiguous()
        iu, iv = il[:, 0].contiguous(), il[:, 1].contiguous()
        iw = insert_weights.to(dev, weights.dtype).contiguous()
        cap = targets.numel() + 2 * iu.numel()
        oo = torch.empty(n_new + 1, dtype=torch.int64, device=dev)
        ot = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        ow = torch.empty(max(cap, 1), dtype=weights.dtype, device=dev)
        na = ctypes.c_int64()
        rc = self._lib.louvain_update_graph(self._h, offsets.numel() - 1, targets.numel(), offsets.data_ptr(),
                                            targets.data_ptr(), weights.data_ptr(), _wtype(weights), n_new,
                                            du.numel(), du.data_ptr(), dv.data_ptr(), iu.numel(), iu.data_ptr(),
                                            iv.data_ptr(), iw.data_ptr(), _stream_ptr(stream), oo.data_ptr(),
                                            ot.data_ptr(), ow.data_ptr(), cap, ctypes.byref(na))
        self._check(rc)
        a = int(na.value)
        return oo, ot[:a], ow[:a]

    def run_host(self, offsets, targets, weights, params: Params | None = None, membership=None, stream=None,
                 stats_cap: int = 64, **overrides):
        """louvain_run_host on host arrays (numpy or CPU tensors; pinned memory is fastest)."""
        import numpy as np
        p = params if params is not None else default_params(**overrides)

        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        n = (offsets.numel() if hasattr(offsets, "numel") else len(offsets)) - 1
        na = targets.numel() if hasattr(targets, "numel") else len(targets)
        wdt = weights.dtype
        fp = str(wdt) in ("torch.float32", "float32")
        if membership is None:
            membership = np.empty(max(n, 0), dtype=np.int32)
        res = Result()
        st = (PassStats * max(stats_cap, 1))()
        nst = ctypes.c_int32(0)
        rc = self._lib.louvain_run_host(self._h, n, na, ptr(offsets), ptr(targets), ptr(weights),
                                        W_FP32 if fp else W_INT32, ctypes.byref(p), _stream_ptr(stream),
                                        ptr(membership), ctypes.byref(res), st, stats_cap, ctypes.byref(nst))
        self._check(rc)
        return membership, RunResult(res.modularity, res.passes, res.total_iterations, res.n_communities,
                                     res.ms_total, res.kernel_launches, _stats_list(st, nst.value))

    def run_batch(self, graph_vtx_offs, offsets, targets, weights, params: Params | None = None, membership=None,
                  stream=None, **overrides):
        """louvain_run_batch: many graphs in one union (segmented CSR).  graph_vtx_offs: host int64
        sequence [G + 1]; offsets: device int64 union row offsets [n + 1]; targets: device int32
        graph-LOCAL ids; weights: device int32/float32.  Returns (membership int32 tensor with
        graph-local ids, list of per-graph dicts, RunResult of the whole call)."""
        import numpy as np
        import torch
        p = params if params is not None else default_params(**overrides)
        vo = np.ascontiguousarray(np.asarray(graph_vtx_offs, dtype=np.int64))
        G = len(vo) - 1
        n = int(vo[-1]) if G >= 0 and len(vo) else 0
        if membership is None:
            membership = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        per = (_native.GraphResult * max(G, 1))()
        res = Result()
        rc = self._lib.louvain_run_batch(self._h, G, vo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         targets.numel(), offsets.data_ptr(), targets.data_ptr(), weights.data_ptr(),
                                         _wtype(weights), ctypes.byref(p), _stream_ptr(stream), membership.data_ptr(),
                                         per, ctypes.byref(res))
        self._check(rc)
        graphs = [dict(modularity=r.modularity, passes=r.passes, total_iterations=r.total_iterations,
                       n_communities=r.n_communities) for r in per[:G]]
        return membership, graphs, RunResult(res.modularity, res.passes, res.total_iterations, res.n_communities,
                                             res.ms_total, res.kernel_launches)

    def autotune(self, offsets, targets, weights, params: Params | None = None, reps: int = 1, stream=None,
                 **overrides):
        """louvain_autotune: (tuned Params, best ms) for this graph."""
        import torch
        p = params if params is not None else default_params(**overrides)
        n = offsets.numel() - 1
        mem = torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
        out = Params()
        ms = ctypes.c_float()
        rc = self._lib.louvain_autotune(self._h, n, targets.numel(), offsets.data_ptr(), targets.data_ptr(),
                                        weights.data_ptr(), _wtype(weights), ctypes.byref(p), _stream_ptr(stream),
                                        mem.data_ptr(), reps, ctypes.byref(out), ctypes.byref(ms))
        self._check(rc)
        return out, float(ms.value)

    def autotune_batch(self, graph_vtx_offs, offsets, targets, weights, params: Params | None = None, reps: int = 1,
                       stream=None, **overrides):
        """louvain_autotune_batch: (tuned Params, best ms) for this batch."""
        import numpy as np
        import torch
        p = params if params is not None else default_params(**overrides)
        vo = np.ascontiguousarray(np.asarray(graph_vtx_offs, dtype=np.int64))
        n = int(vo[-1])
        mem = torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
        out = Params()
        ms = ctypes.c_float()
        rc = self._lib.louvain_autotune_batch(self._h, len(vo) - 1, vo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              targets.numel(), offsets.data_ptr(), targets.data_ptr(),
                                              weights.data_ptr(), _wtype(weights), ctypes.byref(p),
                                              _stream_ptr(stream), mem.data_ptr(), reps, ctypes.byref(out),
                                              ctypes.byref(ms))
        self._check(rc)
        return out, float(ms.value)

    # ---------------------------------------------------------------- steps
    def modularity(self, offsets, targets, weights, membership, stream=None) -> float:
        q = ctypes.c_double()
        rc = self._lib.louvain_modularity(self._h, offsets.numel() - 1, targets.numel(), offsets.data_ptr(),
                                          targets.data_ptr(), weights.data_ptr(), _wtype(weights),
                                          membership.data_ptr(), _stream_ptr(stream), ctypes.byref(q))
        self._check(rc)
        return float(q.value)

    def colour(self, offsets, targets, seed: int, pass_index: int, stream=None):
        import torch
        n = offsets.numel() - 1
        col = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        nc = ctypes.c_int32()
        rc = self._lib.louvain_colour(self._h, n, targets.numel(), offsets.data_ptr(), targets.data_ptr(), seed,
                                      pass_index, _stream_ptr(stream), col.data_ptr(), ctypes.byref(nc))
        self._check(rc)
        return col, int(nc.value)

    def local_move(self, offsets, targets, weights, params: Params | None = None, pass_index: int = 0,
                   tau: float | None = None, stream=None, **overrides):
        import torch
        p = params if params is not None else default_params(**overrides)
        n = offsets.numel() - 1
        cp = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        it = ctypes.c_int32()
        mv = ctypes.c_int64()
        rc = self._lib.louvain_local_move(self._h, n, targets.numel(), offsets.data_ptr(), targets.data_ptr(),
                                          weights.data_ptr(), _wtype(weights), ctypes.byref(p), pass_index,
                                          p.tolerance if tau is None else tau, _stream_ptr(stream), cp.data_ptr(),
                                          ctypes.byref(it), ctypes.byref(mv))
        self._check(rc)
        return cp, int(it.value), int(mv.value)

    def aggregate(self, offsets, targets, weights, membership, n_comm: int, stream=None):
        import torch
        dev = offsets.device
        oo = torch.empty(n_comm + 1, dtype=torch.int64, device=dev)
        ot = torch.empty(max(targets.numel(), 1), dtype=torch.int32, device=dev)
        ow = torch.empty(max(targets.numel(), 1), dtype=weights.dtype, device=dev)
        na = ctypes.c_int64()
        rc = self._lib.louvain_aggregate(self._h, offsets.numel() - 1, targets.numel(), offsets.data_ptr(),
                                         targets.data_ptr(), weights.data_ptr(), _wtype(weights),
                                         membership.data_ptr(), n_comm, _stream_ptr(stream), oo.data_ptr(),
                                         ot.data_ptr(), ow.data_ptr(), ctypes.byref(na))
        self._check(rc)
        a = int(na.value)
        return oo, ot[:a], ow[:a]

    def kernel_profile(self) -> list:
        """Per-kernel-class totals of the last run made with profile=1: name, launches, ms,
        algorithmic bytes and the achieved GB/s those imply."""
        cap = 32
        arr = (_native.KernelStat * cap)()
        n = ctypes.c_int32()
        self._check(self._lib.louvain_kernel_profile(self._h, arr, cap, ctypes.byref(n)))
        out = []
        for k in arr[:n.value]:
            gbs = k.algorithmic_bytes / (k.ms * 1e6) if k.ms > 0 else 0.0
            out.append(dict(name=k.name.decode(), launches=k.launches, ms=k.ms, bytes=k.algorithmic_bytes,
                            gbs=gbs))
        return out

    def exclusive_scan(self, values, stream=None):
        import torch
        _check_scan_args(values, None)
        if values.device != torch.device("cuda", self.device):
            raise ValueError(f"values live on {values.device}; this handle runs on cuda:{self.device}")
        out = torch.empty(values.numel() + 1, dtype=torch.int64, device=values.device)
        tot = ctypes.c_int64()
        rc = self._lib.louvain_exclusive_scan(self._h, values.data_ptr(), out.data_ptr(), values.numel(),
                                              _stream_ptr(stream), ctypes.byref(tot))
        self._check(rc)
        return out, int(tot.value)
