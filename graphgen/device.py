"""The R-MAT generator of graphgen.c written with PyTorch tensor operations, so that graphs too big
for a host-side sort (scale 27: 2.1 billion draws) are drawn, deduplicated and laid out as CSR on
the GPU.  It produces exactly the CSR of graphgen.rmat (same counter-based draws, same weight hash,
rows sorted by target); holds no arithmetic of the Louvain method.

Unsigned 64-bit arithmetic is carried in int64 tensors: additions and multiplications wrap modulo
2^64 like the C code's uint64_t, right shifts are made logical by masking.
"""
from __future__ import annotations

GAMMA = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """The int64 with the same bits as the uint64 x."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(z, s: int):
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix(z):
    z = (z ^ _lsr(z, 30)) * _s64(C1)
    z = (z ^ _lsr(z, 27)) * _s64(C2)
    return z ^ _lsr(z, 31)


def hash3(a, b, c):
    """SplitMix64-chained counter hash of three words (tensors or ints broadcast), as gg_hash3."""
    x = _mix(a + _s64(GAMMA))
    x = _mix(x + b + _s64(2 * GAMMA))
    return _mix(x + c + _s64(3 * GAMMA))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 22,
         fp_weights: bool = False, device="cuda", chunk: int = 1 << 26):
    """(offsets int64 [n+1], targets int32 [A], weights int32 1..8 or float32 (0, 1]) on `device`."""
    import torch
    n = 1 << scale
    draws = edge_factor * n
    t1, t2, t3 = int(65536.0 * a), int(65536.0 * (a + b)), int(65536.0 * (a + b + c))
    sd = torch.tensor(_s64(seed), dtype=torch.int64, device=device)
    keys = []
    for d0 in range(0, draws, chunk):
        d = torch.arange(d0, min(draws, d0 + chunk), dtype=torch.int64, device=device)
        u = torch.zeros_like(d)
        v = torch.zeros_like(d)
        h = None
        for lvl in range(scale):
            if lvl % 4 == 0:
                h = hash3(sd, d, lvl >> 2)
            r = _lsr(h, 16 * (lvl % 4)) & 0xFFFF
            ub = (r >= t2).to(torch.int64)                     # quadrants c and d
            vb = (((r >= t1) & (r < t2)) | (r >= t3)).to(torch.int64)  # quadrants b and d
            u |= ub << (scale - 1 - lvl)
            v |= vb << (scale - 1 - lvl)
            del r, ub, vb
        keep = u != v
        lo = torch.minimum(u, v)[keep]
        hi = torch.maximum(u, v)[keep]
        keys.append((lo << 32) | hi)
        del d, u, v, h, keep, lo, hi
    k = torch.unique(torch.cat(keys)) if keys else torch.zeros(0, dtype=torch.int64, device=device)
    del keys
    return _csr_from_sorted_keys(k, n, seed ^ 0x5BD1E995, fp_weights)


def _csr_from_sorted_keys(k, n: int, wseed: int, fp_weights: bool):
    """CSR of the undirected edges k = (lo << 32) | hi, lo < hi, sorted and unique: both arcs of
    every edge, each row sorted by target (arcs to smaller ids, then to larger ids)."""
    import torch
    dev = k.device
    lo = (k >> 32).to(torch.int32)
    hi = (k & 0xFFFFFFFF).to(torch.int32)
    hw = hash3(torch.tensor(_s64(wseed), dtype=torch.int64, device=dev), lo.to(torch.int64), hi.to(torch.int64))
    if fp_weights:
        w_edge = ((_lsr(hw, 40) + 1).to(torch.float64) * (1.0 / 16777216.0)).to(torch.float32)
    else:
        w_edge = (1 + (hw & 7)).to(torch.int32)
    del hw, k
    n_small = torch.bincount(hi.to(torch.int64), minlength=n)  # arcs of row x to smaller ids
    n_large = torch.bincount(lo.to(torch.int64), minlength=n)  # arcs of row x to larger ids
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(n_small + n_large, 0, out=offsets[1:])
    A = int(offsets[-1])
    targets = torch.empty(A, dtype=torch.int32, device=dev)
    weights = torch.empty(A, dtype=w_edge.dtype, device=dev)
    # arcs to larger ids: row lo, already ordered by (lo, hi)
    E = lo.numel()
    start_lo = torch.zeros(n, dtype=torch.int64, device=dev)
    torch.cumsum(n_large, 0, out=start_lo)
    start_lo -= n_large
    p = torch.arange(E, dtype=torch.int64, device=dev)
    lo64 = lo.to(torch.int64)
    pos = offsets[:-1][lo64] + n_small[lo64] + (p - start_lo[lo64])
    targets[pos] = hi
    weights[pos] = w_edge
    del pos, start_lo, lo64
    # arcs to smaller ids: row hi, ordered by (hi, lo) -- a stable sort by hi keeps lo ascending
    order = torch.sort(hi, stable=True).indices
    hs = hi[order].to(torch.int64)
    start_hi = torch.zeros(n, dtype=torch.int64, device=dev)
    torch.cumsum(n_small, 0, out=start_hi)
    start_hi -= n_small
    pos = offsets[:-1][hs] + (p - start_hi[hs])
    targets[pos] = lo[order]
    weights[pos] = w_edge[order]
    return offsets, targets, weights
