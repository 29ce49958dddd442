"""Independent test-side statements used to pin the oracle and check GPU results.

Nothing here calls the oracle or the GPU library: these are the definitions written out a
second, differently-structured way (pair sums, dense matrices, brute-force enumeration).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np

import graphgen as gg


def dense_adjacency(g) -> np.ndarray:
    """Dense symmetric matrix A[i, j] = weight of arc i->j (self-loop once on the diagonal)."""
    a = np.zeros((g.n, g.n), dtype=np.float64 if g.is_fp else np.int64)
    for i in range(g.n):
        for e in range(g.offsets[i], g.offsets[i + 1]):
            a[i, g.targets[e]] += g.weights[e]
    return a


def q_pairsum(a: np.ndarray, membership) -> float:
    """Newman's pair-sum form of Eq. 1 over ALL ordered pairs:
    Q = 1/2m sum_ij [A_ij - K_i K_j / 2m] delta(C_i, C_j)."""
    m = np.asarray(membership)
    k = a.sum(axis=1).astype(np.float64)
    two_m = float(a.sum())
    same = (m[:, None] == m[None, :])
    return float(((a - np.outer(k, k) / two_m) * same).sum() / two_m)


def q_exact(a: np.ndarray, membership) -> Fraction:
    """Eq. 1 as an exact rational from an integer matrix (pair-sum form)."""
    m = list(membership)
    n = a.shape[0]
    k = [int(a[i].sum()) for i in range(n)]
    two_m = sum(k)
    tot = Fraction(0)
    for i in range(n):
        for j in range(n):
            if m[i] == m[j]:
                tot += Fraction(int(a[i, j])) - Fraction(k[i] * k[j], two_m)
    return tot / two_m


def set_partitions(n: int):
    """All set partitions of range(n) as restricted-growth strings (Bell(n) of them)."""
    out = []
    rgs = [0] * n

    def rec(i, mx):
        if i == n:
            out.append(list(rgs))
            return
        for v in range(mx + 2):
            rgs[i] = v
            rec(i + 1, max(mx, v))

    if n == 0:
        return [[]]
    rgs[0] = 0
    rec(1, 0)
    return out


def brute_force_max_q(a: np.ndarray) -> float:
    """Maximum of Eq. 1 over every partition (vectorised pair-sum)."""
    n = a.shape[0]
    parts = np.array(set_partitions(n), dtype=np.int32)
    k = a.sum(axis=1).astype(np.float64)
    two_m = float(a.sum())
    b = (a - np.outer(k, k) / two_m) / two_m
    best = -1.0
    for chunk in np.array_split(parts, max(1, len(parts) // 4096)):
        same = chunk[:, :, None] == chunk[:, None, :]
        q = (same * b[None]).sum(axis=(1, 2))
        best = max(best, float(q.max()))
    return best


def random_graph(n: int, p: float, rng, weights: str = "int", self_loops: bool = False):
    edges, ws = [], []
    for u, v in combinations(range(n), 2):
        if rng.random() < p:
            edges.append((u, v))
            ws.append(int(rng.integers(1, 9)) if weights == "int" else float(rng.uniform(0.05, 1.0)))
    if self_loops:
        for u in range(n):
            if rng.random() < 0.3:
                edges.append((u, u))
                ws.append(int(rng.integers(1, 9)) if weights == "int" else float(rng.uniform(0.05, 1.0)))
    return gg.from_edges(n, edges, ws, fp=(weights != "int"))


def cliques(k: int, s: int, ring: bool = False):
    edges = []
    for b in range(k):
        base = b * s
        edges += [(base + i, base + j) for i, j in combinations(range(s), 2)]
    if ring:
        for b in range(k):
            edges.append((b * s + s - 1, ((b + 1) % k) * s))
    return gg.from_edges(k * s, edges)


def canonical(membership) -> np.ndarray:
    """Rank-renumber ids by order of the smallest occupied id (reading R6 of the oracle)."""
    m = np.asarray(membership)
    ids = np.unique(m)
    remap = {c: r for r, c in enumerate(ids)}
    return np.array([remap[c] for c in m], dtype=np.int32)


def same_partition(a, b) -> bool:
    """True if two memberships induce the same partition (labels may differ)."""
    a = np.asarray(a); b = np.asarray(b)
    if a.shape != b.shape:
        return False
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def check_csr(g) -> None:
    """Structural validity of a symmetric CSR from the generators."""
    offs, tg = g.offsets, g.targets
    assert offs[0] == 0 and offs[-1] == len(tg)
    assert np.all(np.diff(offs) >= 0)
    assert tg.min(initial=0) >= 0 and tg.max(initial=-1) < g.n
