"""Hand-traced local-moving cases for three readings of Algorithm 2 that decide results bit for bit.

Each case is a graph of 3-5 vertices with its seed, the colour classes that seed gives (greedy in
decreasing priority hash3(seed, pass, v)), and the C', iteration count l_i and move count of one
local-moving phase from singletons, all written out by hand from the trace in the case's comment.
Eq. 2 numerators are N(i: d -> c) = 2m (K_i->c - K_i->d) - K_i (Sigma_c - Sigma_d + K_i).

  tie_star      R2: of equal best numerators the smallest community id wins
  zero_triangle R2: a best numerator of exactly 0 does not move the vertex (N > 0 is strict)
  zero_loops    R2 again, with self-loops (which K_i counts and K_i->c does not)
  marks_path    R3: marks set by a class make later classes of the SAME iteration eligible
                (deferring them to the next iteration changes C', l_i and the move count)

Nothing here calls the oracle or the GPU library; tests/test_oracle_pins.py checks the oracle
against these values and tests/test_gpu_parity.py checks the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Case:
    name: str
    offsets: np.ndarray
    targets: np.ndarray
    weights: np.ndarray
    seed: int
    tau: float
    colours: tuple      # expected colour of each vertex at pass 0
    cp: tuple           # expected C' after the phase (ids not renumbered)
    iterations: int
    moves: int


def _csr(rows):
    """rows: list per vertex of (target, weight), kept in the given order."""
    offs = np.zeros(len(rows) + 1, dtype=np.int64)
    for i, r in enumerate(rows):
        offs[i + 1] = offs[i] + len(r)
    tg = np.array([t for r in rows for t, _ in r], dtype=np.int32)
    w = np.array([x for r in rows for _, x in r], dtype=np.int32)
    return offs, tg, w


# Star K_{1,3}, unit weights, centre 0; the centre's row lists its leaves in the order 2, 1, 3 so
# that "first seen", "last seen" and "largest id" each pick a different leaf than "smallest id".
# 2m = 6, K_0 = 3, K_leaf = 1.  Seed 2: the centre has the top priority -> classes {0}, {1, 2, 3}.
# Iteration 1, class 0: centre (d = 0) scores each leaf c: N = 6*1 - 3*(1 - 3 + 3) = 3, a three-way
#   tie -> community 1.  Apply: Sigma_1 = 4, Sigma_0 = 0, sum N = 3, marks 1, 2, 3.
# Class 1 (class-start Sigma_1 = 4): leaf 1 has only its own community as a neighbour -> stays;
#   leaves 2 and 3: N(1) = 6*1 - 1*(4 - 1 + 1) = 2 > 0 -> both join 1.  sum N = 7; marks 0.
# Iteration 2: only the centre is flagged; all its neighbours are in its community -> no candidate.
#   sum N = 0 -> converged at l_i = 2 with 3 moves.
_so, _st, _sw = _csr([[(2, 1), (1, 1), (3, 1)], [(0, 1)], [(0, 1)], [(0, 1)]])
TIE_STAR = Case("tie_star", _so, _st, _sw, seed=2, tau=0.01, colours=(0, 1, 1, 1), cp=(1, 1, 1, 1),
                iterations=2, moves=3)

# Unit triangle 0-1-2.  2m = 6, K = (2, 2, 2).  Seed 9: classes {1}, {0}, {2}.
# Iteration 1, class {1}: N(0) = N(2) = 6*1 - 2*(2 - 2 + 2) = 2, tie -> 1 joins 0.
#   Sigma_0 = 4, Sigma_1 = 0, sum N = 2, marks 0 and 2.
# Class {0} (d = 0, K_0->d = 1 through vertex 1): N(2) = 6*(1 - 1) - 2*(2 - 4 + 2) = 0 exactly
#   (Eq. 1 gives Delta Q = 0 too) -> under the strict rule vertex 0 stays.
# Class {2}: K_2->0 = 2 (vertices 0 and 1): N(0) = 6*2 - 2*(4 - 2 + 2) = 4 > 0 -> joins 0.
#   Sigma_0 = 6, sum N = 6, marks 0 and 1.
# Iteration 2: 1 and 0 are flagged but every neighbour is in their community -> no candidate;
#   sum N = 0 -> l_i = 2, 2 moves, C' = (0, 0, 0).
_to, _tt, _tw = _csr([[(1, 1), (2, 1)], [(0, 1), (2, 1)], [(0, 1), (1, 1)]])
ZERO_TRIANGLE = Case("zero_triangle", _to, _tt, _tw, seed=9, tau=0.01, colours=(1, 0, 2), cp=(0, 0, 0),
                     iterations=2, moves=2)

# Two vertices, each with a self-loop of weight 1, joined by an edge of weight 1.
# K_0 = K_1 = 2 (self-loop counted once), 2m = 4; scanCommunities skips the self-loop, so
# K_0->1 = 1, K_0->0 = 0: N(0 -> 1) = 4*1 - 2*(2 - 2 + 2) = 0, and the same for vertex 1.
# Neither moves: l_i = 1, no moves.  (Q is 0 both as singletons and merged.)
_lo, _lt, _lw = _csr([[(0, 1), (1, 1)], [(0, 1), (1, 1)]])
ZERO_LOOPS = Case("zero_loops", _lo, _lt, _lw, seed=0, tau=0.01, colours=None, cp=(0, 1), iterations=1, moves=0)

# Path 0-1-2-3-4 with weights w01 = 3, w12 = 4, w23 = 2, w34 = 1.  2m = 20, K = (3, 7, 6, 3, 1).
# Seed 14: classes {1, 3}, {0, 2, 4}.
# Iteration 1, class {1, 3} against Sigma = K:
#   vertex 1: N(0) = 20*3 - 7*(3 - 7 + 7) = 39, N(2) = 20*4 - 7*(6 - 7 + 7) = 38 -> joins 0;
#   vertex 3: N(2) = 20*2 - 3*(6 - 3 + 3) = 22, N(4) = 20*1 - 3*(1 - 3 + 3) = 17 -> joins 2.
#   Apply: Sigma_0 = 10, Sigma_1 = 0, Sigma_2 = 9, Sigma_3 = 0; sum N = 61; marks 0, 2, 4.
# Class {0, 2, 4} (all flagged; the marks just set keep them eligible in this iteration):
#   vertex 0: its only neighbour is in its community -> stays;
#   vertex 2 (d = 2, K_2->2 = 2 via vertex 3): N(0) = 20*(4 - 2) - 6*(10 - 9 + 6) = -2 -> stays;
#   vertex 4: N(2) = 20*1 - 1*(9 - 1 + 1) = 11 -> joins 2.  Sigma_2 = 10; sum N = 72; marks 3.
#   Every vertex of this class cleared its flag when it was processed.
# Iteration 2: only vertex 3 is flagged; its neighbours are both in community 2 -> stays.
#   sum N = 0 -> l_i = 2, 3 moves, C' = (0, 0, 2, 2, 2).
# Had the marks of class {1, 3} waited for iteration 2, vertex 2 would be decided again there
# against Sigma_2 = 10: N(0) = 20*(4 - 2) - 6*(10 - 10 + 6) = 4 > 0, and it would join 0.
_po, _pt, _pw = _csr([[(1, 3)], [(0, 3), (2, 4)], [(1, 4), (3, 2)], [(2, 2), (4, 1)], [(3, 1)]])
MARKS_PATH = Case("marks_path", _po, _pt, _pw, seed=14, tau=0.01, colours=(1, 0, 1, 0, 1), cp=(0, 0, 2, 2, 2),
                  iterations=2, moves=3)

CASES = [TIE_STAR, ZERO_TRIANGLE, ZERO_LOOPS, MARKS_PATH]
