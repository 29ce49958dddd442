"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each check is independent of the oracle's own code: closed forms, a brute-force enumeration, a
second formula (pair-sum form of Eq. 1, exact rationals), a library routine (networkx), or a
published test vector.  A dropped term, a wrong sign or a transposed index in the oracle fails
at least one of them.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import hand_traced
import oracle
from helpers import (brute_force_max_q, canonical, cliques, dense_adjacency, q_exact, q_pairsum, random_graph,
                     same_partition)


# ---------------------------------------------------------------- counter hash (published vector)
def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567: the first outputs of the reference C implementation.
    assert gg.splitmix64_nth(1234567, 0) == 6457827717110365317
    assert gg.splitmix64_nth(1234567, 1) == 3203168211198807973
    assert gg.splitmix64_nth(1234567, 2) == 9817491932198370423


def test_oracle_hash_matches_generator_hash():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b, c = (int(x) for x in rng.integers(0, 2**63, size=3, dtype=np.int64))
        assert oracle.hash3(a, b, c) == gg.hash3(a, b, c)


# ---------------------------------------------------------------- Eq. 1 (modularity)
@pytest.mark.parametrize("seed", range(6))
def test_modularity_vs_pairsum_int(seed):
    rng = np.random.default_rng(seed)
    g = random_graph(11, 0.35, rng)
    a = dense_adjacency(g)
    for _ in range(20):
        mem = rng.integers(0, 4, size=g.n).astype(np.int32)
        q = oracle.modularity(g.offsets, g.targets, g.weights, mem)
        exact = q_exact(a, mem)
        assert q == float(exact)  # one correctly rounded division of exact integers


@pytest.mark.parametrize("seed", range(4))
def test_modularity_vs_pairsum_fp(seed):
    rng = np.random.default_rng(100 + seed)
    g = random_graph(12, 0.4, rng, weights="fp")
    a = dense_adjacency(g)
    for _ in range(10):
        mem = rng.integers(0, 5, size=g.n).astype(np.int32)
        assert oracle.modularity(g.offsets, g.targets, g.weights, mem) == pytest.approx(q_pairsum(a, mem), abs=1e-12)


def test_modularity_vs_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(7)
    g = random_graph(30, 0.2, rng)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for i in range(g.n):
        for e in range(g.offsets[i], g.offsets[i + 1]):
            j = int(g.targets[e])
            if i < j:
                G.add_edge(i, j, weight=int(g.weights[e]))
    for _ in range(10):
        mem = rng.integers(0, 6, size=g.n).astype(np.int32)
        comms = [set(np.flatnonzero(mem == c).tolist()) for c in np.unique(mem)]
        ref = nx.algorithms.community.modularity(G, comms, weight="weight")
        assert oracle.modularity(g.offsets, g.targets, g.weights, mem) == pytest.approx(ref, abs=1e-12)


@pytest.mark.parametrize("k,s", [(2, 5), (3, 4), (7, 6), (10, 3)])
def test_modularity_disjoint_cliques(k, s):
    g = cliques(k, s)
    mem = np.repeat(np.arange(k), s).astype(np.int32)
    # Q = 1 - 1/k, i.e. the rational (k-1)/k, correctly rounded
    assert oracle.modularity(g.offsets, g.targets, g.weights, mem) == (k - 1) / k


@pytest.mark.parametrize("k,s", [(3, 4), (4, 5), (9, 3)])
def test_modularity_ring_of_cliques(k, s):
    g = cliques(k, s, ring=True)
    mem = np.repeat(np.arange(k), s).astype(np.int32)
    closed = Fraction(s * (s - 1), s * (s - 1) + 2) - Fraction(1, k)
    assert oracle.modularity(g.offsets, g.targets, g.weights, mem) == float(closed)


def test_modularity_singletons_closed_form():
    rng = np.random.default_rng(3)
    g = random_graph(15, 0.3, rng)
    k = np.array([int(g.weights[g.offsets[i]:g.offsets[i + 1]].sum()) for i in range(g.n)])
    two_m = int(k.sum())
    q = oracle.modularity(g.offsets, g.targets, g.weights, np.arange(g.n, dtype=np.int32))
    assert q == float(Fraction(-int((k * k).sum()), two_m * two_m))


# ---------------------------------------------------------------- Eq. 2 (delta modularity)
@pytest.mark.parametrize("seed,loops", [(0, False), (1, False), (2, True), (3, True)])
def test_move_score_equals_exact_delta_q(seed, loops):
    """2N/(2m)^2 equals Q(after) - Q(before) exactly for every single-vertex move."""
    rng = np.random.default_rng(seed)
    g = random_graph(9, 0.45, rng, self_loops=loops)
    a = dense_adjacency(g)
    two_m = int(a.sum())
    for _ in range(4):
        mem = rng.integers(0, 4, size=g.n).astype(np.int32)
        q0 = q_exact(a, mem)
        for i in range(g.n):
            for c in range(g.n):
                if c == mem[i]:
                    continue
                nscore = oracle.move_score(g.offsets, g.targets, g.weights, mem, i, c)
                m2 = mem.copy()
                m2[i] = c
                assert Fraction(2 * nscore, two_m * two_m) == q_exact(a, m2) - q0


# ---------------------------------------------------------------- convergence of the local-moving phase
@pytest.mark.parametrize("schedule", [0, 1])
def test_local_move_tolerance_limits(schedule):
    """Algorithm 2's per-iteration test: an infinite tolerance ends the phase after its first
    iteration; MAX_ITERATIONS caps the count; every iteration but a converged one moves something."""
    rng = np.random.default_rng(7)
    g = random_graph(40, 0.15, rng)
    _, it_inf, mv_inf = oracle.local_move(g.offsets, g.targets, g.weights,
                                           oracle.default_params(schedule=schedule), tau=float("inf"))
    assert it_inf == 1 and mv_inf > 0
    for cap in (1, 2, 3):
        _, it, _ = oracle.local_move(g.offsets, g.targets, g.weights,
                                     oracle.default_params(schedule=schedule, max_iterations=cap), tau=0.0)
        assert it <= cap
    _, it0, mv0 = oracle.local_move(g.offsets, g.targets, g.weights,
                                    oracle.default_params(schedule=schedule, max_iterations=1000), tau=0.0)
    assert it0 >= 2 and mv0 >= it0 - 1  # the last iteration may move nothing; every earlier one moved


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("schedule", [0, 1])
def test_local_move_zero_tolerance_reaches_single_move_optimum(seed, schedule):
    """With tolerance 0 and pruning off the phase stops only after an iteration with no move, so
    no single vertex can then raise Q by changing to a neighbouring community: every such move has
    exact Delta Q <= 0 (Eq. 1 evaluated before and after, in rationals).  The sequential schedule
    raises Q with every move and must stop.  The colour-synchronous one need not: vertices of a
    class that join one community together lose a cross term -2 K_u K_v / (2m)^2 that neither
    score sees, and seed 0 settles into a two-iteration cycle (Q 0.19216 / 0.16723), which is what
    the paper's positive tolerance and iteration cap bound."""
    rng = np.random.default_rng(100 + seed)
    g = random_graph(12, 0.35, rng, self_loops=seed % 2 == 1)
    a = dense_adjacency(g)
    cap = 1000

    def run(max_it):
        return oracle.local_move(g.offsets, g.targets, g.weights,
                                 oracle.default_params(schedule=schedule, pruning=0, max_iterations=max_it),
                                 tau=0.0)

    cp, it, _ = run(cap)
    if schedule == 0 and seed == 0:
        assert it == cap
        cp1, _, _ = run(cap + 1)
        cp2, _, _ = run(cap + 2)
        assert q_exact(a, cp1) < q_exact(a, cp) and same_partition(cp2, cp)
        return
    assert it < cap
    q0 = q_exact(a, cp)
    for i in range(g.n):
        for c in {int(cp[j]) for j in np.flatnonzero(a[i]) if j != i}:
            if c == cp[i]:
                continue
            m2 = cp.copy()
            m2[i] = c
            assert q_exact(a, m2) - q0 <= 0


# ---------------------------------------------------------------- colouring (deterministic schedule)
def _greedy_reference(g, seed, pass_index):
    order = sorted(range(g.n), key=lambda v: (gg.hash3(seed, pass_index, v), v), reverse=True)
    col = [-1] * g.n
    for v in order:
        used = {col[int(u)] for u in g.targets[g.offsets[v]:g.offsets[v + 1]] if u != v and col[int(u)] >= 0}
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return np.array(col, dtype=np.int32)


@pytest.mark.parametrize("seed", range(3))
def test_colouring_is_proper_and_greedy(seed):
    rng = np.random.default_rng(seed)
    g = random_graph(40, 0.15, rng, self_loops=True)
    col, nc = oracle.colour(g.offsets, g.targets, seed=11 + seed, pass_index=seed)
    for i in range(g.n):
        for u in g.targets[g.offsets[i]:g.offsets[i + 1]]:
            if u != i:
                assert col[i] != col[u]
    assert nc == col.max() + 1
    assert np.array_equal(col, _greedy_reference(g, 11 + seed, seed))


def test_colouring_complete_graph():
    g = cliques(1, 9)
    col, nc = oracle.colour(g.offsets, g.targets, 5, 0)
    assert nc == 9 and sorted(col.tolist()) == list(range(9))


# ---------------------------------------------------------------- Algorithm 3 (aggregation)
@pytest.mark.parametrize("seed,fp", [(0, False), (1, False), (2, True)])
def test_aggregate_vs_dense_scatter(seed, fp):
    rng = np.random.default_rng(seed)
    g = random_graph(25, 0.2, rng, weights="fp" if fp else "int", self_loops=True)
    nc = 6
    mem = rng.integers(0, nc, size=g.n).astype(np.int32)
    mem[:nc] = np.arange(nc)  # every community occupied
    oo, ot, ow = oracle.aggregate(g.offsets, g.targets, g.weights, mem, nc)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    ref = np.zeros((nc, nc), dtype=np.float64)
    np.add.at(ref, (mem[src], mem[g.targets]), g.weights.astype(np.float64))
    got = np.zeros((nc, nc), dtype=np.float64)
    for c in range(nc):
        row = ot[oo[c]:oo[c + 1]]
        assert np.all(np.diff(row) > 0)  # sorted, unique
        got[c, row] = ow[oo[c]:oo[c + 1]]
    assert np.allclose(got, ref, rtol=0, atol=1e-9 if fp else 0)
    assert np.count_nonzero(ref) == len(ot)


@pytest.mark.parametrize("seed", range(3))
def test_aggregate_preserves_modularity_and_2m(seed):
    rng = np.random.default_rng(seed)
    g = random_graph(30, 0.2, rng, self_loops=(seed == 2))
    mem = canonical(rng.integers(0, 7, size=g.n))
    nc = int(mem.max()) + 1
    oo, ot, ow = oracle.aggregate(g.offsets, g.targets, g.weights, mem, nc)
    assert int(ow.sum()) == int(g.weights.sum())
    q_orig = oracle.modularity(g.offsets, g.targets, g.weights, mem)
    q_super = oracle.modularity(oo, ot, ow.astype(np.int32), np.arange(nc, dtype=np.int32))
    assert q_super == q_orig
    assert Fraction(q_orig) == Fraction(float(q_exact(dense_adjacency(g), mem)))


# ---------------------------------------------------------------- Algorithms 1-2 (full method)
def test_two_vertices_hand_traced():
    g = gg.from_edges(2, [(0, 1)])
    mem, q, passes, stats = oracle.louvain(g.offsets, g.targets, g.weights)
    # pass 0: one vertex joins the other (N = 2m*1 - 1*1 = 1 > 0), second iteration converges
    assert stats[0]["iterations"] == 2 and stats[0]["moves"] == 1
    # pass 1: the single super-vertex has only its self-loop, so l_i = 1 and the passes stop
    assert passes == 2 and stats[1]["iterations"] == 1
    assert mem.tolist() == [0, 0] and q == 0.0


def test_isolated_and_empty():
    g = gg.from_edges(5, [])
    mem, q, passes, _ = oracle.louvain(g.offsets, g.targets, g.weights)
    assert mem.tolist() == [0, 1, 2, 3, 4] and q == 0.0 and passes == 1
    g0 = gg.from_edges(0, [])
    mem, q, passes, _ = oracle.louvain(g0.offsets, g0.targets, g0.weights)
    assert len(mem) == 0 and q == 0.0


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("schedule", [0, 1])
def test_louvain_never_beats_brute_force(seed, schedule):
    rng = np.random.default_rng(seed)
    g = random_graph(8, 0.4, rng)
    if g.n_arcs == 0:
        pytest.skip("empty draw")
    mem, q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(schedule=schedule))
    a = dense_adjacency(g)
    assert q == pytest.approx(q_pairsum(a, mem), abs=1e-12)
    assert q <= brute_force_max_q(a) + 1e-12


def test_two_cliques_with_bridge_reach_optimum():
    g = cliques(2, 5, ring=False)
    g = gg.from_edges(10, [(i, j) for i in range(5) for j in range(i + 1, 5)] +
                      [(5 + i, 5 + j) for i in range(5) for j in range(i + 1, 5)] + [(4, 5)])
    mem, q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights)
    assert same_partition(mem, [0] * 5 + [1] * 5)
    assert q == pytest.approx(brute_force_max_q(dense_adjacency(g)), abs=1e-12)


@pytest.mark.parametrize("schedule", [0, 1])
def test_ring_of_cliques_recovered(schedule):
    k, s = 4, 5
    g = cliques(k, s, ring=True)
    mem, q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights,
                                  oracle.default_params(schedule=schedule, max_passes=100))
    assert same_partition(mem, np.repeat(np.arange(k), s))
    assert q == float(Fraction(s * (s - 1), s * (s - 1) + 2) - Fraction(1, k))


@pytest.mark.parametrize("schedule", [0, 1])
def test_karate_club_below_published_optimum(schedule):
    """Zachary's karate club (networkx's copy, unweighted): the maximum modularity over all
    partitions is 0.4197896, proved optimal by integer linear programming (Brandes et al., "On
    Modularity Clustering", IEEE TKDE 2008).  Louvain may not exceed it and lands close to it; its
    Q is a rational with denominator (2m)^2 in integer mode and equals networkx's Eq. 1."""
    nx = pytest.importorskip("networkx")
    kc = nx.karate_club_graph()
    edges = sorted((min(u, v), max(u, v)) for u, v in kc.edges())
    assert kc.number_of_nodes() == 34 and len(edges) == 78
    g = gg.from_edges(34, edges)
    mem, q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(schedule=schedule))
    assert 0.41 <= q <= 0.4197896 + 1e-7
    two_m = 2 * len(edges)
    assert abs(q * two_m * two_m - round(q * two_m * two_m)) < 1e-6
    h = nx.Graph()
    h.add_nodes_from(range(34))
    h.add_edges_from(edges)
    parts = [set(np.flatnonzero(mem == c).tolist()) for c in np.unique(mem)]
    assert q == pytest.approx(nx.community.modularity(h, parts), abs=1e-12)


@pytest.mark.parametrize("tau_agg,passes", [(0.8, 1), (0.96, 1), (101 / 105, 2), (0.97, 2)])
def test_aggregation_tolerance_stops_the_pass_loop(tau_agg, passes):
    """Algorithm 1 stops after a pass whose community count is more than tau_agg of its vertices.
    A 5-clique plus 100 isolated vertices: pass 0 merges the clique, |Gamma| / |V'| = 101 / 105 =
    0.9619; a larger ratio than tau_agg (strictly) ends the run, otherwise the aggregated graph gets
    a second pass, which moves nothing and ends after one iteration.  Q = 1 - 1^2 = 0 (one
    community holds every edge)."""
    g = gg.from_edges(105, [(i, j) for i in range(5) for j in range(i + 1, 5)])
    mem, q, n_passes, stats = oracle.louvain(g.offsets, g.targets, g.weights,
                                             oracle.default_params(aggregation_tolerance=tau_agg))
    assert n_passes == passes
    assert (stats[0]["n_vertices"], stats[0]["n_communities"]) == (105, 101)
    if passes == 2:
        assert (stats[1]["n_vertices"], stats[1]["iterations"], stats[1]["moves"]) == (101, 1, 0)
    assert same_partition(mem, [0] * 5 + list(range(1, 101)))
    assert q == 0.0


def _replay_passes(g, p, next_tau):
    """Algorithm 1's loop written out over the single steps (each pinned on its own): local moving
    from singletons with the pass's tolerance, renumbering by rank, the two pass tests, aggregation,
    then the next tolerance.  Returns (iterations, moves) per pass."""
    offs, tg, w = g.offsets, g.targets, g.weights
    tau, seq = p.tolerance, []
    for k in range(p.max_passes):
        cp, it, mv = oracle.local_move(offs, tg, w, p, k, tau=tau)
        seq.append((it, mv))
        ids = np.unique(cp)
        if it <= 1 or len(ids) / len(cp) > p.aggregation_tolerance:
            break
        offs, tg, w = oracle.aggregate(offs, tg, w, np.searchsorted(ids, cp).astype(np.int32), len(ids))
        tau = next_tau(tau, p.tolerance_drop)
    return seq


@pytest.mark.parametrize("name", ["sbm2k", "rmat12", "rmat14"])
def test_threshold_scaling_between_passes(name):
    """Threshold scaling (Section 4.1.3): pass p runs with tolerance tau_0 / drop^p.  The run's
    per-pass iterations and moves equal the replay that divides, and differ from replays that
    multiply or keep tau (so the check sees the drop's direction)."""
    g = {"sbm2k": lambda: gg.sbm(2000, 20, 0.1, 0.002, 7),
         "rmat12": lambda: gg.rmat(12, weights=gg.W_INT8, seed=3),
         "rmat14": lambda: gg.rmat(14, weights=gg.W_INT8, seed=22)}[name]()
    p = oracle.default_params()
    _, _, passes, stats = oracle.louvain(g.offsets, g.targets, g.weights, p)
    run = [(s["iterations"], s["moves"]) for s in stats]
    assert passes >= 2 and run == _replay_passes(g, p, lambda t, d: t / d)
    assert run != _replay_passes(g, p, lambda t, d: t * d)
    assert run != _replay_passes(g, p, lambda t, d: t)


def test_planted_partition_sbm_10k():
    g = gg.sbm(10000, 100, 0.1, 0.0005, 1)
    planted = gg.planted_blocks(10000, 100)
    q_planted = oracle.modularity(g.offsets, g.targets, g.weights, planted)
    mem, q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(max_passes=100))
    assert q > q_planted - 0.005
    # most vertices sit with the majority of their planted block
    agree = 0
    for b in range(100):
        ids = mem[planted == b]
        agree += np.bincount(ids).max()
    assert agree / g.n > 0.97


def test_fp_and_int_instantiations_agree_on_integral_weights():
    rng = np.random.default_rng(5)
    g = random_graph(60, 0.08, rng)
    gf = gg.Graph(g.n, g.offsets, g.targets, g.weights.astype(np.float32))
    for schedule in (0, 1):
        p = oracle.default_params(schedule=schedule)
        mi, qi, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, p)
        mf, qf, _, _ = oracle.louvain(gf.offsets, gf.targets, gf.weights, p)
        assert np.array_equal(mi, mf)
        assert qi == pytest.approx(qf, abs=1e-12)


def test_overflow_rejected():
    g = gg.from_edges(2, [(0, 1)], [2**30])
    with pytest.raises(OverflowError):
        oracle.louvain(g.offsets, g.targets, g.weights)


# ---------------------------------------------------------------- hand-traced readings of Algorithm 2
@pytest.mark.parametrize("case", hand_traced.CASES, ids=lambda c: c.name)
def test_hand_traced_local_move(case):
    """R2 (ties to the smallest id, strict N > 0) and R3 (marks of a class make later classes of
    the same iteration eligible) on graphs traced by hand; the trace is in tests/hand_traced.py."""
    if case.colours is not None:
        col, _ = oracle.colour(case.offsets, case.targets, case.seed, 0)
        assert tuple(col.tolist()) == case.colours
    cp, it, mv = oracle.local_move(case.offsets, case.targets, case.weights,
                                   oracle.default_params(seed=case.seed), 0, tau=case.tau)
    assert tuple(cp.tolist()) == case.cp
    assert (it, mv) == (case.iterations, case.moves)


def test_hand_traced_zero_gain_is_zero_by_eq1():
    """The zero-gain moves of the strict-rule cases change Eq. 1 by exactly 0 (exact rationals)."""
    c = hand_traced.ZERO_LOOPS
    a = dense_adjacency(gg.Graph(n=2, offsets=c.offsets, targets=c.targets, weights=c.weights))
    assert q_exact(a, [0, 1]) == q_exact(a, [1, 1]) == 0
    t = hand_traced.ZERO_TRIANGLE
    a = dense_adjacency(gg.Graph(n=3, offsets=t.offsets, targets=t.targets, weights=t.weights))
    # vertex 0 leaving {0, 1} for {2}, the state after class {1} of the trace
    assert q_exact(a, [0, 0, 2]) == q_exact(a, [2, 0, 2])


# Each entry plants one plausible mistake in a copy of the oracle's source: (old text, new text)
# replacements that must each match exactly once.
_MUTANTS = {
    "tie_to_largest_id": [("(nscore == best && c < bc)", "(nscore == best && c > bc)")],
    "tie_to_first_seen": [(" || (nscore == best && c < bc)", "")],
    "tie_to_last_seen": [("nscore > best || (nscore == best && c < bc)", "nscore >= best")],
    "move_on_zero_gain": [("return found && best > W(0);", "return found && best >= W(0);")],
    "marks_wait_for_next_iteration": [
        ("int64_t moves = 0;", "int64_t moves = 0;\n  std::vector<int32_t> later;"),
        ("if (g.tg[e] != i) flag[g.tg[e]] = 1;", "if (g.tg[e] != i) later.push_back(g.tg[e]);"),
        ("li = it + 1;", "for (int32_t v : later) flag[v] = 1;\n      later.clear();\n      li = it + 1;"),
    ],
}


# Plausible mistakes elsewhere in the method: each must fail at least one pin of this file.
_METHOD_MUTANTS = {
    # Eq. 2 without its K_i (Sigma_c - Sigma_d + K_i) correction: the K_i term dropped
    "score_drops_ki_term": [("K[i] * (Sig[c] - Sig[d] + K[i]);", "K[i] * (Sig[c] - Sig[d]);")],
    # scanCommunities with self = true in the local move: i's self-loop counted in K_i->d
    "local_move_counts_own_loop": [("      if (j == i) continue;  // scanCommunities with self = false\n", "")],
    # a self-loop counted twice in K_i (R1)
    "loop_counted_twice_in_k": [("K[i] += g.w[e];", "K[i] += g.tg[e] == i ? 2 * g.w[e] : g.w[e];")],
    # Eq. 1 with the null-model term added instead of subtracted
    "modularity_sign": [("int64_t num = two_m * sigma_in - sq,", "int64_t num = two_m * sigma_in + sq,")],
    # the super-graph loses its self-loops (intra-community arcs dropped)
    "aggregate_drops_self_loops": [("H.add(Cp[g.tg[e]], g.w[e]);",
                                    "if (Cp[g.tg[e]] != (int32_t)c) H.add(Cp[g.tg[e]], g.w[e]);")],
    # the aggregation tolerance test reversed (R5)
    "aggregation_tolerance_reversed": [("(double)nc / (double)gp.n > p.aggregation_tolerance",
                                        "(double)nc / (double)gp.n < p.aggregation_tolerance")],
    # no threshold scaling between passes
    "no_threshold_scaling": [("tau /= p.tolerance_drop;", "tau *= 1.0;")],
    # the greedy colouring taken in increasing priority
    "colouring_in_increasing_priority": [("return a.first != b.first ? a.first > b.first : a.second > b.second;",
                                          "return a.first != b.first ? a.first < b.first : a.second < b.second;")],
    # the tolerance test strict (R4)
    "tolerance_test_strict": [("return lhs <= tau * (t * t);", "return lhs < tau * (t * t);")],
    # l_i counted from 0 (R4)
    "iterations_zero_based": [("      li = it + 1;", "      li = it;")],
    # the pass loop stopping at two iterations instead of one (Alg. 1)
    "pass_loop_stops_at_two_iterations": [("if (li <= 1) break;", "if (li <= 2) break;")],
    # renumbering by decreasing id instead of the rank among occupied ids (R6)
    "renumber_reversed": [("for (int32_t& c : C) c = (int32_t)rank[c];",
                           "for (int32_t& c : C) c = (int32_t)(r - 1 - rank[c]);")],
    # the last pass's membership not looked up into the dendrogram (R6)
    "last_lookup_skipped": [("  if (pending)\n    for (int64_t v = 0; v < n; v++) C[v] = Cp[C[v]];", "")],
    # a processed vertex keeps its flag (pruning never clears)
    "flag_never_cleared": [("            flag[v] = 0;\n            int32_t c; W ns;\n            if (decide(v, &c, &ns)) dec",
                            "            int32_t c; W ns;\n            if (decide(v, &c, &ns)) dec")],
    # a colour class applying each move at once instead of after the class (R3)
    "class_moves_applied_at_once": [("            if (decide(v, &c, &ns)) dec.push_back({v, c, ns});",
                                     "            if (decide(v, &c, &ns)) apply(v, c, ns, sum_n, p.pruning);")],
}


def _run_pins_against(tmp_path, mutants: dict, select: str) -> dict:
    """Compile each mutated copy of the oracle (and an unchanged one), run the selected pins of
    this file against it in a child process; returns {name: pytest exit code}."""
    import os
    import subprocess
    import sys
    src = open(os.path.join(os.path.dirname(oracle.__file__), "louvain_oracle.cpp")).read()
    builds = {}
    for name, edits in list(mutants.items()) + [("unchanged", [])]:
        text = src
        for old, new in edits:
            assert text.count(old) == 1, (name, old)
            text = text.replace(old, new)
        cpp = tmp_path / f"{name}.cpp"
        cpp.write_text(text)
        so = tmp_path / f"{name}.so"
        builds[name] = (so, subprocess.Popen(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-o", str(so), str(cpp)]))
    here = os.path.dirname(os.path.abspath(__file__))
    codes = {}
    for name, (so, proc) in builds.items():
        assert proc.wait() == 0, name
        env = dict(os.environ, LOUVAIN_ORACLE_SO=str(so))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            os.path.join(here, "test_oracle_pins.py"), "-k", select],
                           env=env, capture_output=True, text=True, cwd=os.path.dirname(here))
        codes[name] = (r.returncode, r.stdout[-1500:])
    return codes


def test_pins_catch_planted_mistakes_in_the_method(tmp_path):
    """Every planted mistake in Eq. 1, Eq. 2, R1, R3-R6, the aggregation, the pass loop or the
    colouring fails at least one pin of this file; the unchanged source, built the same way, passes
    them all."""
    codes = _run_pins_against(tmp_path, _METHOD_MUTANTS, "not catch_planted")
    assert codes["unchanged"][0] == 0, codes["unchanged"][1]
    for name in _METHOD_MUTANTS:
        assert codes[name][0] == 1, (name, codes[name][1])


def test_hand_traced_pins_catch_planted_mistakes(tmp_path):
    """Every planted mistake in R2 / R3 fails at least one hand-traced pin, run in a child process
    against the mutated copy of the oracle (LOUVAIN_ORACLE_SO)."""
    import os
    import subprocess
    import sys
    src = open(os.path.join(os.path.dirname(oracle.__file__), "louvain_oracle.cpp")).read()
    builds = {}
    for name, edits in _MUTANTS.items():
        text = src
        for old, new in edits:
            assert text.count(old) == 1, (name, old)
            text = text.replace(old, new)
        cpp = tmp_path / f"{name}.cpp"
        cpp.write_text(text)
        so = tmp_path / f"{name}.so"
        builds[name] = (so, subprocess.Popen(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-o", str(so), str(cpp)]))
    here = os.path.dirname(os.path.abspath(__file__))
    for name, (so, proc) in builds.items():
        assert proc.wait() == 0, name
        env = dict(os.environ, LOUVAIN_ORACLE_SO=str(so))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            os.path.join(here, "test_oracle_pins.py"), "-k", "test_hand_traced_local_move"],
                           env=env, capture_output=True, text=True, cwd=os.path.dirname(here))
        assert r.returncode == 1, (name, r.stdout[-2000:])
        assert "failed" in r.stdout, name


# ---------------------------------------------------------------- dynamic graphs: batch update and warm start
def _random_update(g, rng, n_new, n_del, n_ins):
    """Deletions: existing edges plus a pair that is not an edge; insertions: new pairs, an existing
    edge again (its arcs duplicate) and a self-loop; ids may reach the new rows n..n_new-1."""
    edges = [(u, int(v)) for u in range(g.n) for v in g.targets[g.offsets[u]:g.offsets[u + 1]] if u <= v]
    pick = rng.choice(len(edges), size=min(n_del, len(edges)), replace=False)
    dels = [edges[k] for k in pick] + [(0, n_new - 1)]
    ins = [(int(rng.integers(0, n_new)), int(rng.integers(0, n_new))) for _ in range(n_ins)]
    ins += [edges[int(pick[0])], (3, 3)]
    iw = rng.integers(1, 9, size=len(ins)).astype(np.int32)
    return dels, ins, iw


@pytest.mark.parametrize("seed", range(4))
def test_update_graph_vs_dense_matrix(seed):
    """The updated CSR's dense matrix equals the old one with every deleted pair zeroed (both
    directions) and each insertion added at (u, v) and (v, u) (once on the diagonal)."""
    rng = np.random.default_rng(seed)
    g = random_graph(14, 0.3, rng, self_loops=seed % 2 == 1)
    n_new = g.n + 3
    dels, ins, iw = _random_update(g, rng, n_new, 6, 8)
    oo, ot, ow = oracle.update_graph(g.offsets, g.targets, g.weights, n_new, dels, ins, iw)
    a = np.zeros((n_new, n_new), dtype=np.int64)
    a[:g.n, :g.n] = dense_adjacency(g)
    for u, v in dels:
        a[u, v] = a[v, u] = 0
    for (u, v), w in zip(ins, iw):
        a[u, v] += w
        if u != v:
            a[v, u] += w
    h = gg.Graph(n=n_new, offsets=oo, targets=ot, weights=ow)
    assert np.array_equal(dense_adjacency(h), a)
    # rows keep their surviving arcs in order, then the inserted ones in list order
    r = ins[0][0]
    assert ot[oo[r + 1] - 1] in [v for (u, v) in ins if u == r] + [u for (u, v) in ins if v == r]


def test_warm_start_from_singletons_is_the_cold_run():
    g = gg.sbm(600, 6, 0.2, 0.01, 3)
    for sched in (0, 1):
        p = oracle.default_params(schedule=sched, seed=4)
        cold = oracle.louvain(g.offsets, g.targets, g.weights, p)
        warm = oracle.louvain_from(g.offsets, g.targets, g.weights, np.arange(g.n), p)
        assert np.array_equal(cold[0], warm[0]) and cold[1:3] == warm[1:3]
        assert [s["iterations"] for s in cold[3]] == [s["iterations"] for s in warm[3]]


@pytest.mark.parametrize("schedule", [0, 1])
def test_warm_start_at_a_clique_partition_stays_put(schedule):
    """Ring of k K_s cliques started from its cliques (ids shuffled): a member of clique c gains
    K_i->c' = 1 by joining the neighbouring clique and loses K_i->c = s - 1, so no N is positive;
    the first iteration moves nothing, l_i = 1 ends the run after one pass, and the output is the
    cliques with the closed-form modularity s(s-1)/(s(s-1)+2) - 1/k."""
    k, s = 5, 6
    g = cliques(k, s, ring=True)
    ids = np.random.default_rng(1).permutation(g.n)[:k]
    init = np.repeat(ids, s).astype(np.int32)
    mem, q, passes, stats = oracle.louvain_from(g.offsets, g.targets, g.weights, init,
                                                oracle.default_params(schedule=schedule))
    assert passes == 1 and stats[0]["iterations"] == 1 and stats[0]["moves"] == 0
    assert mem.tolist() == canonical(init).tolist()
    assert q == float(Fraction(s * (s - 1), s * (s - 1) + 2) - Fraction(1, k))


def test_warm_start_cannot_split_one_community():
    """Every vertex in one community: each vertex's neighbours are all in its own community, so it
    has no candidate; nothing moves and the result is that one community, Q = 1 - 1 = 0."""
    g = cliques(3, 5, ring=True)
    mem, q, passes, stats = oracle.louvain_from(g.offsets, g.targets, g.weights, np.full(g.n, 7, dtype=np.int32))
    assert mem.tolist() == [0] * g.n and q == 0.0 and passes == 1 and stats[0]["moves"] == 0


@pytest.mark.parametrize("seed", range(6))
def test_sequential_warm_start_never_loses_modularity(seed):
    """Under the sequential schedule every move has N > 0 (Delta Q > 0) and aggregation keeps Q, so
    a warm start ends at or above the modularity of the membership it started from."""
    rng = np.random.default_rng(50 + seed)
    g = random_graph(30, 0.15, rng)
    init = rng.integers(0, 6, size=g.n).astype(np.int32)
    _, q, _, _ = oracle.louvain_from(g.offsets, g.targets, g.weights, init, oracle.default_params(schedule=1))
    assert q >= float(q_exact(dense_adjacency(g), init)) - 1e-15


def test_warm_start_after_a_small_update_matches_the_cold_run():
    """A planted partition, 1% of its edges deleted and as many random edges inserted: the warm start
    from the old result reaches the cold run's modularity on the updated graph within 0.005."""
    g = gg.sbm(3000, 30, 0.1, 0.001, 8)
    rng = np.random.default_rng(2)
    mem, _, _, _ = oracle.louvain(g.offsets, g.targets, g.weights)
    m = g.n_arcs // 2
    dels, ins, iw = _random_update(g, rng, g.n, m // 100, m // 100)
    oo, ot, ow = oracle.update_graph(g.offsets, g.targets, g.weights, g.n, dels, ins, iw)
    cold_m, cold_q, _, _ = oracle.louvain(oo, ot, ow)
    warm_m, warm_q, _, _ = oracle.louvain_from(oo, ot, ow, mem)
    assert abs(warm_q - cold_q) <= 0.005
    assert warm_q == pytest.approx(oracle.modularity(oo, ot, ow, warm_m), abs=0)
