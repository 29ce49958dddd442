"""Batched runs (louvain_run_batch): many graphs as one union, each graph's result identical to
the CPU oracle's on that graph alone (deterministic mode, integer weights: membership arrays equal,
modularity equal, passes and total iterations equal) and to louvain_run on the graph alone.
Fast mode: valid partitions within 0.005 of the oracle's modularity; fp32 weights within 1e-4.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import cliques, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def L(cuda_ok):
    import paper_2312_04876_gb300 as lv
    h = lv.Louvain(0)
    yield h
    h.close()


def mixed_graphs():
    """Shapes that exercise every kernel path: planted blocks, R-MAT hubs, self-loops, rings of
    cliques, a star (one hub), an empty graph, isolated vertices only, a single vertex."""
    return [
        gg.sbm(2000, 20, 0.1, 0.002, 7),
        gg.rmat(12, weights=gg.W_INT8, seed=3),
        gg.from_edges(0, []),
        random_graph(300, 0.03, np.random.default_rng(1), self_loops=True),
        cliques(8, 6, ring=True),
        gg.from_edges(5, []),
        gg.from_edges(3000, [(0, i) for i in range(1, 3000)]),
        gg.from_edges(1, []),
        gg.sbm(500, 4, 0.2, 0.01, 9),
        gg.rmat(10, weights=gg.W_INT8, seed=5),
    ]


def upload(graphs):
    vo, offs, tg, w = gg.concat(graphs)
    return vo, torch.from_numpy(offs).to(DEV), torch.from_numpy(tg).to(DEV), torch.from_numpy(w).to(DEV)


def split(mem, vo):
    m = mem.cpu().numpy()
    return [m[vo[k]:vo[k + 1]] for k in range(len(vo) - 1)]


@pytest.mark.parametrize("compact", [1, 0])
def test_batch_deterministic_matches_oracle(L, compact):
    graphs = mixed_graphs()
    vo, o, t, w = upload(graphs)
    mem, per, res = L.run_batch(vo, o, t, w, mode="deterministic", compact=compact)
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        ref_mem, ref_q, ref_passes, ref_stats = oracle.louvain(g.offsets, g.targets, g.weights,
                                                               oracle.default_params())
        assert np.array_equal(m, ref_mem), f"graph {k}"
        assert per[k]["modularity"] == ref_q, f"graph {k}"
        assert per[k]["passes"] == ref_passes, f"graph {k}"
        assert per[k]["total_iterations"] == sum(s["iterations"] for s in ref_stats), f"graph {k}"
        assert per[k]["n_communities"] == (int(ref_mem.max()) + 1 if g.n else 0)


def test_batch_equals_single_runs(L):
    """The same graph alone (louvain_run) and inside the batch: identical results."""
    graphs = mixed_graphs()
    vo, o, t, w = upload(graphs)
    mem, per, _ = L.run_batch(vo, o, t, w, mode="deterministic", seed=11)
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        if g.n == 0:
            continue
        go, gt, gw = (torch.from_numpy(a).to(DEV) for a in (g.offsets, g.targets, g.weights))
        m1, r1 = L.run(go, gt, gw, mode="deterministic", seed=11)
        assert np.array_equal(m1.cpu().numpy(), m), f"graph {k}"
        assert r1.modularity == per[k]["modularity"]
        assert r1.passes == per[k]["passes"]


def test_batch_sbm_family_matches_oracle(L):
    """Members of the batched planted-partition family (sizes scaled down for the oracle)."""
    graphs = [gg.batch_sbm(4, k, n_lo=500.0, n_hi=6000.0) for k in range(24)]
    vo, o, t, w = upload(graphs)
    mem, per, res = L.run_batch(vo, o, t, w, mode="deterministic")
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        ref_mem, ref_q, ref_passes, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
        assert np.array_equal(m, ref_mem), f"graph {k}"
        assert per[k]["modularity"] == ref_q


@pytest.mark.parametrize("pruning", [1, 0])
def test_batch_fast_mode_valid_and_close(L, pruning):
    """Fast mode on graphs that fit in flight (a batch: its mean graph) runs the colour-synchronous
    schedule, so every graph of the batch reaches the oracle's modularity within 0.005 -- here
    exactly, since that is the oracle's schedule."""
    graphs = [gg.batch_sbm(4, k, n_lo=1000.0, n_hi=20000.0) for k in range(16)] + [gg.rmat(12, seed=3)]
    vo, o, t, w = upload(graphs)
    mem, per, _ = L.run_batch(vo, o, t, w, mode="fast", pruning=pruning, validate=0)
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        nc = per[k]["n_communities"]
        assert m.min() == 0 and m.max() == nc - 1 and len(np.unique(m)) == nc, f"graph {k}"
        q = oracle.modularity(g.offsets, g.targets, g.weights, m)
        assert abs(q - per[k]["modularity"]) <= 1e-12
        _, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(pruning=pruning))
        assert q >= ref_q - 0.005, f"graph {k}"


def test_batch_fast_mode_asynchronous_waves(L):
    """fast_sync_small = 1 keeps the asynchronous random-class schedule on small graphs: valid
    partitions, modularity within 0.005 of the oracle on the batch mean (one graph's result is a
    sample of a random schedule: 2-3% of small graphs land 0.03-0.066 below the oracle)."""
    graphs = [gg.batch_sbm(4, k, n_lo=1000.0, n_hi=20000.0) for k in range(16)]
    vo, o, t, w = upload(graphs)
    mem, per, _ = L.run_batch(vo, o, t, w, mode="fast", fast_sync_small=1, validate=0)
    qs, refs = [], []
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        nc = per[k]["n_communities"]
        assert m.min() == 0 and m.max() == nc - 1 and len(np.unique(m)) == nc, f"graph {k}"
        qs.append(oracle.modularity(g.offsets, g.targets, g.weights, m))
        refs.append(oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())[1])
    assert np.mean(qs) >= np.mean(refs) - 0.005


def test_batch_fp32(L):
    graphs = [gg.rmat(11, weights=gg.W_FP32, seed=k) for k in range(4)]
    vo, o, t, w = upload(graphs)
    mem, per, _ = L.run_batch(vo, o, t, w, mode="deterministic")
    for k, (g, m) in enumerate(zip(graphs, split(mem, vo))):
        assert abs(oracle.modularity(g.offsets, g.targets, g.weights, m) - per[k]["modularity"]) <= 1e-10
        _, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
        assert abs(per[k]["modularity"] - ref_q) <= 1e-4


def test_batch_max_passes_zero_gives_local_singletons(L):
    graphs = [gg.sbm(100, 4, 0.3, 0.01, 1), gg.sbm(50, 2, 0.3, 0.01, 2)]
    vo, o, t, w = upload(graphs)
    mem, per, _ = L.run_batch(vo, o, t, w, max_passes=0)
    for k, m in enumerate(split(mem, vo)):
        assert np.array_equal(m, np.arange(len(m)))
        assert per[k]["passes"] == 0 and per[k]["n_communities"] == len(m)


def test_batch_rejects_bad_input(L):
    import paper_2312_04876_gb300 as lv
    graphs = [gg.sbm(100, 4, 0.3, 0.01, 1), gg.sbm(50, 2, 0.3, 0.01, 2)]
    vo, o, t, w = upload(graphs)
    t_bad = t.clone()
    t_bad[-1] = 50  # graph 1 has local ids 0..49
    with pytest.raises(lv.LouvainError):
        L.run_batch(vo, o, t_bad, w)
    with pytest.raises(lv.LouvainError):
        L.run_batch([0, 120, 150], o, t, w)  # ranges that cut rows apart (asymmetric union)
    with pytest.raises(lv.LouvainError):
        L.run_batch([1, 100, 150], o, t, w)
    # the handle still works afterwards
    mem, per, _ = L.run_batch(vo, o, t, w)
    assert per[0]["n_communities"] >= 1
