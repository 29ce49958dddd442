"""Dynamic graphs through the C ABI: louvain_update_graph (a batch of edge deletions and insertions)
against the oracle's update, and louvain_run_from (a warm start from a given membership) against
the oracle's warm start -- bit-exact in deterministic integer mode."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import canonical, cliques, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def L(cuda_ok):
    import paper_2312_04876_gb300 as lv
    h = lv.Louvain(0)
    yield h
    h.close()


def dev(*arrays):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrays)


def rows(offs, tg, w):
    """Each row as a sorted list of (target, weight): the order of inserted arcs is unspecified."""
    return [sorted(zip(tg[offs[r]:offs[r + 1]].tolist(), w[offs[r]:offs[r + 1]].tolist()))
            for r in range(len(offs) - 1)]


def random_update(g, rng, n_new, n_del, n_ins):
    edges = [(u, int(v)) for u in range(g.n) for v in g.targets[g.offsets[u]:g.offsets[u + 1]] if u <= v]
    pick = rng.choice(len(edges), size=min(n_del, len(edges)), replace=False) if edges else []
    dels = [edges[k] for k in pick] + [(0, n_new - 1)]
    ins = [(int(rng.integers(0, n_new)), int(rng.integers(0, n_new))) for _ in range(n_ins)]
    if edges:
        ins.append(edges[0])
    ins.append((1, 1))
    iw = rng.integers(1, 9, size=len(ins)).astype(np.int32)
    return np.array(dels, dtype=np.int32).reshape(-1, 2), np.array(ins, dtype=np.int32).reshape(-1, 2), iw


@pytest.mark.parametrize("name", ["small", "loops", "rmat14", "empty_batch", "delete_only", "grow"])
def test_update_graph_matches_oracle(L, name):
    rng = np.random.default_rng(7)
    if name == "rmat14":
        g = gg.rmat(14, weights=gg.W_INT8, seed=5)
    elif name == "loops":
        g = random_graph(200, 0.05, rng, self_loops=True)
    else:
        g = random_graph(60, 0.1, rng)
    n_new = g.n + (25 if name == "grow" else 0)
    m = g.n_arcs // 2
    dels, ins, iw = random_update(g, rng, n_new, max(1, m // 50), max(1, m // 50))
    if name == "empty_batch":
        dels, ins, iw = dels[:0], ins[:0], iw[:0]
    if name == "delete_only":
        ins, iw = ins[:0], iw[:0]
    ref = oracle.update_graph(g.offsets, g.targets, g.weights, n_new, dels, ins, iw)
    o, t, w = dev(g.offsets, g.targets, g.weights)
    oo, ot, ow = L.update_graph(o, t, w, n_new, torch.from_numpy(dels), torch.from_numpy(ins), torch.from_numpy(iw))
    oo, ot, ow = oo.cpu().numpy(), ot.cpu().numpy(), ow.cpu().numpy()
    assert np.array_equal(oo, ref[0])
    assert rows(oo, ot, ow) == rows(*ref)
    # each row holds its surviving arcs first, then the inserted ones
    added = np.zeros(n_new, dtype=np.int64)
    for u, v in ins:
        added[u] += 1
        if u != v:
            added[v] += 1
    for r in range(n_new):
        k = int(ref[0][r + 1] - ref[0][r] - added[r])
        got = sorted(zip(ot[oo[r]:oo[r] + k].tolist(), ow[oo[r]:oo[r] + k].tolist()))
        want = sorted(zip(ref[1][ref[0][r]:ref[0][r] + k].tolist(), ref[2][ref[0][r]:ref[0][r] + k].tolist()))
        assert got == want, r


def test_update_graph_rejects_bad_ids_and_small_output(L):
    import paper_2312_04876_gb300 as lv
    g = random_graph(30, 0.2, np.random.default_rng(3))
    o, t, w = dev(g.offsets, g.targets, g.weights)
    with pytest.raises(lv.LouvainError):
        L.update_graph(o, t, w, g.n, torch.zeros((0, 2), dtype=torch.int32),
                       torch.tensor([[0, g.n]], dtype=torch.int32), torch.ones(1, dtype=torch.int32))
    # an output too small for the result is refused and the needed count reported
    import ctypes
    oo = torch.empty(g.n + 1, dtype=torch.int64, device=DEV)
    ot = torch.empty(4, dtype=torch.int32, device=DEV)
    ow = torch.empty(4, dtype=torch.int32, device=DEV)
    na = ctypes.c_int64()
    rc = L._lib.louvain_update_graph(L._h, g.n, g.n_arcs, o.data_ptr(), t.data_ptr(), w.data_ptr(), 0, g.n, 0, None,
                                     None, 0, None, None, None, None, oo.data_ptr(), ot.data_ptr(), ow.data_ptr(), 4,
                                     ctypes.byref(na))
    assert rc == 1 and na.value == g.n_arcs
    # the handle still works
    oo2, _, _ = L.update_graph(o, t, w, g.n, torch.zeros((0, 2), dtype=torch.int32),
                               torch.zeros((0, 2), dtype=torch.int32), torch.zeros(0, dtype=torch.int32))
    assert np.array_equal(oo2.cpu().numpy(), g.offsets)


@pytest.mark.parametrize("name", ["sbm3k_updated", "rmat14_updated", "random_init", "grown"])
def test_warm_start_deterministic_bit_exact(L, name):
    """Warm start after a batch update (the previous result as the initial membership, new vertices
    as singletons), and from an arbitrary membership: identical to the oracle's warm start."""
    rng = np.random.default_rng(11)
    g = gg.sbm(3000, 30, 0.1, 0.001, 8) if name != "rmat14_updated" else gg.rmat(14, weights=gg.W_INT8, seed=5)
    o, t, w = dev(g.offsets, g.targets, g.weights)
    prev, _ = L.run(o, t, w, mode="deterministic")
    prev = prev.cpu().numpy()
    n_new = g.n + (40 if name == "grown" else 0)
    m = g.n_arcs // 2
    dels, ins, iw = random_update(g, rng, n_new, m // 100, m // 100)
    oo, ot, ow = L.update_graph(o, t, w, n_new, torch.from_numpy(dels), torch.from_numpy(ins), torch.from_numpy(iw))
    init = np.concatenate([prev, np.arange(g.n, n_new)]).astype(np.int32)
    if name == "random_init":
        init = rng.integers(0, 50, size=n_new).astype(np.int32)
    mem, res = L.run_from(oo, ot, ow, torch.from_numpy(init).to(DEV), mode="deterministic", seed=3)
    ref_mem, ref_q, ref_passes, ref_stats = oracle.louvain_from(oo.cpu().numpy(), ot.cpu().numpy(), ow.cpu().numpy(),
                                                                init, oracle.default_params(seed=3))
    assert np.array_equal(mem.cpu().numpy(), ref_mem)
    assert res.modularity == ref_q and res.passes == ref_passes
    assert [s["iterations"] for s in res.stats] == [s["iterations"] for s in ref_stats]


def test_warm_start_fixed_point_and_invalid_init(L):
    import paper_2312_04876_gb300 as lv
    k, s = 6, 5
    g = cliques(k, s, ring=True)
    o, t, w = dev(g.offsets, g.targets, g.weights)
    init = np.repeat(np.arange(k) * 3 + 2, s).astype(np.int32)
    mem, res = L.run_from(o, t, w, torch.from_numpy(init).to(DEV), mode="deterministic")
    assert mem.cpu().tolist() == canonical(init).tolist() and res.passes == 1 and res.total_iterations == 1
    bad = torch.from_numpy(init).to(DEV)
    bad[3] = g.n
    with pytest.raises(lv.LouvainError):
        L.run_from(o, t, w, bad, mode="deterministic")


def test_warm_start_fast_mode_quality(L):
    """Fast mode from the previous result after a 1% update: a valid partition whose modularity is
    within 0.005 of the oracle's warm start (or above it)."""
    rng = np.random.default_rng(5)
    g = gg.rmat(16, weights=gg.W_INT8, seed=22)
    o, t, w = dev(g.offsets, g.targets, g.weights)
    prev, _ = L.run(o, t, w, mode="fast")
    m = g.n_arcs // 2
    dels, ins, iw = random_update(g, rng, g.n, m // 100, m // 100)
    oo, ot, ow = L.update_graph(o, t, w, g.n, torch.from_numpy(dels), torch.from_numpy(ins), torch.from_numpy(iw))
    mem, res = L.run_from(oo, ot, ow, prev, mode="fast", validate=1)
    mm = mem.cpu().numpy()
    assert mm.min() == 0 and mm.max() == res.n_communities - 1 and len(np.unique(mm)) == res.n_communities
    _, ref_q, _, _ = oracle.louvain_from(oo.cpu().numpy(), ot.cpu().numpy(), ow.cpu().numpy(), prev.cpu().numpy())
    assert res.modularity >= ref_q - 0.005
