"""Fast mode's schedule choice (reading R12): an input graph that fits what the GPU holds in flight
and is not carried by hubs runs the colour-synchronous schedule of the deterministic mode in every
pass -- the oracle's own schedule, so the result is the oracle's -- while a graph larger than that,
or one whose rows of more than 512 arcs carry over a fifth of its arcs, keeps the asynchronous
random classes in every pass.  The per-pass statistics show which ran (colours > 0: classes came
from the colouring)."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L(cuda_ok):
    import paper_2312_04876_gb300 as lv
    h = lv.Louvain(0)
    yield h
    h.close()


def dev(g):
    d = torch.device("cuda:0")
    return tuple(torch.from_numpy(a).to(d) for a in (g.offsets, g.targets, g.weights))


def hub_share(g):
    d = np.diff(g.offsets)
    return d[d > 512].sum() / max(1, d.sum())


@pytest.mark.parametrize("name", ["sbm2k", "sbm10k", "rmat12"])
def test_small_graph_runs_the_oracles_schedule(L, name):
    g = {"sbm2k": lambda: gg.sbm(2000, 20, 0.1, 0.002, 7),
         "sbm10k": lambda: gg.sbm(10000, 100, 0.1, 0.0005, 1),
         "rmat12": lambda: gg.rmat(12, weights=gg.W_INT8, seed=3)}[name]()
    assert hub_share(g) <= 0.2
    mem, r = L.run(*dev(g), mode="fast", validate=0)
    assert all(s["colours"] > 0 for s in r.stats)  # every pass coloured: colour-synchronous
    ref_mem, ref_q, ref_passes, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
    assert np.array_equal(mem.cpu().numpy(), ref_mem) and r.modularity == ref_q and r.passes == ref_passes


def test_hub_carried_small_graph_stays_asynchronous(L):
    g = gg.rmat(14, weights=gg.W_INT8, seed=22)
    assert g.n <= torch.cuda.get_device_properties(0).multi_processor_count * 1024 and hub_share(g) > 0.2
    mem, r = L.run(*dev(g), mode="fast", validate=0)
    assert all(s["colours"] == 0 for s in r.stats)  # random classes in every pass
    # and fast_sync_small = 2 forces the colour-synchronous schedule on it: the oracle's result
    mem2, r2 = L.run(*dev(g), mode="fast", validate=0, fast_sync_small=2)
    assert all(s["colours"] > 0 for s in r2.stats)
    ref_mem, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
    assert np.array_equal(mem2.cpu().numpy(), ref_mem) and r2.modularity == ref_q


def test_large_graph_is_asynchronous_in_every_pass(L):
    """R-MAT 18 (262k vertices) is larger than the window: its late super-vertex graphs are small,
    but the first phase's choice holds for the whole call."""
    g = gg.rmat(18, weights=gg.W_INT8, seed=22)
    assert g.n > torch.cuda.get_device_properties(0).multi_processor_count * 1024
    _, r = L.run(*dev(g), mode="fast", validate=0)
    assert r.passes >= 2 and all(s["colours"] == 0 for s in r.stats)
    # fast_sync_small = 1 keeps random classes on small graphs too
    _, r1 = L.run(*dev(gg.sbm(2000, 20, 0.1, 0.002, 7)), mode="fast", validate=0, fast_sync_small=1)
    assert all(s["colours"] == 0 for s in r1.stats)
